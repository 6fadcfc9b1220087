"""The C ABI used from a plain C99 program (tests/c/grf_c_example.c) built
with gcc against include/grf.h and the shared library: no C++, no Python
between the caller and the library.  Host entry points on the CPU; the
device path (plan, upload, synthesis, status) on the GPU, each checked
against the FP64 oracle."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import field as ofield
from oracle import modes as omodes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NM, NX, NY = 257, 40, 30


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import __graft_entry__
    __graft_entry__.build()
    pkg = os.path.join(ROOT, "paper_2212_10961_gb300")
    exe = str(tmp_path_factory.mktemp("cabi") / "grf_c_example")
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c", "grf_c_example.c"),
           "-o", exe, "-L", pkg, "-lgrf", "-Wl,-rpath," + pkg, "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _run(program, mode, out_dir):
    r = subprocess.run([program, mode, str(out_dir)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def _oracle_modes():
    return omodes.gen_modes(omodes.GAUSSIAN, 1.5, (0.15, 0.1), 2, NM, 99)


def test_c_client_draws_the_oracle_modes(program, tmp_path):
    out = _run(program, "host", tmp_path)
    assert "bad sigma2 -> -1" in out and "host ok" in out
    buf = np.fromfile(tmp_path / "modes.bin", dtype=np.float64)
    a, amp, psi = buf[:2 * NM].reshape(NM, 2), buf[2 * NM:3 * NM], buf[3 * NM:]
    om = _oracle_modes()
    np.testing.assert_allclose(a, om["a"], rtol=4e-15, atol=1e-300)
    np.testing.assert_allclose(amp, om["amp"], rtol=4e-15, atol=1e-300)
    np.testing.assert_allclose(psi, om["psi"], rtol=4e-15, atol=1e-300)


@pytest.mark.gpu
def test_c_client_synthesises_on_the_device(program, tmp_path):
    out = _run(program, "gpu", tmp_path)
    assert "gpu ok" in out
    Y = np.fromfile(tmp_path / "Y.bin", dtype=np.float32).astype(np.float64)
    K = np.fromfile(tmp_path / "K.bin", dtype=np.float32).astype(np.float64)
    fac = np.fromfile(tmp_path / "facies.bin", dtype=np.uint8)
    ii, jj = np.meshgrid(np.arange(NX), np.arange(NY))
    cells = np.stack([((ii + 0.5) / NX).ravel().astype(np.float32), ((jj + 0.5) / NY).ravel().astype(np.float32)],
                     axis=-1).astype(np.float64)
    om = _oracle_modes()
    y_or = ofield.synth(om["a"], om["amp"], om["psi"], 0.25, cells)
    sig = math.sqrt(1.5)
    assert np.max(np.abs(Y - y_or)) <= 1e-5 * sig
    assert np.max(np.abs(K - np.exp(y_or)) / np.exp(y_or)) <= 1e-5 * sig + 2.0 ** -21
    lab = ofield.indicator(y_or, [0.25])
    band = np.abs(y_or - 0.25) <= 2e-5 * sig
    assert np.array_equal(fac[~band], lab[~band])
