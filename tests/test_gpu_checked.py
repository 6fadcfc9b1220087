"""The checked library (libgrf_checked.so: the same kernels with device-side
index checks, the stand-in for a memory sanitizer) on the GPU.

Each case runs in a child process with GRF_LIBRARY=checked, because a
process loads one flavour of the library.  (1) On valid inputs the checked
kernels give the oracle's results and skip nothing.  (2) A plan whose
permutation holds one index out of range is caught: the checked forward and
adjoint skip that cell's accesses (one store in the forward, one gradient
read per warp of modes in the adjoint), count them, and every other cell is
still right.  Case (2) corrupts the plan only after the child has confirmed
that the checked flavour is loaded; the release library is never given it.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, math, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
from helpers import check_forward, oracle_field, oracle_modes, GRAD_TOL
from oracle import field as of
from oracle import native
from paper_2212_10961_gb300 import _abi, field as F, workloads as W
import ctypes

L = _abi.lib()
assert L.grf_checked_build() == 1, "the checked library is not the one loaded"

def faults():
    c = ctypes.c_int64(-1)
    _abi.check(L.grf_take_index_faults(ctypes.byref(c)))
    return c.value

cells = W.jittered_lattice((37, 29, 23), 1.0 / 32, 0.3, seed=12)
n = len(cells[0])
dev = [torch.from_numpy(c).cuda() for c in cells]
sig2, ell, N = 1.7, (0.15, 0.25, 0.1), 700
p = F.FieldParams(family="matern", nu=1.5, sigma2=sig2, ell=ell, dim=3, n_modes=N, seed=8)
gf = F.GaussianField(p)
om = oracle_modes("matern", sig2, ell, 3, N, 8, nu=1.5)
y_or = oracle_field(om, 0.0, cells)
c3 = np.stack(cells, axis=-1)
g_host = np.random.default_rng(4).standard_normal(n).astype(np.float32) / n
res = {}

def grads(plan):
    g = F.backward(gf.table, p, plan, torch.from_numpy(g_host).cuda())
    return {k: g[k].cpu().numpy() for k in ("dA", "dpsi", "da")}

def oracle_grads(gv):
    s_cos, s_sin, s_sinx = native.mode_sums(om["a"], om["psi"], c3, gv.astype(np.float64))
    return of.grads_from_sums(s_cos, s_sin, s_sinx, om["amp"], om["a"], math.sqrt(sig2), ell, gv.astype(np.float64))

if MODE == "valid":
    faults()
    plan = F.CellPlan(*dev)
    y = gf.synth(plan, F.MapSpec(y=True))["Y"].cpu().numpy()
    check_forward(y, y_or, math.sqrt(sig2), "checked forward")
    got, want = grads(plan), oracle_grads(g_host)
    for k in got:
        scale = np.max(np.abs(want[k]))
        assert np.max(np.abs(got[k].reshape(want[k].shape) - want[k])) <= GRAD_TOL * scale, k
    assert plan.status() == 0
    res["faults"] = faults()
else:
    plan = F.CellPlan(*dev)
    torch.cuda.synchronize()
    faults()
    # plan header: int64 byte offset of the permutation (int32 per sorted cell) at byte 56
    off_perm = int(plan.buf[56:64].cpu().numpy().view(np.int64)[0])
    perm = plan.buf[off_perm:off_perm + 4 * n].view(torch.int32)
    k_bad = 1234
    victim = int(perm[k_bad].item())
    perm[k_bad] = n + 4321
    out = {"Y": torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")}
    F.synth(gf.table, p, plan, 0, F.MapSpec(y=True), out)
    y = out["Y"].cpu().numpy()
    res["faults_forward"] = faults()
    assert math.isnan(y[victim]), "the skipped cell was written"
    keep = np.arange(n) != victim
    check_forward(y[keep], y_or[keep], math.sqrt(sig2), "other cells")
    got = grads(plan)
    res["faults_adjoint"] = faults()
    gz = g_host.copy()
    gz[victim] = 0.0  # the checked adjoint reads g = 0 for the skipped cell
    want = oracle_grads(gz)
    for k in got:
        scale = np.max(np.abs(want[k]))
        assert np.max(np.abs(got[k].reshape(want[k].shape) - want[k])) <= GRAD_TOL * scale, k
print("RESULT " + json.dumps(res))
'''


def _run(mode):
    env = dict(os.environ, GRF_LIBRARY="checked")
    code = "ROOT = %r\nMODE = %r\n" % (ROOT, mode) + CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_checked_library_matches_oracle_and_skips_nothing():
    import __graft_entry__
    __graft_entry__.build()
    res = _run("valid")
    assert res["faults"] == 0


def test_checked_library_catches_a_corrupted_permutation():
    import __graft_entry__
    __graft_entry__.build()
    res = _run("corrupt")
    assert res["faults_forward"] == 1  # the one store of the victim cell
    # the adjoint reads the cell's gradient once per warp of 128 modes (N = 700)
    assert res["faults_adjoint"] == -(-700 // 128)
