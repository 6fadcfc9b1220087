"""Pins of the oracle's counter-based generator (no GPU).

The generator's definition is the published Philox4x32-10; its known-answer
vectors (tests/golden/philox4x32_10_kat.txt) fix every round constant, the
round function and the key schedule.  The uniform and normal conversions are
pinned by exact values and by distribution tests.
"""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answer_vectors(golden_dir):
    rows = _kat(golden_dir)
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = philox.philox4x32_10(np.array(ctr), np.array(key))
        assert [int(w) for w in got] == want


def test_kat_vectorised_matches_scalar(golden_dir):
    rows = _kat(golden_dir)
    ctr = np.array([r[0] for r in rows])
    key = np.array([r[1] for r in rows])
    got = philox.philox4x32_10(ctr, key)
    assert [[int(w) for w in g] for g in got] == [r[2] for r in rows]


def test_uniform_conversion_exact_values():
    w = np.array([[0, 0, 0xFFFFFFFF, 0xFFFFFFFF], [0x00001000, 0, 0, 0x80000000]], dtype=np.uint64)
    u = philox.words_to_uniforms(w)
    assert u[0, 0] == 0.5 * 2.0 ** -52
    assert u[0, 1] == 1.0 - 2.0 ** -53
    assert u[1, 0] == 1.5 * 2.0 ** -52
    assert u[1, 1] == 0.5 + 0.5 * 2.0 ** -52


def test_stream_layout():
    # counter = (j lo, block, stream, j hi); key = (seed lo, seed hi)
    seed = (7 << 32) | 11
    j = (3 << 32) | 5
    got = philox.block(seed, 9, j, 2)
    want = philox.philox4x32_10(np.array([5, 2, 9, 3]), np.array([11, 7]))
    assert np.array_equal(got, want)


def test_uniforms_distribution():
    u = philox.uniforms(1234, 0, np.arange(100000), 0).ravel()
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_normals_distribution_and_independence():
    j = np.arange(60000)
    n0 = philox.normal(99, 0, j, 0)
    n1 = philox.normal(99, 0, j, 1)
    n2 = philox.normal(99, 0, j, 2)
    for n in (n0, n1, n2):
        assert stats.kstest(n, "norm").pvalue > 1e-3
    for x, y in ((n0, n1), (n0, n2), (n1, n2)):
        r = np.corrcoef(x, y)[0, 1]
        assert abs(r) < 5.0 / np.sqrt(len(j))


def test_box_muller_closed_form():
    # u0 = exp(-1/2) gives radius 1; u1 = 1/8 gives angle pi/4
    n0, n1 = philox.box_muller(np.exp(-0.5), 0.125)
    assert n0 == pytest.approx(np.sqrt(0.5), abs=1e-15)
    assert n1 == pytest.approx(np.sqrt(0.5), abs=1e-15)
