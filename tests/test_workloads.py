"""The seeded synthetic inputs (the recipe of the benchmark and the parity
tests) have the sizes and structure the documentation states: the 256^3 and
64^2 grids, the jittered 2M-cell lattice, the HRL-shaped grid and the
256-realisation ensemble (totals, shapes, mode counts, determinism)."""
import math

import numpy as np

from paper_2212_10961_gb300 import workloads as W


def test_grids_are_cell_centres_x_fastest():
    x, y = W.grid_centres((4, 3))
    assert np.array_equal(x[:4], np.array([0.125, 0.375, 0.625, 0.875], dtype=np.float32))
    assert np.all(y[:4] == np.float32(1.0 / 6.0))
    cells = W.workload_cells("grid3d_256")
    assert len(cells) == 3 and len(cells[0]) == 256 ** 3
    assert cells[0].dtype == np.float32 and float(cells[0].max()) == (255.5 / 256)


def test_jittered_lattice_recipe():
    w = W.WORKLOADS["jitter3d_2m"]
    cells = W.workload_cells("jitter3d_2m")
    n = 252 * 126 * 63
    assert len(cells[0]) == n == 2000376
    h = w["h"]
    base = W.grid_centres(w["shape"], tuple(s * h for s in w["shape"]))
    for c, b in zip(cells, base):
        d = c.astype(np.float64) - b.astype(np.float64)
        assert np.max(np.abs(d)) <= 0.4 * h * (1 + 1e-6)
        assert np.std(d) > 0.2 * h  # uniform on (-0.4 h, 0.4 h): std 0.23 h
    again = W.workload_cells("jitter3d_2m")
    assert all(np.array_equal(a, b) for a, b in zip(cells, again))  # seeded


def test_hrl2d_recipe():
    w = W.WORKLOADS["hrl2d"]
    x, y = W.workload_cells("hrl2d")
    assert len(x) == 1024 * 512 and float(x.max()) < 2.0 and float(y.max()) < 1.0
    assert w["ell"] == (0.2, 0.05) and w["sigma2"] == 2.0 and w["n_modes"] == 4096
    assert list(w["values"]) == sorted(w["values"]) and len(w["values"]) == len(w["quantiles"]) + 1


def test_ensemble_recipe_totals():
    r = W.ensemble_recipe()
    assert len(r) == 256
    cells = sum(int(np.prod(e["shape"])) for e in r)
    cm = sum(int(np.prod(e["shape"])) * e["n_modes"] for e in r)
    assert cells == 19960894
    assert math.isclose(cm, 5.1955861504e10, rel_tol=1e-9)
    assert {e["n_modes"] for e in r} <= {1024, 2048, 4096}
    for e in r:
        assert e["shape"] == (64, 64, 64) or (len(e["shape"]) == 2 and 32 <= e["shape"][0] <= 512)
    assert r == W.ensemble_recipe()  # seeded
