"""GPU parity of the tensor-core grid adjoint against the FP64 oracle.

On a Cartesian grid handed over x-fastest the adjoint's per-mode sums
(derivative of Eq. DiscreteFT, Sec. 4.1) factorise: the x cells are a matrix
product on the tensor cores, the y and z phasors are contracted per mode on
the CUDA cores.  These tests compare every gradient family with the oracle's
on ragged shapes (x chunks, y blocks and z patches that do not fill), 2-D and
3-D grids, several mode tiles, rotated and periodic anisotropy, non-uniform
axes far from the origin, and check the power-of-two scaling of g, the unit
counter, determinism and the agreement with the CUDA-core adjoint.
"""
import math

import numpy as np
import pytest

from helpers import FAMILY_IDS, GRAD_TOL, gpu_env, to_dev

pytestmark = pytest.mark.gpu

FAMILIES_OUT = ("dA", "dpsi", "da", "dmu", "dsigma", "dsigma2", "dell", "drot", "drho", "dkappa")


@pytest.fixture(scope="module")
def env():
    torch = gpu_env()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    yield torch, F, W
    F.grid_path(True)


def _check(got, ref, name):
    got = np.asarray(got, dtype=np.float64).reshape(np.shape(ref))
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(got - ref))
    assert err <= GRAD_TOL * scale, "%s: max err %.3e vs scale %.3e" % (name, err, scale)
    return err / scale if scale > 0 else 0.0


def _oracle_reparam(family, sigma2, ell, dim, n_modes, seed, cells, g, rot=None, period=None):
    from oracle import field as of
    from oracle import modes as omod
    from oracle import native
    ell3 = list(ell) + [1.0] * (3 - len(ell))
    om = omod.gen_modes(FAMILY_IDS[family], sigma2, ell3, dim, n_modes, seed, nu=1.5, rot=rot, period=period)
    c = np.stack(cells, axis=-1)
    return of.grads_reparam(*native.mode_sums(om["a"], om["psi"], c, g.astype(np.float64)), om["kappa"], om["rho"],
                            math.sqrt(sigma2), ell, g.astype(np.float64), rot=rot, period=period)


def _grid_backward(env, p, cells, g, mode="always"):
    torch, F, W = env
    plan = F.CellPlan(*to_dev(torch, cells))
    gf = F.GaussianField(p)
    F.grid_path(mode)
    try:
        F.take_grid_adjoint_units()
        gr = F.backward(gf.table, p, plan, torch.from_numpy(g).cuda())
        torch.cuda.synchronize()
        units = F.take_grid_adjoint_units()
    finally:
        F.grid_path(True)
    assert plan.status() == 0
    return {k: v.cpu().numpy() for k, v in gr.items()}, units, plan


@pytest.mark.parametrize("shape,family,n_modes,transform", [
    ((24, 20, 18), "gaussian", 600, None),
    ((70, 33, 17), "exponential", 777, "rotation"),
    ((130, 9, 5), "matern", 500, None),
    ((48, 40, 36), "gaussian", 3000, "general"),
    ((90, 70), "exponential", 640, None),
    ((300, 41), "gaussian", 1000, "rotation"),
])
def test_grid_adjoint_against_oracle(env, shape, family, n_modes, transform):
    torch, F, W = env
    dim = len(shape)
    cells = W.grid_centres(shape)
    ell = (0.2, 0.11, 0.07)[:dim]
    R = None
    if transform == "rotation":
        a_ = 0.4
        R = np.eye(3)
        R[:2, :2] = [[math.cos(a_), -math.sin(a_)], [math.sin(a_), math.cos(a_)]]
    elif transform == "general":
        R = np.array([[1.1, 0.5, 0.0], [0.0, 0.8, 0.3], [0.2, 0.0, 1.3]])
    Rd = None if R is None else R[:dim, :dim]
    p = F.FieldParams(family=family, sigma2=1.3, mean=0.05, ell=ell, dim=dim, n_modes=n_modes, seed=61, nu=1.5,
                      rot=None if Rd is None else Rd.tolist())
    g = np.random.default_rng(7).standard_normal(len(cells[0])).astype(np.float32)
    gr, units, _ = _grid_backward(env, p, cells, g)
    assert units > 0
    ref = _oracle_reparam(family, 1.3, ell, dim, n_modes, 61, cells, g, rot=Rd)
    errs = {k: _check(gr[k], ref[k], k) for k in FAMILIES_OUT}
    print(shape, family, transform, "grid adjoint errors:", errs)


def test_grid_adjoint_periodic(env):
    # periodic axes: frequencies rounded to multiples of 1/L, whose dL/da
    # reaches neither kappa, l nor R (Appendix B reading of the library)
    torch, F, W = env
    cells = W.grid_centres((80, 48, 20))
    ell = (0.15, 0.1, 0.08)
    period = (1.0, 1.0, 0.0)
    p = F.FieldParams(family="gaussian", sigma2=0.8, ell=ell, dim=3, n_modes=900, seed=13, period=period)
    g = np.random.default_rng(3).standard_normal(len(cells[0])).astype(np.float32)
    gr, units, _ = _grid_backward(env, p, cells, g)
    assert units > 0
    ref = _oracle_reparam("gaussian", 0.8, ell, 3, 900, 13, cells, g, period=period)
    for k in FAMILIES_OUT:
        _check(gr[k], ref[k], k)


def test_grid_adjoint_rectilinear_far_from_origin(env):
    # non-uniform axes far from the origin: the x weights are taken relative
    # to the first x cell and the y, z weights likewise, then shifted back
    torch, F, W = env
    rng = np.random.default_rng(8)
    ax = [np.float32(1000.0) + np.cumsum(rng.uniform(0.002, 0.02, n)).astype(np.float32) for n in (150, 33, 9)]
    mesh = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    cells = [np.ascontiguousarray(m.ravel()) for m in mesh[::-1]]
    ell = (0.1, 0.08, 0.05)
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=ell, dim=3, n_modes=700, seed=31)
    g = np.random.default_rng(9).standard_normal(len(cells[0])).astype(np.float32)
    gr, units, plan = _grid_backward(env, p, cells, g)
    assert plan.grid_shape() == (150, 33, 9) and units > 0
    ref = _oracle_reparam("gaussian", 1.0, ell, 3, 700, 31, cells, g)
    for k in FAMILIES_OUT:
        _check(gr[k], ref[k], k)


def test_grid_adjoint_power_of_two_scaling_is_exact(env):
    # g is brought below 1 by a power of two before the FP16 split, so g 2^-90
    # and g 2^60 give the FP16 operands of g itself: every gradient scales
    # exactly; g = 0 gives zeros
    torch, F, W = env
    cells = W.grid_centres((64, 40, 24))
    p = F.FieldParams(family="exponential", sigma2=2.0, ell=(0.2, 0.1, 0.1), dim=3, n_modes=512, seed=4)
    g = np.random.default_rng(5).standard_normal(len(cells[0])).astype(np.float32)
    base, _, _ = _grid_backward(env, p, cells, g)
    for e in (-90, 60):
        sc, _, _ = _grid_backward(env, p, cells, (g * np.float32(2.0 ** e)).astype(np.float32))
        for k in FAMILIES_OUT:
            assert np.array_equal(sc[k], base[k] * 2.0 ** e), (e, k)
    zero, _, _ = _grid_backward(env, p, cells, np.zeros_like(g))
    for k in FAMILIES_OUT:
        assert not np.any(zero[k]), k


def test_grid_adjoint_units_and_determinism(env):
    torch, F, W = env
    shape = (100, 70, 20)
    cells = W.grid_centres(shape)
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1, 0.1), dim=3, n_modes=1000, seed=2)
    g = np.random.default_rng(1).standard_normal(len(cells[0])).astype(np.float32)
    a, units_a, _ = _grid_backward(env, p, cells, g)
    b, units_b, _ = _grid_backward(env, p, cells, g)
    for k in FAMILIES_OUT:
        assert np.array_equal(a[k], b[k]), k
    # units: mode tiles (1000 modes -> 1024 slots: 8) x x chunks (100 -> 2) x
    # patches; the 70 x 20 (y, z) cells waste the fewest columns in patches of
    # 16 x 4 cells (80 x 20 columns: 5 y blocks x 5 z blocks)
    assert units_a == units_b == 8 * 2 * 5 * 5
    _, units_off, _ = _grid_backward(env, p, cells, g, mode=False)
    assert units_off == 0


def test_grid_adjoint_matches_cuda_core_adjoint(env):
    torch, F, W = env
    cells = W.grid_centres((128, 64, 40))
    p = F.FieldParams(family="matern", sigma2=1.5, ell=(0.15, 0.1, 0.07), dim=3, n_modes=1024, seed=21, nu=1.5)
    g = np.random.default_rng(2).standard_normal(len(cells[0])).astype(np.float32)
    on, units, _ = _grid_backward(env, p, cells, g)
    off, units_off, _ = _grid_backward(env, p, cells, g, mode=False)
    assert units > 0 and units_off == 0
    errs = {k: _check(on[k], off[k], k) for k in FAMILIES_OUT}
    print("grid vs CUDA-core adjoint:", errs)


def test_auto_setting_uses_grid_adjoint(env):
    # the default setting takes the grid adjoint for every grid plan, as the
    # forward
    torch, F, W = env
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=256, seed=3)
    for shape in ((64, 64), (896, 128), (1024, 128)):
        cells = W.grid_centres(shape)
        g = np.random.default_rng(4).standard_normal(len(cells[0])).astype(np.float32)
        gr, units, _ = _grid_backward(env, p, cells, g, mode=True)
        assert units > 0, shape
        ref = _oracle_reparam("gaussian", 1.0, (0.1, 0.1), 2, 256, 3, cells, g)
        for k in ("dA", "dpsi", "da", "dmu", "dsigma", "dell"):
            _check(gr[k], ref[k], k)


@pytest.mark.slow
def test_grid_adjoint_256_cube_matches_cuda_core(env):
    # the full 256^3 cube (4 x chunks, 4 y blocks, 256 z cells per mode tile,
    # a 134 MB B table): every gradient family of the grid adjoint against the
    # CUDA-core adjoint on the same g
    torch, F, W = env
    cells = W.workload_cells("grid3d_256")
    p = F.FieldParams(family="exponential", sigma2=4.0, ell=(0.2, 0.2, 0.05), dim=3, n_modes=1024, seed=3)
    g = np.random.default_rng(6).standard_normal(len(cells[0])).astype(np.float32)
    on, units, plan = _grid_backward(env, p, cells, g)
    assert plan.grid_shape() == (256, 256, 256) and units == 8 * 4 * 4 * 256
    off, units_off, _ = _grid_backward(env, p, cells, g, mode=False)
    assert units_off == 0
    errs = {k: _check(on[k], off[k], k) for k in FAMILIES_OUT}
    print("256^3 grid vs CUDA-core adjoint:", errs)
