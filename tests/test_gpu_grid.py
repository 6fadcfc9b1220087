"""GPU parity of the tensor-core Cartesian-grid path against the FP64 oracle.

Cells handed over x-fastest on the tensor product of three axes make the
spectral sum (Eq. DiscreteFT) a matrix product per block of 128 x-cells by
128 (y, z)-cells; the library detects such plans and evaluates them on the
tensor cores.  These tests check the MMA plumbing on exact integer products,
the detection, and the field and maps against the oracle on ragged shapes,
every fold interval, non-uniform axes and far-from-origin coordinates.
"""
import math

import numpy as np
import pytest

from helpers import check_facies, check_forward, check_lognormal, gpu_env, oracle_field, oracle_modes, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = gpu_env()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    yield torch, F, W
    F.grid_path(True)


def test_mma_selftest_exact_integers(env):
    # small integers: every product and partial sum is exact in FP32, so D
    # must equal the integer product whatever the accumulation order; random
    # entries catch any transposed, permuted or misplaced core matrix
    torch, F, W = env
    rng = np.random.default_rng(1)
    for k in (1, 3):
        A = rng.integers(-16, 17, size=(128, 64 * k))
        B = rng.integers(-16, 17, size=(128, 64 * k))
        D, st = F.mma_selftest(torch.tensor(A, dtype=torch.float16, device="cuda"),
                               torch.tensor(B, dtype=torch.float16, device="cuda"))
        torch.cuda.synchronize()
        assert st.item() == 0
        assert np.array_equal(D.cpu().numpy().astype(np.int64), A.astype(np.int64) @ B.T.astype(np.int64))


def test_mma_selftest_one_hot_layout(env):
    # A[r, k] = 1 only at k = (5 r) mod 64 + 64 (r mod 2): D[r, c] = B[c, that k]
    torch, F, W = env
    A = np.zeros((128, 128))
    kk = (5 * np.arange(128)) % 64 + 64 * (np.arange(128) % 2)
    A[np.arange(128), kk] = 1.0
    B = np.random.default_rng(2).integers(-1000, 1000, size=(128, 128))
    D, st = F.mma_selftest(torch.tensor(A, dtype=torch.float16, device="cuda"),
                           torch.tensor(B, dtype=torch.float16, device="cuda"))
    torch.cuda.synchronize()
    assert st.item() == 0
    assert np.array_equal(D.cpu().numpy(), B[:, kk].T.astype(np.float32))


def test_mma_selftest_accumulation_bound(env):
    # FP16 values in [-1, 1], K = 2048 in one FP32 accumulator: the error of
    # each entry stays within K ulps of the largest partial sum
    torch, F, W = env
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, size=(128, 2048)).astype(np.float16)
    B = rng.uniform(-1, 1, size=(128, 2048)).astype(np.float16)
    D, st = F.mma_selftest(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"))
    torch.cuda.synchronize()
    assert st.item() == 0
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    bound = 2048 * 2.0 ** -23 * np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    assert np.all(np.abs(D.cpu().numpy() - ref) <= bound)


def test_grid_detection(env):
    torch, F, W = env
    for shape, expect in (((40, 36, 30), (40, 36, 30)), ((90, 64), (90, 64, 1)), ((128, 2, 3), (128, 2, 3))):
        plan = F.CellPlan(*to_dev(torch, W.grid_centres(shape)))
        assert plan.grid_shape() == expect, shape
    cells = W.grid_centres((40, 36, 30))
    sh, _ = W.shuffled(cells, 5)
    assert F.CellPlan(*to_dev(torch, sh)).grid_shape() == (0, 0, 0)
    jit = W.jittered_lattice((20, 16, 12), 0.05, 0.3, 7)
    assert F.CellPlan(*to_dev(torch, jit)).grid_shape() == (0, 0, 0)
    # one cell moved by one ulp
    bad = [c.copy() for c in cells]
    bad[1][12345] = np.nextafter(bad[1][12345], np.float32(2.0))
    assert F.CellPlan(*to_dev(torch, bad)).grid_shape() == (0, 0, 0)
    # y-fastest order is not x-fastest
    yf = W.grid_centres((36, 40, 30))
    assert F.CellPlan(*to_dev(torch, [yf[1], yf[0], yf[2]])).grid_shape() == (0, 0, 0)
    # two segments: no grid path
    a = W.grid_centres((40, 30))
    two = [np.concatenate([u, u]) for u in a]
    assert F.CellPlan(*to_dev(torch, two), segments=[1200, 1200]).grid_shape() == (0, 0, 0)
    # a single row (ny = 1) is left to the general path
    row = [np.arange(300, dtype=np.float32) / 300, np.zeros(300, np.float32)]
    assert F.CellPlan(*to_dev(torch, row)).grid_shape() == (0, 0, 0)


def _grid_run(env, cells, family, sigma2, ell, n_modes, seed, mean, fold=4, thresholds=(0.0,)):
    torch, F, W = env
    d = len(cells)
    p = F.FieldParams(family=family, sigma2=sigma2, mean=mean, ell=ell, dim=d, n_modes=n_modes, seed=seed, nu=1.5)
    gf = F.GaussianField(p)
    plan = F.CellPlan(*to_dev(torch, cells))
    F.grid_path("always", fold)
    F.take_grid_tiles()
    F.take_path_counts()
    out = gf.synth(plan, F.MapSpec(y=True, lognormal=True, thresholds=thresholds, facies=True))
    torch.cuda.synchronize()
    assert plan.status() == 0
    tiles = F.take_grid_tiles()
    assert tiles > 0, "grid path not taken"
    assert F.take_path_counts() == (0, 0)
    F.grid_path(True)
    return {k: v.cpu().numpy() for k, v in out.items()}, p


@pytest.mark.parametrize("shape", [(128, 16, 8), (200, 24, 11), (257, 5, 3), (300, 70), (64, 48), (37, 130, 2)])
@pytest.mark.parametrize("fold", [1, 2, 4, 8])
def test_grid_path_against_oracle(env, shape, fold):
    torch, F, W = env
    cells = W.grid_centres(shape, extent=(2.0, 1.0, 0.5)[:len(shape)])
    d = len(shape)
    ell = (0.2, 0.1, 0.05)[:d]
    out, p = _grid_run(env, cells, "exponential", 2.0, ell, 300, 17, 0.3, fold=fold)
    y_or = oracle_field(oracle_modes("exponential", 2.0, ell, d, 300, 17), 0.3, cells)
    s = math.sqrt(2.0)
    check_forward(out["Y"], y_or, s, "grid %s fold %d" % (shape, fold))
    check_lognormal(out["K"], y_or, s)
    check_facies(out["facies"], y_or, (0.0,), s)


@pytest.mark.parametrize("family", ["gaussian", "matern"])
def test_grid_path_families_many_modes(env, family):
    torch, F, W = env
    cells = W.grid_centres((96, 40, 36))
    ell = (0.13, 0.1, 0.07)
    out, p = _grid_run(env, cells, family, 1.6, ell, 2500, 29, -0.2)
    y_or = oracle_field(oracle_modes(family, 1.6, ell, 3, 2500, 29), -0.2, cells)
    check_forward(out["Y"], y_or, math.sqrt(1.6), "grid %s" % family)


def test_grid_path_rectilinear_far_from_origin(env):
    # non-uniform axes (random spacing) far from the origin: each axis phase
    # is reduced exactly at its own coordinate, so the offset costs nothing
    torch, F, W = env
    rng = np.random.default_rng(8)
    ax = [np.float32(1000.0) + np.cumsum(rng.uniform(0.002, 0.02, n)).astype(np.float32) for n in (150, 33, 9)]
    mesh = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    cells = [np.ascontiguousarray(m.ravel()) for m in mesh[::-1]]
    plan = F.CellPlan(*to_dev(torch, cells))
    assert plan.grid_shape() == (150, 33, 9)
    ell = (0.1, 0.08, 0.05)
    out, p = _grid_run(env, cells, "gaussian", 1.0, ell, 700, 31, 0.0)
    y_or = oracle_field(oracle_modes("gaussian", 1.0, ell, 3, 700, 31), 0.0, cells)
    check_forward(out["Y"], y_or, 1.0, "rectilinear far from origin")


def test_grid_path_matches_general_path(env):
    torch, F, W = env
    cells = W.grid_centres((130, 40, 12))
    ell = (0.2, 0.1, 0.05)
    p = F.FieldParams(family="exponential", sigma2=4.0, mean=0.0, ell=ell, dim=3, n_modes=1000, seed=5)
    gf = F.GaussianField(p)
    plan = F.CellPlan(*to_dev(torch, cells))
    maps = F.MapSpec(y=True, lognormal=True, thresholds=(-0.861454, 0.861454), facies=True)
    y_or = oracle_field(oracle_modes("exponential", 4.0, ell, 3, 1000, 5), 0.0, cells)
    res = {}
    for on in (False, True):
        F.grid_path("always" if on else False)
        F.take_grid_tiles()
        out = gf.synth(plan, maps)
        torch.cuda.synchronize()
        assert (F.take_grid_tiles() > 0) == on
        res[on] = {k: v.cpu().numpy() for k, v in out.items()}
        check_forward(res[on]["Y"], y_or, 2.0, "grid path %s" % on)
        check_facies(res[on]["facies"], y_or, (-0.861454, 0.861454), 2.0)
    F.grid_path(True)
    assert np.max(np.abs(res[True]["Y"].astype(np.float64) - res[False]["Y"])) <= 2e-5 * 2.0


def test_auto_setting_small_and_large_grids(env):
    # the default setting takes the grid path for every grid plan (grids of
    # few tiles split their modes over several CTAs), and the CUDA-core
    # kernels for cells that are not a grid
    torch, F, W = env
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=256, seed=3)
    gf = F.GaussianField(p)
    jit = W.jittered_lattice((64, 64), 1.0 / 64, 0.3, seed=2)
    plan = F.CellPlan(*to_dev(torch, jit))
    F.take_grid_tiles()
    gf.synth(plan, F.MapSpec(y=True))
    torch.cuda.synchronize()
    assert F.take_grid_tiles() == 0
    for shape, grid in (((64, 64), True), ((896, 128), True), ((1024, 128), True)):
        plan = F.CellPlan(*to_dev(torch, W.grid_centres(shape)))
        F.take_grid_tiles()
        F.take_path_counts()
        out = gf.synth(plan, F.MapSpec(y=True))
        torch.cuda.synchronize()
        assert (F.take_grid_tiles() > 0) == grid, shape
        assert (sum(F.take_path_counts()) == 0) == grid, shape
        y_or = oracle_field(oracle_modes("gaussian", 1.0, (0.1, 0.1), 2, 256, 3), 0.0, W.grid_centres(shape))
        check_forward(out["Y"].cpu().numpy(), y_or, 1.0, "auto %s" % (shape,))


def test_grid3d_256_full_size_grid_path_sampled(env):
    # the headline workload: 256^3 cube, N = 4096, exponential l = (0.2, 0.2,
    # 0.05), sigma^2 = 4, three facies; a seeded sample of cells
    torch, F, W = env
    w = W.WORKLOADS["grid3d_256"]
    cells = W.workload_cells("grid3d_256")
    p = F.FieldParams(family=w["family"], sigma2=w["sigma2"], mean=w["mean"], ell=w["ell"], dim=3,
                      n_modes=w["n_modes"], seed=w["seed"])
    gf = F.GaussianField(p)
    plan = F.CellPlan(*to_dev(torch, cells))
    assert plan.grid_shape() == (256, 256, 256)
    F.take_grid_tiles()
    s = math.sqrt(w["sigma2"])
    thr = W.quantile_thresholds(0.0, s, w["quantiles"])
    out = gf.synth(plan, F.MapSpec(y=True, lognormal=True, thresholds=thr, facies=True))
    torch.cuda.synchronize()
    assert F.take_grid_tiles() == 2 * 16 * 32
    idx = np.random.default_rng(4).choice(len(cells[0]), 200_000, replace=False)
    om = oracle_modes(w["family"], w["sigma2"], w["ell"], 3, w["n_modes"], w["seed"])
    y_or = oracle_field(om, w["mean"], cells, idx)
    check_forward(out["Y"].cpu().numpy()[idx], y_or, s, "grid3d_256 grid path")
    check_lognormal(out["K"].cpu().numpy()[idx], y_or, s)
    check_facies(out["facies"].cpu().numpy()[idx], y_or, thr, s)


@pytest.mark.parametrize("shape", [(150, 90), (100, 40, 24)])
def test_mode_split_fields_and_fused_mismatch(env, shape):
    # grids of few tiles split each tile's modes over several CTAs (partial
    # fields summed in split order by a finalize kernel, which also applies the
    # maps and the loss): the same field as the unsplit CUDA-core path within
    # the tolerance, the fused loss and gradient equal to synthesis followed by
    # the standalone loss, and both against the oracle
    torch, F, W = env
    from oracle import field as of
    dim = len(shape)
    cells = W.grid_centres(shape)
    ell = (0.15, 0.1, 0.2)[:dim]
    p = F.FieldParams(family="exponential", sigma2=1.2, mean=0.05, ell=ell, dim=dim, n_modes=900, seed=31)
    pt = F.FieldParams(family="exponential", sigma2=1.2, mean=0.05, ell=ell, dim=dim, n_modes=900, seed=32)
    plan = F.CellPlan(*to_dev(torch, cells))
    gf = F.GaussianField(p)
    F.grid_path(False)
    T = F.GaussianField(pt).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    core = gf.synth(plan, F.MapSpec(y=True))["Y"]
    F.grid_path("always")
    try:
        F.take_grid_tiles()
        ref = gf.synth(plan, F.MapSpec(y=True, lognormal=True))
        loss_u, gY_u = F.mismatch_grad(ref["K"], T)
        loss, gY, out = F.synth_mismatch(gf.table, p, plan, T, want_Y=True, want_K=True)
        torch.cuda.synchronize()
        assert F.take_grid_tiles() > 0
    finally:
        F.grid_path(True)
    assert torch.equal(out["Y"], ref["Y"]) and torch.equal(out["K"], ref["K"])
    assert torch.equal(gY, gY_u)
    assert loss.item() == pytest.approx(loss_u.item(), rel=1e-12)
    assert np.max(np.abs(out["Y"].cpu().numpy().astype(np.float64) - core.cpu().numpy())) <= 2e-5 * math.sqrt(1.2)
    y_or = oracle_field(oracle_modes("exponential", 1.2, ell, dim, 900, 31), 0.05, cells)
    check_forward(out["Y"].cpu().numpy(), y_or, math.sqrt(1.2), "split %s" % (shape,))
    l_or, g_or = of.mismatch_loss(np.exp(y_or), T.cpu().numpy().astype(np.float64))
    assert loss.item() == pytest.approx(l_or, rel=1e-4)
    assert np.max(np.abs(gY.cpu().numpy() - g_or)) <= 1e-4 * np.max(np.abs(g_or))


def test_grid_path_not_offered_when_tables_outgrow_the_cells(env):
    # N = 2^20 modes on a 64^2 grid: the grid tables would be far larger than
    # max(1 GB, 64 B per cell), so the workspace queries return 0 (forward and
    # adjoint) and the CUDA-core kernels compute the field
    torch, F, W = env
    cells = W.grid_centres((64, 64))
    n_modes = 1 << 20
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.2, 0.1), dim=2, n_modes=n_modes, seed=12)
    plan = F.CellPlan(*to_dev(torch, cells))
    assert F.lib().grf_synth_grid_workspace_bytes(plan.ptr, 0, n_modes) == 0
    assert F.lib().grf_backward_grid_workspace_bytes(plan.ptr, 0, n_modes) == 0
    assert F.lib().grf_synth_grid_workspace_bytes(plan.ptr, 0, 4096) > 0
    gf = F.GaussianField(p)
    F.take_grid_tiles()
    out = gf.synth(plan, F.MapSpec(y=True))
    torch.cuda.synchronize()
    assert F.take_grid_tiles() == 0
    idx = np.arange(0, len(cells[0]), 97)
    y_or = oracle_field(oracle_modes("gaussian", 1.0, (0.2, 0.1), 2, n_modes, 12), 0.0, cells, idx)
    check_forward(out["Y"].cpu().numpy()[idx], y_or, 1.0, "2^20 modes on a 64^2 grid")
