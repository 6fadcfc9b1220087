"""GPU parity of the forward synthesis and maps against the FP64 oracle.

Every case runs the CUDA path through the C ABI and the oracle on the same
seeded inputs.  Small cases compare every cell (several warp tiles and a
ragged tail); full-size workloads compare a seeded sample of cells.
"""
import math

import numpy as np
import pytest

from helpers import (check_facies, check_forward, check_lognormal, gpu_env, oracle_field, oracle_modes,
                     to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = gpu_env()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    return torch, F, W


def run(env, cells, family, sigma2, ell, n_modes, seed, mean=0.0, nu=1.5, maps=None, plan=None):
    torch, F, W = env
    dim = len(cells)
    p = F.FieldParams(family=family, sigma2=sigma2, mean=mean, ell=ell, dim=dim, n_modes=n_modes, seed=seed, nu=nu)
    gf = F.GaussianField(p)
    if plan is None:
        plan = F.CellPlan(*to_dev(torch, cells))
    out = gf.synth(plan, maps or F.MapSpec(y=True))
    torch.cuda.synchronize()
    assert plan.status() == 0
    return {k: v.cpu().numpy() for k, v in out.items()}, p, plan


def test_grid2d_64_all_cells(env):
    torch, F, W = env
    w = W.WORKLOADS["grid2d_64"]
    cells = W.workload_cells("grid2d_64")
    maps = F.MapSpec(y=True, lognormal=True, thresholds=(0.0,), facies=True)
    out, p, _ = run(env, cells, w["family"], w["sigma2"], w["ell"], w["n_modes"], w["seed"], maps=maps)
    om = oracle_modes(w["family"], w["sigma2"], w["ell"], 2, w["n_modes"], w["seed"])
    y_or = oracle_field(om, 0.0, cells)
    check_forward(out["Y"], y_or, 1.0, "grid2d_64")
    check_lognormal(out["K"], y_or, 1.0)
    check_facies(out["facies"], y_or, [0.0], 1.0)
    # binary facies at t = 0 is the sign of Y - mu away from the band
    far = np.abs(y_or) > 1e-4
    assert np.array_equal(out["facies"][far], (y_or[far] > 0).astype(np.uint8))


@pytest.mark.parametrize("family,nu", [("gaussian", 1.5), ("exponential", 0.5), ("matern", 1.5),
                                       ("matern", 0.7)])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_families_and_dims_ragged(env, family, nu, dim):
    rng = np.random.default_rng(10 * dim + len(family))
    n_cells = 3000 + 77  # several tiles and a ragged tail
    cells = [rng.random(n_cells).astype(np.float32) * e for e in (2.0, 1.0, 0.5)[:dim]]
    ell = (0.2, 0.1, 0.05)[:dim]
    out, p, _ = run(env, cells, family, 2.0, ell, 300, seed=11, mean=0.3, nu=nu)
    om = oracle_modes(family, 2.0, ell, dim, 300, 11, nu=nu)
    check_forward(out["Y"], oracle_field(om, 0.3, cells), math.sqrt(2.0), "%s d%d" % (family, dim))


@pytest.mark.parametrize("n_cells,n_modes", [(1, 1), (31, 129), (257, 128), (1025, 1000)])
def test_edge_sizes(env, n_cells, n_modes):
    rng = np.random.default_rng(n_cells)
    cells = [rng.random(n_cells).astype(np.float32) for _ in range(3)]
    out, p, _ = run(env, cells, "gaussian", 1.0, (0.1, 0.1, 0.1), n_modes, seed=3)
    om = oracle_modes("gaussian", 1.0, (0.1, 0.1, 0.1), 3, n_modes, 3)
    check_forward(out["Y"], oracle_field(om, 0.0, cells), 1.0, "edge %d/%d" % (n_cells, n_modes))


def test_grid3d_256_reduced_all_cells(env):
    torch, F, W = env
    w = W.WORKLOADS["grid3d_256"]
    cells = W.grid_centres((64, 64, 64))
    sig = math.sqrt(w["sigma2"])
    thr = W.quantile_thresholds(0.0, sig, w["quantiles"])
    maps = F.MapSpec(y=True, lognormal=True, thresholds=thr, facies=True)
    out, p, _ = run(env, cells, w["family"], w["sigma2"], w["ell"], w["n_modes"], w["seed"], maps=maps)
    om = oracle_modes(w["family"], w["sigma2"], w["ell"], 3, w["n_modes"], w["seed"])
    idx = np.random.default_rng(0).choice(len(cells[0]), 60000, replace=False)
    y_or = oracle_field(om, 0.0, cells, idx)
    err = check_forward(out["Y"][idx], y_or, sig, "grid3d 64^3")
    check_lognormal(out["K"][idx], y_or, sig)
    check_facies(out["facies"][idx], y_or, thr, sig)
    print("grid3d 64^3 max err %.3e sigma" % err)


def test_grid3d_256_full_size_sampled(env):
    torch, F, W = env
    w = W.WORKLOADS["grid3d_256"]
    cells = W.workload_cells("grid3d_256")
    sig = math.sqrt(w["sigma2"])
    thr = W.quantile_thresholds(0.0, sig, w["quantiles"])
    maps = F.MapSpec(y=True, lognormal=True, thresholds=thr, facies=True)
    out, p, _ = run(env, cells, w["family"], w["sigma2"], w["ell"], w["n_modes"], w["seed"], maps=maps)
    om = oracle_modes(w["family"], w["sigma2"], w["ell"], 3, w["n_modes"], w["seed"])
    rng = np.random.default_rng(1)
    # one million sampled cells (plus the first and last ones) against the FP64 oracle
    idx = np.concatenate([rng.choice(len(cells[0]), 1000000, replace=False),
                          np.arange(256), len(cells[0]) - 1 - np.arange(256)])
    y_or = oracle_field(om, 0.0, cells, idx)
    err = check_forward(out["Y"][idx], y_or, sig, "grid3d 256^3")
    check_lognormal(out["K"][idx], y_or, sig)
    nb = check_facies(out["facies"][idx], y_or, thr, sig)
    print("grid3d 256^3 sampled max err %.3e sigma, %d cells in the threshold band" % (err, nb))


def test_jitter3d_reduced_and_full_sampled(env):
    torch, F, W = env
    w = W.WORKLOADS["jitter3d_2m"]
    sig = math.sqrt(w["sigma2"])
    om = oracle_modes(w["family"], w["sigma2"], w["ell"], 3, w["n_modes"], w["seed"], nu=w["nu"])
    small = W.workload_cells("jitter3d_2m", scale=4)
    out, _, _ = run(env, small, w["family"], w["sigma2"], w["ell"], w["n_modes"], w["seed"], nu=w["nu"])
    check_forward(out["Y"], oracle_field(om, 0.0, small), sig, "jitter reduced")
    cells = W.workload_cells("jitter3d_2m")
    assert len(cells[0]) == 2000376
    out, _, _ = run(env, cells, w["family"], w["sigma2"], w["ell"], w["n_modes"], w["seed"], nu=w["nu"])
    idx = np.random.default_rng(2).choice(len(cells[0]), 1000000, replace=False)
    err = check_forward(out["Y"][idx], oracle_field(om, 0.0, cells, idx), sig, "jitter full")
    print("jitter3d full sampled max err %.3e sigma" % err)


def test_shuffled_cells_and_determinism(env):
    torch, F, W = env
    cells = W.grid_centres((48, 40, 20))
    sh, perm = W.shuffled(cells, 9)
    out1, p, plan = run(env, sh, "exponential", 4.0, (0.2, 0.2, 0.05), 1024, seed=4)
    om = oracle_modes("exponential", 4.0, (0.2, 0.2, 0.05), 3, 1024, 4)
    check_forward(out1["Y"], oracle_field(om, 0.0, sh), 2.0, "shuffled")
    out2, _, _ = run(env, sh, "exponential", 4.0, (0.2, 0.2, 0.05), 1024, seed=4, plan=plan)
    assert np.array_equal(out1["Y"], out2["Y"])  # deterministic
    out3, _, _ = run(env, sh, "exponential", 4.0, (0.2, 0.2, 0.05), 1024, seed=4)
    assert np.array_equal(out1["Y"], out3["Y"])  # plan is deterministic too


def test_large_coordinates_exact_path(env):
    # cells far from the origin: phases of hundreds of thousands of turns
    rng = np.random.default_rng(5)
    cells = [(1000.0 + rng.random(5000)).astype(np.float32) for _ in range(3)]
    out, p, _ = run(env, cells, "exponential", 1.0, (0.05, 0.05, 0.05), 512, seed=8)
    om = oracle_modes("exponential", 1.0, (0.05, 0.05, 0.05), 3, 512, 8)
    check_forward(out["Y"], oracle_field(om, 0.0, cells), 1.0, "far cells")


def test_rough_field_medium_and_super_classes(env):
    # correlation length five times smaller than the cell spacing, exponential
    # (Cauchy-like spectrum): most modes span more than the light-class limit
    # over a warp tile, so the lane-origin and per-cell exact paths carry much
    # of the sum; every cell against the oracle
    torch, F, W = env
    cells = W.grid_centres((64, 64, 64))
    ell = (0.003, 0.003, 0.003)
    out, p, _ = run(env, cells, "exponential", 2.0, ell, 1500, seed=13)
    om = oracle_modes("exponential", 2.0, ell, 3, 1500, 13)
    span = np.sum(np.abs(om["a"]), axis=1) * (4.0 / 64.0)  # turns over a warp tile's half-extent
    assert np.mean(span > 8.0) > 0.5  # the light class is the minority here
    check_forward(out["Y"], oracle_field(om, 0.0, cells), math.sqrt(2.0), "rough field")


def test_maps_standalone_and_fused(env):
    torch, F, W = env
    rng = np.random.default_rng(6)
    cells = [rng.random(5000).astype(np.float32) for _ in range(2)]
    thr = (-0.5, 0.25, 1.0)
    vals = (10.0, 20.0, 30.0, 40.0)
    maps = F.MapSpec(y=True, lognormal=True, k_ref=2.5, thresholds=thr, facies=True, values=vals)
    out, p, plan = run(env, cells, "matern", 1.5, (0.1, 0.1), 500, seed=2, mean=0.2, maps=maps)
    Yd = torch.from_numpy(out["Y"]).cuda()
    st = F.map_property(Yd, F.MapSpec(y=False, lognormal=True, k_ref=2.5, thresholds=thr, facies=True,
                                      values=vals), 0.2, math.sqrt(1.5))
    torch.cuda.synchronize()
    assert np.array_equal(st["K"].cpu().numpy(), out["K"])
    assert np.array_equal(st["facies"].cpu().numpy(), out["facies"])
    assert np.array_equal(st["prop"].cpu().numpy(), out["prop"])
    lab = out["facies"]
    assert np.array_equal(out["prop"], np.asarray(vals, dtype=np.float32)[lab])
    # porosity map
    por = F.map_property(Yd, F.MapSpec(y=False, porosity=(0.25, 0.05, 0.1, 0.35)), 0.2, math.sqrt(1.5))
    torch.cuda.synchronize()
    from oracle import field as of
    want = of.porosity(out["Y"].astype(np.float64), 0.2, math.sqrt(1.5), 0.25, 0.05, 0.1, 0.35)
    np.testing.assert_allclose(por["prop"].cpu().numpy(), want, rtol=0, atol=1e-6)
    om = oracle_modes("matern", 1.5, (0.1, 0.1), 2, 500, 2)
    y_or = oracle_field(om, 0.2, cells)
    check_lognormal(out["K"], y_or, math.sqrt(1.5), k_ref=2.5)
    check_facies(out["facies"], y_or, thr, math.sqrt(1.5))


def test_most_thresholds_and_fused_porosity(env):
    # the largest truncation rule (GRF_MAX_THRESHOLDS thresholds, 16 facies with
    # values) and the porosity map, both fused into the synthesis kernel
    torch, F, W = env
    from paper_2212_10961_gb300 import _abi
    from oracle import field as of
    rng = np.random.default_rng(17)
    cells = [rng.random(3000).astype(np.float32) for _ in range(2)]
    sig = math.sqrt(2.0)
    q = (np.arange(_abi.GRF_MAX_THRESHOLDS) + 1.0) / (_abi.GRF_MAX_THRESHOLDS + 1.0)
    thr = tuple(W.quantile_thresholds(-0.3, sig, q))
    vals = tuple(float(v) for v in 10.0 ** np.arange(len(thr) + 1))
    maps = F.MapSpec(y=True, thresholds=thr, facies=True, values=vals)
    out, p, plan = run(env, cells, "gaussian", 2.0, (0.15, 0.1), 400, seed=23, mean=-0.3, maps=maps)
    om = oracle_modes("gaussian", 2.0, (0.15, 0.1), 2, 400, 23)
    y_or = oracle_field(om, -0.3, cells)
    check_forward(out["Y"], y_or, sig, "16 facies")
    check_facies(out["facies"], y_or, thr, sig)
    assert np.array_equal(out["prop"], np.asarray(vals, dtype=np.float32)[out["facies"]])
    assert len(np.unique(out["facies"])) == len(thr) + 1  # every facies occurs
    pmap = F.MapSpec(y=False, porosity=(0.25, 0.05, 0.1, 0.35))
    por, _, _ = run(env, cells, "gaussian", 2.0, (0.15, 0.1), 400, seed=23, mean=-0.3, maps=pmap, plan=plan)
    want = of.porosity(y_or, -0.3, sig, 0.25, 0.05, 0.1, 0.35)
    # porosity is affine in Y with slope 0.05 / sigma, then clamped
    np.testing.assert_allclose(por["prop"], want, rtol=0, atol=0.05 / sig * 1e-5 * sig + 1e-6)


@pytest.mark.parametrize("off,n", [(0, 5000), (1, 4999), (0, 2051), (4, 4093), (3, 1)])
def test_map_standalone_ragged_and_misaligned(env, off, n):
    # offsets that break the 16-byte alignment of Y take the per-cell path;
    # sizes that end inside a thread's groups take the ragged tail
    torch, F, W = env
    rng = np.random.default_rng(16)
    cells = [rng.random(5000).astype(np.float32) for _ in range(2)]
    thr = (-0.5, 0.25, 1.0)
    maps = F.MapSpec(y=True, lognormal=True, k_ref=2.5, thresholds=thr, facies=True)
    out, p, plan = run(env, cells, "gaussian", 1.0, (0.1, 0.1), 256, seed=4, maps=maps)
    Yd = torch.from_numpy(out["Y"]).cuda()[off:off + n]
    st = F.map_property(Yd, F.MapSpec(y=False, lognormal=True, k_ref=2.5, thresholds=thr, facies=True),
                        0.0, 1.0)
    torch.cuda.synchronize()
    assert np.array_equal(st["K"].cpu().numpy(), out["K"][off:off + n])
    assert np.array_equal(st["facies"].cpu().numpy(), out["facies"][off:off + n])


def test_lognormal_map_exponential_accuracy(env):
    # K = k_ref exp(Y) over a wide range of Y, against FP64 exp of the same FP32 values
    torch, F, W = env
    y = np.concatenate([np.linspace(-80.0, 80.0, 200001), np.random.default_rng(3).normal(0.0, 3.0, 100000)])
    y = y.astype(np.float32)
    st = F.map_property(torch.from_numpy(y).cuda(), F.MapSpec(y=False, lognormal=True, k_ref=1.0), 0.0, 1.0)
    torch.cuda.synchronize()
    k = st["K"].cpu().numpy().astype(np.float64)
    want = np.exp(y.astype(np.float64))
    rel = np.abs(k - want) / want
    assert np.max(rel) <= 2.0 ** -20, "max relative error %.3e" % np.max(rel)


def test_segments_share_one_plan(env):
    torch, F, W = env
    a = W.grid_centres((40, 30))
    b = W.grid_centres((17, 23))
    cells = [np.concatenate([a[k], b[k] * 3.0]) for k in range(2)]
    plan = F.CellPlan(*to_dev(torch, cells), segments=[1200, 391])
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=700, seed=21)
    gf = F.GaussianField(p)
    om = oracle_modes("gaussian", 1.0, (0.1, 0.1), 2, 700, 21)
    for s, c in ((0, a), (1, [b[0] * 3.0, b[1] * 3.0])):
        out = gf.synth(plan, F.MapSpec(y=True), segment=s)
        torch.cuda.synchronize()
        check_forward(out["Y"].cpu().numpy(), oracle_field(om, 0.0, c), 1.0, "segment %d" % s)


def test_many_segments_coarsen_the_sort_grid(env):
    # 2^17 one-cell segments after a 2M-cell one: the segment index takes 18
    # key bits, so the quantisation grid of the large segment is made coarser
    # (4 bits per axis instead of 6) to keep 32-bit sort keys.
    torch, F, W = env
    big = W.jittered_lattice((160, 128, 104), 1.0 / 128, 0.3, seed=5)
    n_small = 1 << 17
    rng = np.random.default_rng(6)
    small = [rng.uniform(-2.0, 2.0, n_small).astype(np.float32) for _ in range(3)]
    cells = [np.concatenate([big[k], small[k]]) for k in range(3)]
    sizes = [len(big[0])] + [1] * n_small
    plan = F.CellPlan(*to_dev(torch, cells), segments=sizes)
    p = F.FieldParams(family="exponential", sigma2=2.0, ell=(0.2, 0.15, 0.1), dim=3, n_modes=1024, seed=31)
    gf = F.GaussianField(p)
    om = oracle_modes("exponential", 2.0, (0.2, 0.15, 0.1), 3, 1024, 31)
    sig = math.sqrt(2.0)
    y = gf.synth(plan, F.MapSpec(y=True), segment=0)["Y"].cpu().numpy()
    idx = np.random.default_rng(7).choice(len(y), 20000, replace=False)
    check_forward(y[idx], oracle_field(om, 0.0, big, idx), sig, "large segment")
    for s in (1, 2, 777, n_small):
        ys = gf.synth(plan, F.MapSpec(y=True), segment=s)["Y"].cpu().numpy()
        c = [small[k][s - 1:s] for k in range(3)]
        check_forward(ys, oracle_field(om, 0.0, c), sig, "one-cell segment %d" % s)
    torch.cuda.synchronize()
    assert plan.status() == 0


def test_empty_plan_and_empty_segment(env):
    # no cells at all, and an empty segment between two others: nothing to
    # compute, no error, and the neighbouring segments are unaffected
    torch, F, W = env
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    plan0 = F.CellPlan(e, e, e)
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1, 0.1), dim=3, n_modes=300, seed=4)
    gf = F.GaussianField(p)
    out = gf.synth(plan0, F.MapSpec(y=True, lognormal=True, thresholds=(0.0,), facies=True))
    assert all(v.numel() == 0 for v in out.values())
    g0 = F.backward(gf.table, p, plan0, torch.empty(0, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert plan0.status() == 0
    assert float(g0["dA"].abs().max()) == 0.0 and float(g0["dmu"].abs().max()) == 0.0
    rng = np.random.default_rng(5)
    a = [rng.random(100).astype(np.float32) for _ in range(3)]
    b = [rng.random(57).astype(np.float32) + 2.0 for _ in range(3)]
    cells = [np.concatenate([a[k], b[k]]) for k in range(3)]
    plan = F.CellPlan(*to_dev(torch, cells), segments=[100, 0, 57])
    om = oracle_modes("gaussian", 1.0, (0.1, 0.1, 0.1), 3, 300, 4)
    assert gf.synth(plan, F.MapSpec(y=True), segment=1)["Y"].numel() == 0
    for s, c in ((0, a), (2, b)):
        y = gf.synth(plan, F.MapSpec(y=True), segment=s)["Y"].cpu().numpy()
        check_forward(y, oracle_field(om, 0.0, c), 1.0, "segment %d" % s)
    torch.cuda.synchronize()
    assert plan.status() == 0


def test_maximum_mode_count(env):
    # N = GRF_MAX_MODES = 2^24 modes (131,072 chunks of 128) on a few hundred
    # cells, checked against the oracle on a sample of them
    torch, F, W = env
    from paper_2212_10961_gb300 import _abi
    n_modes = _abi.GRF_MAX_MODES
    rng = np.random.default_rng(8)
    cells = [rng.random(300).astype(np.float32) for _ in range(3)]
    out, p, plan = run(env, cells, "gaussian", 1.0, (0.3, 0.2, 0.1), n_modes, seed=6)
    om = oracle_modes("gaussian", 1.0, (0.3, 0.2, 0.1), 3, n_modes, 6)
    idx = np.arange(0, 300, 15)
    err = check_forward(out["Y"][idx], oracle_field(om, 0.0, cells, idx), 1.0, "2^24 modes")
    print("max-abs field error with 2^24 modes: %.3e sigma" % err)


def test_rejects_bad_calls(env):
    torch, F, W = env
    from paper_2212_10961_gb300 import _abi
    cells = W.grid_centres((16, 16))
    plan = F.CellPlan(*to_dev(torch, cells))
    p = F.FieldParams(dim=2, ell=(0.1, 0.1), n_modes=64)
    gf = F.GaussianField(p)
    with pytest.raises(_abi.GRFError) as e:
        F.synth(gf.table, p, plan, segment=1)
    assert e.value.code == _abi.GRF_EINVAL
    with pytest.raises(_abi.GRFError):
        F.synth(gf.table, p, plan, maps=F.MapSpec(y=False))
    g = torch.zeros(256, dtype=torch.float32, device="cuda")
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    import ctypes
    gs = _abi.grf_grads()
    bufs = [torch.empty(64 * 2, dtype=torch.float64, device="cuda") for _ in range(6)]
    for k, bb in zip(("dA", "dpsi", "da", "dmu", "dsigma", "dell"), bufs):
        setattr(gs, k, bb.data_ptr())
    rc = _abi.lib().grf_synth_backward(gf.table.ptr, ctypes.byref(p.to_c()), plan.ptr, 0,
                                       ctypes.c_void_p(g.data_ptr()), ctypes.byref(gs),
                                       ctypes.c_void_p(ws.data_ptr()), 1024, None)
    assert rc == _abi.GRF_EWORKSPACE
    assert plan.status() == 0


def test_mode_split_matches_unsplit_and_oracle(env):
    # a small segment (few cell tiles) is split over mode groups through the
    # workspace; partials are combined in a fixed order
    torch, F, W = env
    cells = W.grid_centres((40, 36, 30))
    plan = F.CellPlan(*to_dev(torch, cells))
    p = F.FieldParams(family="exponential", sigma2=4.0, ell=(0.2, 0.2, 0.05), dim=3, n_modes=3000, seed=12)
    gf = F.GaussianField(p)
    maps = F.MapSpec(y=True, lognormal=True, thresholds=(-0.5, 0.5), facies=True)
    F.grid_path(False)  # the CUDA-core kernel's mode split (the grid path has its own tests)
    try:
        split = F.synth(gf.table, p, plan, 0, maps)
        split2 = F.synth(gf.table, p, plan, 0, maps)
        whole = F.synth(gf.table, p, plan, 0, maps, workspace=False)
        torch.cuda.synchronize()
    finally:
        F.grid_path(True)
    ys, yw = split["Y"].cpu().numpy(), whole["Y"].cpu().numpy()
    assert np.array_equal(ys, split2["Y"].cpu().numpy())
    assert np.max(np.abs(ys - yw)) <= 2e-6 * 2.0
    om = oracle_modes("exponential", 4.0, (0.2, 0.2, 0.05), 3, 3000, 12)
    y_or = oracle_field(om, 0.0, cells)
    check_forward(ys, y_or, 2.0, "split")
    check_lognormal(split["K"].cpu().numpy(), y_or, 2.0)
    check_facies(split["facies"].cpu().numpy(), y_or, (-0.5, 0.5), 2.0)
    assert plan.status() == 0


@pytest.mark.parametrize("angle", [None, 0.5])
def test_periodic_field_repeats(env, angle):
    # Appendix B `periodic`: with L = (1, 1) the field at x + (1, 0) and
    # x + (0, 1) equals the field at x (frequencies on the reciprocal lattice);
    # also with the anisotropy axes rotated (the snapping follows the rotation)
    torch, F, W = env
    rot = None if angle is None else ((math.cos(angle), math.sin(angle)), (-math.sin(angle), math.cos(angle)))
    # dyadic centres, so that x + 1 and y + 1 are exact in FP32 (otherwise the
    # shifted point itself moves, and high-frequency modes see it)
    base = W.grid_centres((64, 32))
    segs = [base, [base[0] + 1.0, base[1]], [base[0], base[1] + 1.0]]
    for s_ in segs[1:]:
        assert np.array_equal((s_[0].astype(np.float64) - base[0]) % 1.0, np.zeros(len(base[0])))
        assert np.array_equal((s_[1].astype(np.float64) - base[1]) % 1.0, np.zeros(len(base[0])))
    cells = [np.concatenate([s_[k] for s_ in segs]).astype(np.float32) for k in range(2)]
    n = len(base[0])
    plan = F.CellPlan(*to_dev(torch, cells), segments=[n, n, n])
    p = F.FieldParams(family="exponential", sigma2=2.0, ell=(0.2, 0.1), dim=2, n_modes=800, seed=5,
                      period=(1.0, 1.0), rot=rot)
    gf = F.GaussianField(p)
    ys = [gf.synth(plan, F.MapSpec(y=True), segment=k)["Y"].cpu().numpy() for k in range(3)]
    torch.cuda.synchronize()
    sig = math.sqrt(2.0)
    assert np.max(np.abs(ys[1] - ys[0])) <= 2e-5 * sig
    assert np.max(np.abs(ys[2] - ys[0])) <= 2e-5 * sig
    from oracle import modes as om
    m = om.gen_modes(1, 2.0, (0.2, 0.1), 2, 800, 5, period=(1.0, 1.0), rot=None if rot is None else np.array(rot))
    for k in range(3):
        check_forward(ys[k], oracle_field(m, 0.0, segs[k]), sig, "periodic segment %d" % k)


def test_hrl2d_workload_sampled(env):
    torch, F, W = env
    w = W.WORKLOADS["hrl2d"]
    cells = W.workload_cells("hrl2d")
    assert len(cells[0]) == 1024 * 512 and float(cells[0].max()) < 2.0 and float(cells[1].max()) < 1.0
    sig = math.sqrt(w["sigma2"])
    thr = W.quantile_thresholds(0.0, sig, w["quantiles"])
    maps = F.MapSpec(y=True, lognormal=True, thresholds=thr, facies=True, values=w["values"])
    out, p, _ = run(env, cells, w["family"], w["sigma2"], w["ell"], w["n_modes"], w["seed"], maps=maps)
    om = oracle_modes(w["family"], w["sigma2"], w["ell"], 2, w["n_modes"], w["seed"])
    idx = np.random.default_rng(7).choice(len(cells[0]), 20000, replace=False)
    y_or = oracle_field(om, 0.0, cells, idx)
    check_forward(out["Y"][idx], y_or, sig, "hrl2d")
    check_lognormal(out["K"][idx], y_or, sig)
    check_facies(out["facies"][idx], y_or, thr, sig)
    assert np.array_equal(out["prop"], np.asarray(w["values"], dtype=np.float32)[out["facies"]])
    # quartile thresholds: each facies holds about a quarter of the cells
    frac = np.bincount(out["facies"], minlength=4) / len(out["facies"])
    assert np.all(np.abs(frac - 0.25) < 0.15)


@pytest.mark.parametrize("shape,family", [((64, 48), "gaussian"), ((128, 48), "exponential"), ((64, 40), "matern"),
                                          ((64, 64), "gaussian"), ((32, 32, 32), "exponential"),
                                          ((64, 40, 24), "gaussian"), ((64, 64, 8), "matern")])
def test_lattice_lanes_against_oracle(env, shape, family):
    # Cartesian grids in x-fastest order: warps whose lanes all hold 4 x C/4
    # blocks of one spacing take the lattice path (step phasors), the others
    # the general one; grids where only some lanes of a warp are such blocks
    # (one grid spacing not a power of two) mix both kinds of lanes in a warp
    torch, F, W = env
    cells = W.grid_centres(shape)
    d = len(shape)
    ell = (0.13, 0.1, 0.07)[:d]
    p = F.FieldParams(family=family, sigma2=1.6, mean=-0.2, ell=ell, dim=d, n_modes=700, seed=29, nu=1.5)
    plan = F.CellPlan(*to_dev(torch, cells))
    gf = F.GaussianField(p)
    y_or = oracle_field(oracle_modes(family, 1.6, ell, d, 700, 29), -0.2, cells)
    F.grid_path(False)  # the CUDA-core lattice and general paths (the grid path has its own tests)
    for ws in (False, None):  # without and with the mode split
        try:
            out = F.synth(gf.table, p, plan, 0, F.MapSpec(y=True, lognormal=True, thresholds=(0.0,), facies=True),
                          workspace=ws)
            torch.cuda.synchronize()
        finally:
            F.grid_path(True)
        assert plan.status() == 0
        check_forward(out["Y"].cpu().numpy(), y_or, math.sqrt(1.6), "%s %s" % (shape, family))
        check_lognormal(out["K"].cpu().numpy(), y_or, math.sqrt(1.6))
        check_facies(out["facies"].cpu().numpy(), y_or, (0.0,), math.sqrt(1.6))
