"""GPU parity of the adjoint (S5) against the FP64 oracle gradient, the
chain-rule identities at full size, the loss kernel, and the autograd
wrappers."""
import math

import numpy as np
import pytest

from helpers import FAMILY_IDS, GRAD_TOL, gpu_env, oracle_field, oracle_modes, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = gpu_env()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    return torch, F, W


def _oracle_grads(om, cells, g, sigma, ell):
    from oracle import field as of
    from oracle import native
    c = np.stack(cells, axis=-1)
    s_cos, s_sin, s_sinx = native.mode_sums(om["a"], om["psi"], c, g.astype(np.float64))
    return of.grads_from_sums(s_cos, s_sin, s_sinx, om["amp"], om["a"], sigma, ell, g.astype(np.float64))


def _check(got, ref, name):
    got = np.asarray(got, dtype=np.float64).reshape(np.shape(ref))
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(got - ref))
    assert err <= GRAD_TOL * scale, "%s: max err %.3e vs scale %.3e" % (name, err, scale)
    return err / scale


@pytest.mark.parametrize("dim,family", [(3, "gaussian"), (2, "exponential"), (1, "matern")])
def test_backward_matches_oracle(env, dim, family):
    torch, F, W = env
    shape = {3: (24, 20, 18), 2: (90, 70), 1: (4000,)}[dim]
    cells = W.grid_centres(shape)
    ell = (0.1, 0.15, 0.2)[:dim]
    p = F.FieldParams(family=family, sigma2=1.7, mean=0.1, ell=ell, dim=dim, n_modes=600, seed=7)
    gf = F.GaussianField(p)
    plan = F.CellPlan(*to_dev(torch, cells))
    g = np.random.default_rng(dim).standard_normal(len(cells[0])).astype(np.float32)
    gr = F.backward(gf.table, p, plan, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    om = oracle_modes(family, 1.7, ell, dim, 600, 7)
    ref = _oracle_grads(om, cells, g, math.sqrt(1.7), ell)
    for k in ("dA", "dpsi", "da", "dsigma", "dell"):
        _check(gr[k].cpu().numpy(), ref[k], k)
    assert gr["dmu"].item() == pytest.approx(ref["dmu"], rel=1e-9, abs=1e-9)


def test_diff128_loss_and_gradients(env):
    torch, F, W = env
    w = W.WORKLOADS["diff128"]
    # reduced grid for a full oracle comparison, same modes and loss
    cells = W.grid_centres((40, 40, 40))
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=w["ell"], dim=3, n_modes=w["n_modes"], seed=1)
    pt = F.FieldParams(family="gaussian", sigma2=1.0, ell=w["ell"], dim=3, n_modes=w["n_modes"], seed=2)
    plan = F.CellPlan(*to_dev(torch, cells))
    K = F.GaussianField(p).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    T = F.GaussianField(pt).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    loss, gY = F.mismatch_grad(K, T)
    gf = F.GaussianField(p)
    gr = F.backward(gf.table, p, plan, gY)
    torch.cuda.synchronize()
    from oracle import field as of
    om = oracle_modes("gaussian", 1.0, w["ell"], 3, w["n_modes"], 1)
    omt = oracle_modes("gaussian", 1.0, w["ell"], 3, w["n_modes"], 2)
    y_or = oracle_field(om, 0.0, cells)
    t_or = np.exp(oracle_field(omt, 0.0, cells))
    l_or, g_or = of.mismatch_loss(np.exp(y_or), t_or)
    assert loss.item() == pytest.approx(l_or, rel=1e-4)
    g_gpu = gY.cpu().numpy()
    assert np.max(np.abs(g_gpu - g_or)) <= 1e-4 * np.max(np.abs(g_or))
    # oracle gradient from the oracle's own dL/dY (independent of the GPU path)
    ref = _oracle_grads(om, cells, g_or, 1.0, w["ell"])
    errs = {k: _check(gr[k].cpu().numpy(), ref[k], k) for k in ("dA", "dpsi", "da", "dmu", "dsigma", "dell")}
    print("diff 40^3 gradient errors (relative to max):", errs)


def test_diff128_full_size_identities(env):
    torch, F, W = env
    w = W.WORKLOADS["diff128"]
    cells = W.workload_cells("diff128")
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=w["ell"], dim=3, n_modes=w["n_modes"], seed=1)
    pt = F.FieldParams(family="gaussian", sigma2=1.0, ell=w["ell"], dim=3, n_modes=w["n_modes"], seed=2)
    plan = F.CellPlan(*to_dev(torch, cells))
    gf = F.GaussianField(p)
    K = gf.synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    T = F.GaussianField(pt).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    loss, gY = F.mismatch_grad(K, T)
    gr = F.backward(gf.table, p, plan, gY)
    torch.cuda.synchronize()
    amp = gf.modes["amp"]
    a = gf.modes["a"]
    dA = gr["dA"].cpu().numpy()
    da = gr["da"].cpu().numpy()
    # sigma dL/dsigma = sum_j A_j dL/dA_j ; l_c dL/dl_c = -sum_j a_jc dL/da_jc ; dL/dmu = sum g
    assert gr["dsigma"].item() == pytest.approx(np.sum(amp * dA), rel=1e-5)
    np.testing.assert_allclose(np.asarray(w["ell"]) * gr["dell"].cpu().numpy(), -np.sum(a * da, axis=0),
                               rtol=1e-5)
    assert gr["dmu"].item() == pytest.approx(float(np.sum(gY.cpu().numpy().astype(np.float64))), rel=1e-6)
    # per-mode sums on a few modes against the oracle over all 2M cells
    from oracle import native
    om = oracle_modes("gaussian", 1.0, w["ell"], 3, w["n_modes"], 1)
    sel = np.array([0, 1, 2, 100, 1000, 2047])
    c = np.stack(cells, axis=-1)
    s_cos, s_sin, s_sinx = native.mode_sums(om["a"][sel], om["psi"][sel], c, gY.cpu().numpy().astype(np.float64))
    scale = np.max(np.abs(dA))
    assert np.max(np.abs(dA[sel] - s_cos)) <= GRAD_TOL * scale
    dpsi_ref = -2 * np.pi * om["amp"][sel] * s_sin
    assert np.max(np.abs(gr["dpsi"].cpu().numpy()[sel] - dpsi_ref)) <= GRAD_TOL * np.max(np.abs(gr["dpsi"].cpu().numpy()))
    # deterministic
    gr2 = F.backward(gf.table, p, plan, gY)
    torch.cuda.synchronize()
    assert np.array_equal(gr2["dA"].cpu().numpy(), dA)


@pytest.mark.slow
def test_diff128_full_size_against_oracle(env):
    # the 128^3 forward + adjoint workload on all 2,097,152 cells: the GPU field,
    # loss and every gradient against the FP64 oracle's own (C, OpenMP)
    torch, F, W = env
    w = W.WORKLOADS["diff128"]
    cells = W.workload_cells("diff128")
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=w["ell"], dim=3, n_modes=w["n_modes"], seed=1)
    pt = F.FieldParams(family="gaussian", sigma2=1.0, ell=w["ell"], dim=3, n_modes=w["n_modes"], seed=2)
    plan = F.CellPlan(*to_dev(torch, cells))
    gf = F.GaussianField(p)
    out = gf.synth(plan, F.MapSpec(y=True, lognormal=True))
    T = F.GaussianField(pt).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    loss, gY = F.mismatch_grad(out["K"], T)
    gr = F.backward(gf.table, p, plan, gY)
    torch.cuda.synchronize()
    from oracle import field as of
    om = oracle_modes("gaussian", 1.0, w["ell"], 3, w["n_modes"], 1)
    omt = oracle_modes("gaussian", 1.0, w["ell"], 3, w["n_modes"], 2)
    y_or = oracle_field(om, 0.0, cells)
    assert np.max(np.abs(out["Y"].cpu().numpy().astype(np.float64) - y_or)) <= 1e-5
    l_or, g_or = of.mismatch_loss(np.exp(y_or), np.exp(oracle_field(omt, 0.0, cells)))
    assert loss.item() == pytest.approx(l_or, rel=1e-4)
    ref = _oracle_grads(om, cells, g_or, 1.0, w["ell"])
    errs = {k: _check(gr[k].cpu().numpy(), ref[k], k) for k in ("dA", "dpsi", "da", "dmu", "dsigma", "dell")}
    print("diff 128^3 gradient errors (relative to max):", errs)


def test_autograd_wrappers(env):
    torch, F, W = env
    cells = W.grid_centres((30, 30, 12))
    plan = F.CellPlan(*to_dev(torch, cells))
    p = F.FieldParams(family="gaussian", sigma2=1.3, ell=(0.2, 0.15, 0.1), dim=3, n_modes=256, seed=5)
    m = F.gen_modes(p)
    dt = torch.float64
    mu = torch.tensor(0.2, dtype=dt, requires_grad=True)
    sigma2 = torch.tensor(1.3, dtype=dt, requires_grad=True)
    ell = torch.tensor([0.2, 0.15, 0.1], dtype=dt, requires_grad=True)
    rho = torch.tensor(m["rho"], requires_grad=True)
    psi = torch.tensor(m["psi"], requires_grad=True)
    kappa = torch.tensor(m["kappa"], requires_grad=True)
    y = F.spectral_field(mu, sigma2, ell, rho, psi, kappa, plan)
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(y.numel()).astype(np.float32)).cuda()
    (y * g).sum().backward()
    om = oracle_modes("gaussian", 1.3, (0.2, 0.15, 0.1), 3, 256, 5)
    ref = _oracle_grads(om, cells, g.cpu().numpy(), math.sqrt(1.3), (0.2, 0.15, 0.1))
    assert mu.grad.item() == pytest.approx(ref["dmu"], rel=1e-6)
    _check(sigma2.grad.numpy(), ref["dsigma"] / (2 * math.sqrt(1.3)), "dsigma2")
    _check(ell.grad.numpy(), ref["dell"], "dell")
    _check(rho.grad.numpy() / math.sqrt(1.3), ref["dA"], "drho")
    _check(psi.grad.numpy(), ref["dpsi"], "dpsi")
    _check(kappa.grad.numpy() * 2 * np.pi * np.array([0.2, 0.15, 0.1]), ref["da"], "dkappa")
    # direct mode-sum form
    amp = torch.tensor(m["amp"], requires_grad=True)
    a = torch.tensor(m["a"], requires_grad=True)
    psi2 = torch.tensor(m["psi"], requires_grad=True)
    mu2 = torch.tensor(0.2, dtype=dt, requires_grad=True)
    y2 = F.mode_sum(mu2, amp, psi2, a, plan)
    assert torch.allclose(y2, y, atol=1e-6)
    (y2 * g).sum().backward()
    _check(amp.grad.cpu().numpy(), ref["dA"], "dA")
    _check(a.grad.cpu().numpy(), ref["da"], "da")


@pytest.mark.parametrize("case", ["rotated_periodic3d", "general_periodic3d", "periodic2d"])
def test_spectral_field_reparam_autograd(env, case):
    # Sec. 4.1 reparameterisation inside the library (grf_reparam_modes):
    # A = sigma rho, a = R^T kappa / (2 pi l), Appendix B periodic axes
    # rounded; autograd of the differentiable field against the FP64 oracle's
    # gradients of the same parameters (oracle.field.grads_reparam)
    torch, F, W = env
    from oracle import field as of
    from oracle import modes as omod
    from oracle import native
    from helpers import check_forward
    dim = 2 if case == "periodic2d" else 3
    cells = W.grid_centres((26, 22, 18) if dim == 3 else (90, 64))
    plan = F.CellPlan(*to_dev(torch, cells))
    ell = (0.22, 0.13, 0.3)[:dim]
    th = 0.45
    R = None
    if case == "rotated_periodic3d":
        R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    elif case == "general_periodic3d":
        R = np.array([[1.1, 0.5, 0.0], [0.0, 0.8, 0.3], [0.2, 0.0, 1.3]])
    period = (1.0, 0.0, 1.0) if dim == 3 else (0.0, 1.0)
    sigma2 = 1.7
    p = F.FieldParams(family="exponential", sigma2=sigma2, ell=ell, dim=dim, n_modes=640, seed=23)
    m = F.gen_modes(p)  # the draws only; the frequencies are formed below from kappa
    dt = torch.float64
    t_mu = torch.tensor(-0.3, dtype=dt, requires_grad=True)
    t_s2 = torch.tensor(sigma2, dtype=dt, requires_grad=True)
    t_ell = torch.tensor(ell, dtype=dt, requires_grad=True)
    t_rho = torch.tensor(m["rho"], requires_grad=True)
    t_psi = torch.tensor(m["psi"], requires_grad=True)
    t_kap = torch.tensor(m["kappa"], requires_grad=True)
    t_rot = None if R is None else torch.tensor(R, requires_grad=True)
    y = F.spectral_field(t_mu, t_s2, t_ell, t_rho, t_psi, t_kap, plan, rot=t_rot, period=period)
    g = np.random.default_rng(5).standard_normal(y.numel()).astype(np.float32)
    (y * torch.from_numpy(g).cuda()).sum().backward()
    torch.cuda.synchronize()
    amp, a = omod.reparam(m["kappa"], m["rho"], math.sqrt(sigma2), ell, rot=R, period=period)
    c = np.stack(cells, axis=-1)
    check_forward(y.detach().cpu().numpy(), native.synth(a, amp, m["psi"], -0.3, c), math.sqrt(sigma2), case)
    sums = native.mode_sums(a, m["psi"], c, g.astype(np.float64))
    ref = of.grads_reparam(*sums, m["kappa"], m["rho"], math.sqrt(sigma2), ell, g.astype(np.float64), rot=R,
                           period=period)
    got = {"dmu": t_mu.grad, "dsigma2": t_s2.grad, "dell": t_ell.grad, "drho": t_rho.grad, "dpsi": t_psi.grad,
           "dkappa": t_kap.grad}
    if t_rot is not None:
        got["drot"] = t_rot.grad
    errs = {k: _check(v.numpy(), ref[k], k) for k, v in got.items()}
    print(case, "gradient errors (relative to max):", errs)


@pytest.mark.parametrize("kind", ["rotation", "general"])
def test_rotated_anisotropy_forward_and_adjoint(env, kind):
    # Sec. 4.1: anisotropy axes transformed by R (a rotation with rows = principal
    # axes, or a general invertible matrix); forward parity and the gradients
    # with respect to l and R against the oracle
    torch, F, W = env
    from helpers import check_forward
    a_, b_ = 0.5, -0.3
    Rz = np.array([[math.cos(a_), -math.sin(a_), 0], [math.sin(a_), math.cos(a_), 0], [0, 0, 1.0]])
    Rx = np.array([[1.0, 0, 0], [0, math.cos(b_), -math.sin(b_)], [0, math.sin(b_), math.cos(b_)]])
    R = Rz @ Rx if kind == "rotation" else np.array([[1.1, 0.5, 0.0], [0.0, 0.8, 0.3], [0.2, 0.0, 1.3]])
    ell = (0.25, 0.12, 0.06)
    cells = W.grid_centres((28, 24, 20))
    p = F.FieldParams(family="matern", sigma2=1.4, ell=ell, dim=3, n_modes=700, seed=17, nu=1.5, rot=R.tolist())
    gf = F.GaussianField(p)
    plan = F.CellPlan(*to_dev(torch, cells))
    y = gf.synth(plan, F.MapSpec(y=True))["Y"]
    om = oracle_modes("matern", 1.4, ell, 3, 700, 17, nu=1.5)
    from oracle import modes as omod
    om = omod.gen_modes(2, 1.4, ell, 3, 700, 17, nu=1.5, rot=R)
    check_forward(y.cpu().numpy(), oracle_field(om, 0.0, cells), math.sqrt(1.4), kind)
    g = np.random.default_rng(11).standard_normal(len(cells[0])).astype(np.float32)
    gr = F.backward(gf.table, p, plan, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    from oracle import field as of
    from oracle import native
    c = np.stack(cells, axis=-1)
    s_cos, s_sin, s_sinx = native.mode_sums(om["a"], om["psi"], c, g.astype(np.float64))
    ref = of.grads_from_sums(s_cos, s_sin, s_sinx, om["amp"], om["a"], math.sqrt(1.4), ell, g.astype(np.float64),
                             rot=R)
    for k in ("dA", "dpsi", "da", "dsigma", "dell", "drot"):
        _check(gr[k].cpu().numpy(), ref[k], k)


@pytest.mark.parametrize("shape,family,rotated", [((32, 32, 32), "gaussian", False),
                                                  ((64, 32, 16), "exponential", False),
                                                  ((32, 32, 32), "matern", True),
                                                  ((64, 48, 16), "gaussian", False),
                                                  ((40, 32, 24), "exponential", True),
                                                  ((128, 128, 128), "gaussian", False)])
def test_lattice_adjoint_against_oracle(env, shape, family, rotated):
    # tiles of 256 cells that are four 4 x 4 x 4 bricks of one grid spacing
    # (Cartesian grids handed over x-fastest) take the adjoint's lattice path
    # (Horner sums of the rows' gradients, no sine or cosine per cell); the
    # exponential spectrum brings modes of the exact (heavy) class, and grid
    # spacings that are not powers of two mix lattice and general tiles
    torch, F, W = env
    cells = W.grid_centres(shape)
    ell = (0.2, 0.11, 0.07)
    R = None
    if rotated:
        a_ = 0.4
        R = np.array([[math.cos(a_), -math.sin(a_), 0.0], [math.sin(a_), math.cos(a_), 0.0], [0.0, 0.0, 1.0]])
    p = F.FieldParams(family=family, sigma2=1.3, mean=0.05, ell=ell, dim=3, n_modes=777, seed=61, nu=1.5,
                      rot=None if R is None else R.tolist())
    gf = F.GaussianField(p)
    plan = F.CellPlan(*to_dev(torch, cells))
    g = np.random.default_rng(7).standard_normal(len(cells[0])).astype(np.float32)
    F.grid_path(False)  # the CUDA-core adjoint's lattice tiles (the grid adjoint has its own tests)
    try:
        F.take_adjoint_path_counts()
        gr = F.backward(gf.table, p, plan, torch.from_numpy(g).cuda())
        torch.cuda.synchronize()
        gen, lat = F.take_adjoint_path_counts()
        assert gen + lat > 0  # the CUDA-core adjoint ran
        if shape == (128, 128, 128):
            assert lat > 0
    finally:
        F.grid_path(True)
    assert plan.status() == 0
    from oracle import field as of
    from oracle import modes as omod
    from oracle import native
    om = omod.gen_modes(FAMILY_IDS[family], 1.3, ell, 3, 777, 61, nu=1.5, rot=R)
    c = np.stack(cells, axis=-1)
    ref = of.grads_reparam(*native.mode_sums(om["a"], om["psi"], c, g.astype(np.float64)), om["kappa"], om["rho"],
                           math.sqrt(1.3), ell, g.astype(np.float64), rot=R)
    errs = {k: _check(gr[k].cpu().numpy(), ref[k], k)
            for k in ("dA", "dpsi", "da", "dmu", "dsigma", "dsigma2", "dell", "drot", "drho", "dkappa")}
    print(shape, family, "rotated" if rotated else "", "lattice tiles %d of %d," % (lat, gen + lat),
          "adjoint errors:", errs)


def test_backward_maximum_mode_count(env):
    # N = GRF_MAX_MODES = 2^24 modes on a few hundred cells: the adjoint's
    # partials stay bounded (few cell splits when the mode blocks fill the GPU),
    # the per-mode gradients against the oracle on a sample of modes
    torch, F, W = env
    from paper_2212_10961_gb300 import _abi
    from oracle import native
    n_modes = _abi.GRF_MAX_MODES
    assert F.lib().grf_backward_workspace_bytes(300, n_modes, 3) < (3 << 30)
    rng = np.random.default_rng(8)
    cells = [rng.random(300).astype(np.float32) for _ in range(3)]
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.3, 0.2, 0.1), dim=3, n_modes=n_modes, seed=6)
    gf = F.GaussianField(p)
    plan = F.CellPlan(*to_dev(torch, cells))
    g = np.random.default_rng(3).standard_normal(300).astype(np.float32)
    gr = F.backward(gf.table, p, plan, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    om = oracle_modes("gaussian", 1.0, (0.3, 0.2, 0.1), 3, n_modes, 6)
    sel = np.arange(0, n_modes, n_modes // 1000)
    s_cos, s_sin, s_sinx = native.mode_sums(om["a"][sel], om["psi"][sel], np.stack(cells, axis=-1),
                                            g.astype(np.float64))
    dA = gr["dA"].cpu().numpy()[sel]
    dpsi = gr["dpsi"].cpu().numpy()[sel]
    da = gr["da"].cpu().numpy()[sel]
    assert np.max(np.abs(dA - s_cos)) <= GRAD_TOL * np.max(np.abs(s_cos))
    ref_psi = -2 * np.pi * om["amp"][sel] * s_sin
    assert np.max(np.abs(dpsi - ref_psi)) <= GRAD_TOL * np.max(np.abs(ref_psi))
    ref_a = -2 * np.pi * om["amp"][sel][:, None] * s_sinx
    assert np.max(np.abs(da - ref_a)) <= GRAD_TOL * np.max(np.abs(ref_a))
