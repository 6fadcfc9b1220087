"""GPU checks of the calibration step (forward half fused with the mismatch
loss, grf_synth_mismatch; the differentiable loss spectral_mismatch) and of
the sharded product function parallel.sharded_loss_and_backward run as two
processes with a gloo group on the one GPU (their kernels never wait on each
other; the exchange is gloo's host-side all-reduce)."""
import math
import os
import socket

import numpy as np
import pytest

from helpers import GRAD_TOL, Y_TOL_SIGMA, check_forward, gpu_env, oracle_field, oracle_modes, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = gpu_env()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import workloads as W
    return torch, F, W


def _check(got, ref, name):
    got = np.asarray(got, dtype=np.float64).reshape(np.shape(ref))
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(got - ref))
    assert err <= GRAD_TOL * scale, "%s: max err %.3e vs scale %.3e" % (name, err, scale)
    return err / scale


@pytest.mark.parametrize("shape,dim,split", [((30, 26, 21), 3, True), ((30, 26, 21), 3, False),
                                             ((333, 97), 2, True), ((5001,), 1, False)])
def test_fused_mismatch_equals_synthesis_then_loss(env, shape, dim, split):
    # same FP32 field and gradient as grf_synth_field + grf_mismatch_grad; the
    # FP64 loss differs only in the order of its sum; against the FP64 oracle
    torch, F, W = env
    cells = W.grid_centres(shape)
    ell = (0.15, 0.1, 0.2)[:dim]
    p = F.FieldParams(family="exponential", sigma2=1.2, mean=0.05, ell=ell, dim=dim, n_modes=900, seed=31)
    pt = F.FieldParams(family="exponential", sigma2=1.2, mean=0.05, ell=ell, dim=dim, n_modes=900, seed=32)
    plan = F.CellPlan(*to_dev(torch, cells))
    gf = F.GaussianField(p)
    T = F.GaussianField(pt).synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    ref = gf.synth(plan, F.MapSpec(y=True, lognormal=True))
    loss_u, gY_u = F.mismatch_grad(ref["K"], T)
    if split:
        loss, gY, out = F.synth_mismatch(gf.table, p, plan, T, want_Y=True, want_K=True)
    else:
        # a workspace that holds only the loss partials: no mode split
        n = len(cells[0])
        small = torch.empty(int(F.lib().grf_synth_mismatch_workspace_bytes(n)) -
                            int(F.lib().grf_synth_workspace_bytes(n)), dtype=torch.uint8, device="cuda")

        class Fixed:  # hands out exactly this buffer (a Workspace would grow it)
            def get(self, nbytes, device):
                return small

        loss, gY, out = F.synth_mismatch(gf.table, p, plan, T, want_Y=True, want_K=True, workspace=Fixed())
        ref = F.synth(gf.table, p, plan, 0, F.MapSpec(y=True, lognormal=True), workspace=False)
        loss_u, gY_u = F.mismatch_grad(ref["K"], T)
    torch.cuda.synchronize()
    assert torch.equal(out["Y"], ref["Y"]) and torch.equal(out["K"], ref["K"])
    assert torch.equal(gY, gY_u)
    assert loss.item() == pytest.approx(loss_u.item(), rel=1e-12)
    # against the oracle's own loss and gradient
    from oracle import field as of
    om = oracle_modes("exponential", 1.2, ell, dim, 900, 31)
    y_or = oracle_field(om, 0.05, cells)
    check_forward(out["Y"].cpu().numpy(), y_or, math.sqrt(1.2), "fused")
    l_or, g_or = of.mismatch_loss(np.exp(y_or), T.cpu().numpy().astype(np.float64))
    assert loss.item() == pytest.approx(l_or, rel=1e-4)
    assert np.max(np.abs(gY.cpu().numpy() - g_or)) <= 1e-4 * np.max(np.abs(g_or))


def test_fused_mismatch_mean_count_and_empty_segment(env):
    torch, F, W = env
    cells = W.grid_centres((64, 48))
    n = len(cells[0])
    c2 = [np.concatenate([c, c]) for c in cells]
    plan = F.CellPlan(*to_dev(torch, c2), segments=[0, n, n])  # an empty segment first
    p = F.FieldParams(family="gaussian", sigma2=1.0, ell=(0.1, 0.1), dim=2, n_modes=500, seed=3)
    gf = F.GaussianField(p)
    T = torch.ones(n, dtype=torch.float32, device="cuda")
    l1, g1, _ = F.synth_mismatch(gf.table, p, plan, T, segment=1)
    l2, g2, _ = F.synth_mismatch(gf.table, p, plan, T, segment=1, n_mean=2 * n)
    l0, g0, _ = F.synth_mismatch(gf.table, p, plan, T[:0], segment=0)
    torch.cuda.synchronize()
    # a mean over twice the cells halves the loss and the gradient exactly
    assert l2.item() == 0.5 * l1.item() and torch.equal(g2, 0.5 * g1)
    assert l0.item() == 0.0 and g0.numel() == 0
    with pytest.raises(F._abi.GRFError):
        F.synth_mismatch(gf.table, p, plan, T, segment=1, n_mean=n - 1)
    # the segment's gradient equals the one of a plan of those cells alone
    # (taking the same CUDA-core path: a single-grid plan would otherwise use
    # the tensor-core grid path)
    plan1 = F.CellPlan(*to_dev(torch, cells))
    F.grid_path(False)
    try:
        l3, g3, _ = F.synth_mismatch(gf.table, p, plan1, T)
        torch.cuda.synchronize()
    finally:
        F.grid_path(True)
    assert l3.item() == pytest.approx(l1.item(), rel=1e-6)
    assert torch.max(torch.abs(g3 - g1)).item() <= 1e-6 * torch.max(torch.abs(g1)).item()


@pytest.mark.parametrize("case", ["rotated_periodic3d", "plain2d"])
def test_spectral_mismatch_autograd(env, case):
    # calibration objective through autograd: L = mean (exp(Y) - T)^2 of the
    # Sec. 4.1 reparameterised field, gradients of all parameters against the
    # FP64 oracle (grads_reparam of the oracle's own loss gradient)
    torch, F, W = env
    from oracle import field as of
    from oracle import modes as omod
    from oracle import native
    dim = 3 if case == "rotated_periodic3d" else 2
    cells = W.grid_centres((28, 24, 20) if dim == 3 else (120, 90))
    plan = F.CellPlan(*to_dev(torch, cells))
    ell = (0.2, 0.12, 0.25)[:dim]
    R, period = None, None
    if dim == 3:
        th = 0.35
        R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
        period = (1.0, 0.0, 1.0)
    sigma2 = 0.8
    p = F.FieldParams(family="gaussian", sigma2=sigma2, ell=ell, dim=dim, n_modes=512, seed=41)
    m = F.gen_modes(p)
    c = np.stack(cells, axis=-1)
    mt = omod.gen_modes(0, sigma2, ell, dim, 512, 42)
    T64 = np.exp(native.synth(mt["a"], mt["amp"], mt["psi"], 0.0, c))
    T = torch.from_numpy(T64.astype(np.float32)).cuda()
    dt = torch.float64
    t = {"mu": torch.tensor(0.1, dtype=dt), "sigma2": torch.tensor(sigma2, dtype=dt),
         "ell": torch.tensor(ell, dtype=dt), "rho": torch.tensor(m["rho"]), "psi": torch.tensor(m["psi"]),
         "kappa": torch.tensor(m["kappa"])}
    if R is not None:
        t["rot"] = torch.tensor(R)
    for v in t.values():
        v.requires_grad_(True)
    loss = F.spectral_mismatch(t["mu"], t["sigma2"], t["ell"], t["rho"], t["psi"], t["kappa"], plan, T,
                               rot=t.get("rot"), period=period)
    loss.backward()
    torch.cuda.synchronize()
    amp, a = omod.reparam(m["kappa"], m["rho"], math.sqrt(sigma2), ell, rot=R, period=period)
    y_or = native.synth(a, amp, m["psi"], 0.1, c)
    l_or, g_or = of.mismatch_loss(np.exp(y_or), T.cpu().numpy().astype(np.float64))
    assert loss.item() == pytest.approx(l_or, rel=1e-4)
    ref = of.grads_reparam(*native.mode_sums(a, m["psi"], c, g_or), m["kappa"], m["rho"], math.sqrt(sigma2), ell,
                           g_or, rot=R, period=period)
    names = {"mu": "dmu", "sigma2": "dsigma2", "ell": "dell", "rho": "drho", "psi": "dpsi", "kappa": "dkappa",
             "rot": "drot"}
    errs = {k: _check(t[k].grad.numpy(), ref[names[k]], names[k]) for k in t}
    print(case, "calibration gradient errors (relative to max):", errs)
    # an upstream factor reaches every gradient through the library's device scale
    first = {k: v.grad.clone() for k, v in t.items()}
    for v in t.values():
        v.grad = None
    loss2 = F.spectral_mismatch(t["mu"], t["sigma2"], t["ell"], t["rho"], t["psi"], t["kappa"], plan, T,
                                rot=t.get("rot"), period=period)
    (2.5 * loss2).backward()
    for k in t:
        assert torch.allclose(t[k].grad, 2.5 * first[k], rtol=1e-12, atol=0), k


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sharded_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2212_10961_gb300 import field as F
        from paper_2212_10961_gb300 import parallel
        from paper_2212_10961_gb300 import workloads as W
        cells = W.jittered_lattice((40, 24, 20), 1.0 / 40, 0.3, seed=9)
        b, e = parallel.shard_range(len(cells[0]), rank, world)
        mine = [torch.from_numpy(np.ascontiguousarray(c[b:e])).cuda() for c in cells]
        plan = F.CellPlan(*mine)
        kw = dict(family="exponential", sigma2=1.5, ell=(0.2, 0.1, 0.15), dim=3, n_modes=384)
        p, pt = F.FieldParams(seed=21, **kw), F.FieldParams(seed=22, **kw)
        gf, gt = F.GaussianField(p), F.GaussianField(pt)
        T = gt.synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
        loss, grads = parallel.sharded_loss_and_backward(F, gf.table, p, plan, T)
        Y = gf.synth(plan, F.MapSpec(y=True))["Y"]
        torch.cuda.synchronize()
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), loss=loss.cpu().numpy(), Y=Y.cpu().numpy(),
                 **{k: v.cpu().numpy() for k, v in grads.items()})
    finally:
        dist.destroy_process_group()


def test_sharded_product_function_two_processes(env, tmp_path):
    # parallel.sharded_loss_and_backward on each half of a jittered lattice in
    # two processes (gloo), against the unsharded fused forward and adjoint
    torch, F, W = env
    import torch.multiprocessing as mp
    from paper_2212_10961_gb300 import parallel
    world = 2
    mp.spawn(_sharded_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(str(tmp_path / ("rank%d.npz" % r))) for r in range(world)]
    cells = W.jittered_lattice((40, 24, 20), 1.0 / 40, 0.3, seed=9)
    plan = F.CellPlan(*to_dev(torch, cells))
    kw = dict(family="exponential", sigma2=1.5, ell=(0.2, 0.1, 0.15), dim=3, n_modes=384)
    p, pt = F.FieldParams(seed=21, **kw), F.FieldParams(seed=22, **kw)
    gf, gt = F.GaussianField(p), F.GaussianField(pt)
    T = gt.synth(plan, F.MapSpec(y=False, lognormal=True))["K"]
    loss, gY, out = F.synth_mismatch(gf.table, p, plan, T, want_Y=True)
    g = F.backward(gf.table, p, plan, gY)
    torch.cuda.synchronize()
    sig = math.sqrt(1.5)
    y_sh = np.concatenate([r["Y"] for r in res])
    assert np.max(np.abs(y_sh.astype(np.float64) - out["Y"].cpu().numpy())) <= Y_TOL_SIGMA * sig
    for r in res:  # every rank holds the same global result
        assert r["loss"][0] == pytest.approx(loss.item(), rel=1e-5)
        for k in parallel.GRAD_KEYS:
            _check(r[k], g[k].cpu().numpy(), k)
    assert np.array_equal(res[0]["dA"], res[1]["dA"]) and res[0]["loss"][0] == res[1]["loss"][0]
