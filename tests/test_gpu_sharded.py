"""Sharding of one field over R ranks, emulated on one GPU with host-side
shards (no collective): every shard plans and synthesises its own contiguous
range of cells with the same mode table, and the adjoint of a mean-type loss
is the sum over shards of the per-shard gradients of the rescaled local loss
(the exchange `parallel.allreduce_grads` performs between ranks).  The
product function itself runs as two processes in test_gpu_calibration."""
import math

import numpy as np
import pytest

from helpers import GRAD_TOL, Y_TOL_SIGMA, check_forward, gpu_env, oracle_field, oracle_modes, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3, 7])
def test_sharded_forward_and_adjoint_match_unsharded(world):
    torch = gpu_env()
    from paper_2212_10961_gb300 import field as F
    from paper_2212_10961_gb300 import parallel
    from paper_2212_10961_gb300 import workloads as W
    cells = W.jittered_lattice((40, 24, 20), 1.0 / 40, 0.3, seed=9)
    n = len(cells[0])
    dev = to_dev(torch, cells)
    sigma2, ell, N = 1.5, (0.2, 0.1, 0.15), 384
    p = F.FieldParams(family="exponential", sigma2=sigma2, ell=ell, dim=3, n_modes=N, seed=21)
    pt = F.FieldParams(family="exponential", sigma2=sigma2, ell=ell, dim=3, n_modes=N, seed=22)
    gf, gt = F.GaussianField(p), F.GaussianField(pt)
    maps = F.MapSpec(y=True, lognormal=True)

    # unsharded reference on the GPU
    plan = F.CellPlan(*dev)
    full = gf.synth(plan, maps)
    T = gt.synth(plan, maps)["K"]
    loss_full, gY, _ = F.synth_mismatch(gf.table, p, plan, T)
    g_full = F.backward(gf.table, p, plan, gY)

    # shards
    sig = math.sqrt(sigma2)
    y_parts, loss_sum = [], 0.0
    acc = {k: torch.zeros_like(g_full[k]) for k in parallel.GRAD_KEYS}
    for r in range(world):
        b, e = parallel.shard_range(n, r, world)
        plan_r = F.CellPlan(*[c[b:e] for c in dev])
        out_r = gf.synth(plan_r, maps)
        # the shard's share of the global mean: divided by the global count
        loss_r, gY_r, _ = F.synth_mismatch(gf.table, p, plan_r, T[b:e], n_mean=n)
        g_r = F.backward(gf.table, p, plan_r, gY_r)
        for k in parallel.GRAD_KEYS:
            acc[k] += g_r[k]
        loss_sum += float(loss_r.item())
        y_parts.append(out_r["Y"].cpu().numpy())
    torch.cuda.synchronize()

    y_sh = np.concatenate(y_parts)
    y_full = full["Y"].cpu().numpy()
    # shards group cells into different warp tiles, so the two differ by rounding only
    assert np.max(np.abs(y_sh.astype(np.float64) - y_full)) <= Y_TOL_SIGMA * sig
    om = oracle_modes("exponential", sigma2, ell, 3, N, 21)
    idx = np.random.default_rng(3).choice(n, 4000, replace=False)
    check_forward(y_sh[idx], oracle_field(om, 0.0, cells, idx), sig, "sharded")
    assert abs(loss_sum - float(loss_full.item())) <= 1e-5 * abs(float(loss_full.item()))
    for k in parallel.GRAD_KEYS:
        want = g_full[k].cpu().numpy()
        got = acc[k].cpu().numpy()
        scale = np.max(np.abs(want))
        assert np.max(np.abs(got - want)) <= GRAD_TOL * scale, k
