"""Multi-rank host logic on CPU (gloo, world size 2): cell sharding covers
every cell exactly once, and summing per-shard gradients over ranks with
parallel.allreduce_grads reproduces the unsharded FP64 oracle gradient.
The per-shard gradients come from the oracle (test infrastructure)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2212_10961_gb300 import parallel


def test_shard_ranges_partition():
    for n in (0, 1, 7, 1000, 2000376):
        for world in (1, 2, 3, 7, 8):
            spans = [parallel.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (b0, e0), (b1, e1) in zip(spans, spans[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        parallel.shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import field as of
        from oracle import modes as om
        n3 = 10
        c = (np.arange(n3) + 0.5) / n3
        X, Yg, Z = np.meshgrid(c, c, c, indexing="ij")
        cells = np.stack([X.ravel(), Yg.ravel(), Z.ravel()], axis=-1)
        ell = np.array([0.3, 0.2, 0.25])
        m = om.gen_modes(0, 1.0, ell, 3, 40, seed=3)
        mt = om.gen_modes(0, 1.0, ell, 3, 40, seed=4)
        b, e = parallel.shard_range(len(cells), rank, world)
        mine = cells[b:e]
        K = of.lognormal(of.synth(m["a"], m["amp"], m["psi"], 0.0, mine))
        T = of.lognormal(of.synth(mt["a"], mt["amp"], mt["psi"], 0.0, mine))
        loss_local, g_local = of.mismatch_loss(K, T)
        n_total, frac = parallel.global_scale(len(mine))
        g = g_local * frac
        gr = of.grads_reparam(*of.mode_sums(m["a"], m["psi"], mine, g), m["kappa"], m["rho"], 1.0, ell, g)
        grads = {k: torch.as_tensor(np.asarray(gr[k], dtype=np.float64)).reshape(-1) for k in parallel.GRAD_KEYS}
        parallel.allreduce_grads(grads)
        loss = torch.tensor([loss_local * frac], dtype=torch.float64)
        dist.all_reduce(loss)
        if rank == 0:
            np.savez(out_path, loss=loss.numpy(), n_total=n_total,
                     **{k: grads[k].numpy() for k in parallel.GRAD_KEYS})
    finally:
        dist.destroy_process_group()


def test_sharded_gradient_equals_unsharded(tmp_path):
    world = 2
    out = str(tmp_path / "grads.npz")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    got = np.load(out)
    from oracle import field as of
    from oracle import modes as om
    n3 = 10
    c = (np.arange(n3) + 0.5) / n3
    X, Yg, Z = np.meshgrid(c, c, c, indexing="ij")
    cells = np.stack([X.ravel(), Yg.ravel(), Z.ravel()], axis=-1)
    ell = np.array([0.3, 0.2, 0.25])
    m = om.gen_modes(0, 1.0, ell, 3, 40, seed=3)
    mt = om.gen_modes(0, 1.0, ell, 3, 40, seed=4)
    K = of.lognormal(of.synth(m["a"], m["amp"], m["psi"], 0.0, cells))
    T = of.lognormal(of.synth(mt["a"], mt["amp"], mt["psi"], 0.0, cells))
    loss, g = of.mismatch_loss(K, T)
    ref = of.grads_reparam(*of.mode_sums(m["a"], m["psi"], cells, g), m["kappa"], m["rho"], 1.0, ell, g)
    assert float(got["n_total"]) == len(cells)
    assert got["loss"][0] == pytest.approx(loss, rel=1e-12)
    for k in parallel.GRAD_KEYS:
        np.testing.assert_allclose(got[k], np.asarray(ref[k]).reshape(-1), rtol=1e-10,
                                   atol=1e-12 * np.max(np.abs(ref[k])))
