"""Sharding of the spectral field over ranks (one GPU per process).

Cells are independent in Eq. (DiscreteFT) (Sec. 4.1), so the forward
synthesis shards the cell set into contiguous ranges with no exchange: each
rank plans and synthesises its own range with the same mode table (same seed).
Every gradient of a loss that is a sum over cells is itself a sum over cells
(dA, dpsi, da, dmu, and dsigma, dl which are linear in them), so the adjoint
of a sharded field needs exactly one exchange: a sum over ranks of the
per-rank gradients.  A mean-type loss is first rescaled from the local to the
global cell count.

Uses torch.distributed (NCCL between GPUs, gloo on CPU for tests).
"""
import torch
import torch.distributed as dist

GRAD_KEYS = ("dA", "dpsi", "da", "dmu", "dsigma", "dell", "drot")


def shard_range(n, rank, world):
    """Contiguous [begin, end) of n cells for `rank` of `world` (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(int(n), int(world))
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def global_scale(n_local, group=None):
    """(n_total, n_local / n_total) for rescaling a per-rank mean-type loss."""
    t = torch.tensor([float(n_local)], dtype=torch.float64,
                     device="cuda" if dist.get_backend(group) == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    n_total = float(t.item())
    return n_total, (float(n_local) / n_total if n_total > 0 else 0.0)


def allreduce_grads(grads, group=None):
    """Sum every gradient over ranks in place (one all-reduce of a packed FP64 buffer)."""
    keys = [k for k in GRAD_KEYS if k in grads]
    flat = torch.cat([grads[k].reshape(-1).to(torch.float64) for k in keys])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for k in keys:
        n = grads[k].numel()
        grads[k].copy_(flat[off:off + n].reshape(grads[k].shape))
        off += n
    return grads


def sharded_loss_and_backward(F, table, params, plan, K, K_target, group=None):
    """Mean mismatch loss over all ranks' cells and its gradients.

    F is the field module (paper_2212_10961_gb300.field); K and K_target are
    this rank's lognormal field and target (CUDA float32, original order of
    this rank's cells).  Returns (loss, grads) identical on every rank."""
    loss_local, gY = F.mismatch_grad(K, K_target)
    n_total, frac = global_scale(K.numel(), group)
    gY.mul_(frac)  # d(global mean)/dY = (n_local / n_total) d(local mean)/dY
    grads = F.backward(table, params, plan, gY)
    loss = loss_local * frac
    dist.all_reduce(loss, op=dist.ReduceOp.SUM, group=group)
    allreduce_grads(grads, group)
    return loss, grads
