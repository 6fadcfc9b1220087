"""Sharding of the spectral field over ranks (one GPU per process).

Cells are independent in Eq. (DiscreteFT) (Sec. 4.1), so the forward
synthesis shards the cell set into contiguous ranges with no exchange: each
rank plans and synthesises its own range with the same mode table (same seed).
Every gradient of a loss that is a sum over cells is itself a sum over cells
(dA, dpsi, da, dmu, and dsigma, dl which are linear in them), so the adjoint
of a sharded field needs exactly one exchange: a sum over ranks of the
per-rank gradients.  A mean-type loss divides by the global cell count
from the start (grf_synth_mismatch's n_mean).

Uses torch.distributed (NCCL between GPUs, gloo on CPU for tests).
"""
import torch
import torch.distributed as dist

GRAD_KEYS = ("dA", "dpsi", "da", "dmu", "dsigma", "dell", "drot", "dsigma2", "drho", "dkappa")


def shard_range(n, rank, world):
    """Contiguous [begin, end) of n cells for `rank` of `world` (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(int(n), int(world))
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def global_count(n_local, group=None):
    """Total number of cells over the ranks of `group` (one all-reduce)."""
    t = torch.tensor([float(n_local)], dtype=torch.float64,
                     device="cuda" if dist.get_backend(group) == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(round(float(t.item())))


def global_scale(n_local, group=None):
    """(n_total, n_local / n_total) for rescaling a per-rank mean-type loss."""
    n_total = global_count(n_local, group)
    return float(n_total), (float(n_local) / n_total if n_total > 0 else 0.0)


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


def sharded_loss_and_backward(F, table, params, plan, K_target, segment=0, group=None):
    """Mean mismatch loss over all ranks' cells and its gradients.

    F is the field module (paper_2212_10961_gb300.field); plan holds this
    rank's cells and K_target their target (CUDA float32, original order of
    this rank's cells).  The forward kernel divides by the global cell count
    (grf_synth_mismatch with n_mean = total), so the per-rank losses and
    gradients are the rank's shares of the global ones and the exchange is
    a plain sum.  Returns (loss, grads) identical on every rank."""
    n_total = global_count(plan.segment_size(segment), group)
    loss, gY, _ = F.synth_mismatch(table, params, plan, K_target, segment, n_mean=n_total)
    grads = F.backward(table, params, plan, gY, segment)
    dist.all_reduce(loss, op=dist.ReduceOp.SUM, group=group)
    allreduce_grads(grads, group)
    return loss, grads
