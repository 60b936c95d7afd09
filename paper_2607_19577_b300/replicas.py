"""Host-side aggregation for runs over several ranks (one process per GPU).

Each rank evaluates its own units (a replica of the workload, or a shard of the
settings); the job's time is the slowest rank's and its throughput counts the
units of every rank.  Works with any torch.distributed backend (NCCL on GPUs,
gloo on CPU)."""
import torch


def aggregate(ms_local: float, units_local: float, dist=None, device="cpu"):
    """(max over ranks of ms_local, sum over ranks of units_local).

    With dist None (a single process) the local values are returned."""
    if dist is None:
        return float(ms_local), float(units_local)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def shard(M: int, rank: int, world: int):
    """Contiguous setting range [lo, hi) of rank `rank` out of `world` (sizes
    differ by at most one)."""
    q, r = divmod(M, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shard_rows(row_ptr, lo: int, hi: int):
    """CSR slice of settings [lo, hi): (row_ptr rebased to 0, first entry, end entry)."""
    a, b = int(row_ptr[lo]), int(row_ptr[hi])
    return row_ptr[lo:hi + 1] - a, a, b


def allreduce_evaluation(loss, grad_psi, grad_w, dist=None):
    """The exchange step of the measurement partition (Sec. III-B): every rank has
    evaluated its contiguous shard of the settings with the global normalisation
    B, so the loss, dJ/dpsi^* (= -w_k G psi_k) and dJ/dw (= -h) of the whole
    experiment are the sums of the ranks' values.  One all-reduce (sum) of the
    gradient block [grad_psi as real pairs, grad_w] in its own dtype and one of
    the loss in float64; in place on every rank.  Tensors may live on the GPU
    (NCCL) or the CPU (gloo); with dist None nothing is exchanged."""
    if dist is None:
        return loss, grad_psi, grad_w
    flat = torch.cat([torch.view_as_real(grad_psi).reshape(-1), grad_w.reshape(-1).to(grad_psi.real.dtype)])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    K = grad_w.numel()
    grad_psi.copy_(torch.view_as_complex(flat[:-K].reshape(*grad_psi.shape, 2)))
    grad_w.copy_(flat[-K:].to(grad_w.dtype))
    dist.all_reduce(loss, op=dist.ReduceOp.SUM)
    return loss, grad_psi, grad_w
