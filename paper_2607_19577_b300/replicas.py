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
