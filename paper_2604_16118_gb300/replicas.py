"""Replica bookkeeping for runs with one process per GPU.

The solver has no exchange step that pays across GPUs at the sizes it runs
(one Alg. 2 step is a chain of site-sequential sweeps), so several GPUs run
independent replicas: either copies of one problem (weak scaling of a fixed
per-GPU workload) or disjoint shares of a batch of independent problems.  The
only cross-rank traffic is host-side bookkeeping after the timed region: the
slowest rank's time and the summed work.
"""


def shard(n_units, rank, world):
    """Contiguous range [beg, end) of n_units independent problems owned by
    `rank` of `world`; the first n_units % world ranks take one extra unit."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError(f"rank {rank} outside a world of {world}")
    if n_units < 0:
        raise ValueError("negative unit count")
    base, extra = divmod(n_units, world)
    beg = rank * base + min(rank, extra)
    return beg, beg + base + (1 if rank < extra else 0)


def reduce_timing(total_ms, total_work, dist=None, device=None):
    """(max over ranks of the timed milliseconds, sum over ranks of the work).

    `dist` is torch.distributed (None for a single process); the reduction runs
    on `device` (a CUDA device for NCCL, the CPU for gloo)."""
    if dist is None:
        return float(total_ms), float(total_work)
    import torch

    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(total_work)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
