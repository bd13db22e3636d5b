"""Several GPUs: independent replicas.

The solves of different right-hand sides, masses and gauge configurations are
independent problems, so more GPUs run more of them side by side: every rank
holds its own copy of the gauge fields and solves its own share of the work,
with no collective on the data path.  The only cross-rank steps are host-side
bookkeeping: which share a rank takes, and the job-level throughput (units of
all ranks over the slowest rank's time, the weak-scaling figure).
"""


def shard(n, rank, world):
    """Indices of n independent items that `rank` of `world` takes (round-robin,
    so ranks differ by at most one item and every item has exactly one owner)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError('bad rank %r of world %r' % (rank, world))
    return list(range(rank, n, world))


def _reduce(value, dist, op, dtype_device=None):
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    dev = dtype_device if dtype_device is not None else 'cpu'
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value, dist=None, device=None):
    """Largest value over the ranks (e.g. the slowest rank's time)."""
    return _reduce(value, dist, dist.ReduceOp.MAX if dist is not None else None, device)


def sum_over_ranks(value, dist=None, device=None):
    return _reduce(value, dist, dist.ReduceOp.SUM if dist is not None else None, device)


def job_throughput(units_local, seconds_local, dist=None, device=None):
    """Whole-job throughput: units solved by all ranks divided by the time of the
    slowest rank (every rank started together after a barrier)."""
    units = sum_over_ranks(units_local, dist, device)
    secs = max_over_ranks(seconds_local, dist, device)
    return units / secs if secs > 0 else float('nan')
