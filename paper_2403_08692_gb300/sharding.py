"""Several GPUs: one process per GPU, each showering its own range of event
ids.  Events are independent (Sec. 2: the event-parallel algorithm never
couples two events), so the ranks exchange nothing while they shower; the
only collectives are the job's wall time (the slowest rank) and, outside the
timed region, an optional merge of the ranks' histograms (exact when the
ranks hand over their fixed-point accumulators).  A rank's events
are exactly the events a single batch with the same first event id produces,
so the union over ranks equals one batch of world x n events."""


def shard(rank, world, n_per_rank, first_event=0):
    """(first event id, event count) of rank's range: weak scaling, n_per_rank
    events on every rank, consecutive ranges in rank order."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return first_event + rank * n_per_rank, n_per_rank


def job_time_ms(local_ms, dist=None, device="cpu"):
    """The job's time: the maximum of the ranks' times (all ranks get it)."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def merge_histograms(hist, dist=None):
    """Sum a histogram tensor over the ranks, in place (the bins, the squared
    weights and the counts of Sec. 3.2 all add)."""
    if dist is not None:
        dist.all_reduce(hist, op=dist.ReduceOp.SUM)
    return hist


def add_fixed(a, b):
    """Exact sum of two fixed-point histogram accumulators (uint64 numpy
    arrays of 5 words per cell: sum w low/high, sum w^2 low/high, entries;
    the sums are two's-complement 128-bit integers): 128-bit addition with the
    carry of the low words, so the result does not depend on the order of
    the terms."""
    import numpy as np
    a = np.asarray(a, dtype=np.uint64).reshape(-1, 5)
    b = np.asarray(b, dtype=np.uint64).reshape(-1, 5)
    out = np.empty_like(a)
    for lo in (0, 2):
        s = a[:, lo] + b[:, lo]  # wraps modulo 2^64
        carry = (s < a[:, lo]).astype(np.uint64)
        out[:, lo] = s
        out[:, lo + 1] = a[:, lo + 1] + b[:, lo + 1] + carry
    out[:, 4] = a[:, 4] + b[:, 4]
    return out.reshape(-1)


def merge_hist_fixed(acc, dist=None):
    """The fixed-point accumulators summed exactly over the ranks (every rank
    gets the sum): gathered, then added by 128-bit integer addition in rank
    order -- integer sums, so any order gives the same bits.  acc: a CPU
    torch int64 tensor (the uint64 words' bits)."""
    import numpy as np
    if dist is None:
        return acc
    import torch
    parts = [torch.empty_like(acc) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, acc)
    total = parts[0].numpy().view(np.uint64).copy()
    for p in parts[1:]:
        total = add_fixed(total, p.numpy().view(np.uint64))
    acc.copy_(torch.from_numpy(total.view(np.int64)))
    return acc
