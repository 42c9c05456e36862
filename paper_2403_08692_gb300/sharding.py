"""Several GPUs: one process per GPU, each showering its own range of event
ids.  Events are independent (Sec. 2: the event-parallel algorithm never
couples two events), so the ranks exchange nothing while they shower; the
only collectives are the job's wall time (the slowest rank) and, outside the
timed region, an optional merge of the ranks' histograms.  A rank's events
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
