"""Host-side logic of runs on several GPUs (one process per GPU).

The hot path needs no exchange between ranks here: every rank advances its own
problem (a replica of a workload with its own seed, or its share of a batch of
independent domains), so the only collective is the reduction of the timing
and the work done, after the timed region."""


def aggregate(ms, units, dist=None, device="cpu"):
    """Whole-job figures: (the slowest rank's time, the units all ranks processed)."""
    import torch
    if dist is None:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
