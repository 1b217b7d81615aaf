"""Host-side logic of multi-GPU runs: independent replicas, no data exchange.

The hot path does not shard across GPUs here: each rank advances its own
jets (ensemble members are fully independent), so the only cross-rank
communication is the throughput report at the end -- total particle-steps
over the slowest rank's time (weak scaling).
"""
from __future__ import annotations


def rank_members(rank: int, world: int, n_members: int) -> list:
    """Members (e.g. seeds of an ensemble) owned by `rank`: round-robin."""
    if not (0 <= rank < world):
        raise ValueError("rank %d outside world of %d" % (rank, world))
    return list(range(rank, n_members, world))


def reduce_rate(seconds: float, units: float, dist=None, device=None):
    """Whole-job throughput: sum of the units of all ranks divided by the
    largest per-rank time.  Returns (rate, max_seconds, total_units); with
    dist None (one process) the inputs themselves."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return units / seconds, seconds, units
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())
