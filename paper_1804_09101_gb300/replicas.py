"""Replica timing helpers for multi-GPU runs.

The benchmarked workload is one black hole whose shells exchange boundary
data at every right-hand side, so it does not shard: with N GPUs every rank
evolves its own replica and no collective touches the data path.  Only the
timing is combined: the job's time is the maximum over ranks and its
throughput counts the work of all ranks (weak scaling).
"""
import torch


def max_over_ranks(value, dist=None):
    """Maximum of a float over all ranks of the default process group (or the value itself)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def job_throughput(units_per_rank, world, max_ms):
    """Whole-job units per second: every rank processed units_per_rank in at most max_ms."""
    return world * units_per_rank / (max_ms / 1000.0)
