"""Host side of the multi-GPU path: channels are independent end to end
(correlate, reduce and calibrate are all per channel), so each rank runs the
whole cycle on its own band of channels with no collective on the data path.
The only collective is the max over ranks of the timed region.

Each rank draws its own synthetic channels (weak scaling: the per-rank work
is fixed as ranks are added), from a seed offset by the rank, so that the
bands of different ranks are different, reproducible data.
"""
from __future__ import annotations

RANK_SEED_STRIDE = 1000


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's band of channels."""
    if rank < 0:
        raise ValueError("rank must be >= 0")
    return base_seed + RANK_SEED_STRIDE * rank


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks of the default process group (the value
    itself without one); device is where the reduction tensor lives (a CUDA
    device for NCCL, None / cpu for gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (ms)."""
    if ms <= 0.0:
        raise ValueError("time must be positive")
    return units_per_rank * world / (ms * 1e-3)
