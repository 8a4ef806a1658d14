"""Multi-GPU helpers: frames are independent problems, so N GPUs run N
replicas of the GMM, each encoding its own share of the frames (weak
scaling). No collective touches the data path; the only collectives time the
run (max over ranks) and total the work (sum over ranks).

A single frame could also be split by descriptor rows with one exchange step
(summing the per-share statistics slots, the paper's per-block copies of U
and V, before the finalise); that path is not needed for frame-parallel
workloads and is not built.
"""
from __future__ import annotations


def frame_shard(n_frames: int, rank: int, world: int) -> range:
    """Contiguous share of frame indices [0, n_frames) owned by `rank`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_frames, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def reduce_over_ranks(value: float, op: str = "max", device=None) -> float:
    """All-reduce a scalar over the default process group (max or sum);
    returns the value unchanged when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
