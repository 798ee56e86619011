"""Independent replicas across ranks (one process per GPU, torch.distributed).

Views are independent problems: every rank runs the whole per-frame chain on
its own frames with its own cache, and no data moves between ranks.  Ranks
only meet in a barrier around the timed region and in one max-reduction of the
elapsed times, so the aggregate throughput is (records of all ranks) / (slowest
rank's time)."""
from __future__ import annotations

import torch
import torch.distributed as dist


def frame_indices(rank: int, n_frames: int, path_frames: int) -> list[int]:
    """Frames of the camera path replayed by `rank`: n_frames consecutive frames starting
    rank * n_frames along the path (wrapping), so ranks start on different frames."""
    start = (rank * n_frames) % path_frames
    return [(start + k) % path_frames for k in range(n_frames)]


def barrier(world: int) -> None:
    if world > 1:
        dist.barrier()


def max_over_ranks(values, world: int, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def aggregate_rate(records_per_rank: int, world: int, steps: int, slowest_seconds: float) -> float:
    """Whole-job records per second: every rank processed records_per_rank per step."""
    return world * records_per_rank * steps / slowest_seconds
