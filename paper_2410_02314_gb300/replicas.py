"""Several GPUs of one node: independent replicas, one process per GPU.

Every frame is localized on its own (the net's receptive field never crosses frames and the
decode is per frame), so the path shards by frames with no exchange of data: rank r runs the
whole path on its own frame stacks.  The only collectives are for timing: a barrier and a
device synchronise on both sides of the timed region, and a max over the ranks' times, so
the whole-job rate is all ranks' frames over the slowest rank's time.
"""
from __future__ import annotations

import dataclasses
import os


@dataclasses.dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local: int


def rank_info(env=None) -> RankInfo:
    """Rank, world size and local rank from the torchrun environment (1 process if unset)."""
    env = os.environ if env is None else env
    return RankInfo(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0")))


def frame_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s synthetic frames: each replica localizes different frames."""
    return base + rank


def timed_region(run, dist=None, sync=None):
    """Run `run()` bracketed by a barrier and `sync()` on both sides; return its result."""
    if dist is not None:
        dist.barrier()
    if sync is not None:
        sync()
    out = run()
    if sync is not None:
        sync()
    if dist is not None:
        dist.barrier()
    return out


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest `value` over all ranks (every rank gets it); `value` itself with one rank."""
    if dist is None or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Units per second over the whole job: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds_max
