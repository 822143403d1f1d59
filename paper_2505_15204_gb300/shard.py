"""Work partition over ranks (one process per GPU).

The path shards without any exchange: every (50 ms chunk, channel) block of an observation is imaged
independently (the paper partitions observations into independent time intervals, Sec. 5.1 and 6.1),
so ranks take whole chunks round-robin and never communicate on the data path.  Only the benchmark's
timing uses a collective (the max over ranks).
"""
from __future__ import annotations


def chunks_for_rank(n_chunks: int, rank: int, world: int, first: int = 0) -> list:
    """Chunk indices imaged by `rank`: first + rank, first + rank + world, ... (mod n_chunks).

    With more ranks than chunks, a rank left without a chunk images chunk (first + rank) mod n_chunks as a
    replica, so that every rank does one chunk's work (weak scaling)."""
    if world < 1 or not 0 <= rank < world or n_chunks < 1:
        raise ValueError("bad rank / world / chunk count")
    mine = [(first + c) % n_chunks for c in range(rank, n_chunks, world)]
    return mine or [(first + rank) % n_chunks]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over all ranks (the slowest rank sets the job's time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds_max
