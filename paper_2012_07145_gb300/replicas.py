"""Replica data parallelism: one independent copy of the pipeline per GPU.

The image pipelines have no exchange step between images, so N GPUs serve N
independent streams of images (or requests); nothing is communicated on the
data path.  The only collective is the host-side reduction of each rank's
timing to the job's (the slowest rank bounds the job), done once per run.
"""

import datetime


def shard(n_items: int, rank: int, world: int):
    """Indices of a list of independent items (images, requests) that one rank
    takes: round robin, so every item goes to exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(range(rank, n_items, world))


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the job's step time); identity when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / max_seconds


def init_gloo(rank: int, world: int, port: int, timeout_s: float = 30.0):
    """A CPU process group on 127.0.0.1 (for host-side tests of this logic)."""
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=timeout_s))
