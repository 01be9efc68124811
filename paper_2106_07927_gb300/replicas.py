"""Host side of multi-GPU runs: independent replicas, one process per GPU.

A stereo pair does not shard without a sequential hand-off (the vertical and diagonal paths run
over the whole image height), so several GPUs run independent replicas: each rank computes its own
pairs, nothing crosses between ranks on the data path, and the only collectives are a barrier
around the timed region and the reductions of the timings. Throughput of the whole job is the work
of all ranks over the slowest rank's time (weak scaling: the work per rank is fixed).

The functions take the process group's backend as it is: NCCL with CUDA tensors on the GPUs,
gloo with CPU tensors in the tests.
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _device():
    import torch
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def _reduce(value: float, op) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float) -> float:
    """The largest value over all ranks (the slowest rank's time)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX)


def sum_over_ranks(value: float) -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_throughput(units_this_rank: float, seconds_this_rank: float) -> float:
    """Units all ranks processed per second of the slowest rank."""
    return sum_over_ranks(units_this_rank) / max_over_ranks(seconds_this_rank)


def shard(n: int, world: int, rank: int) -> range:
    """The contiguous block of item indices 0 .. n - 1 that rank owns (sizes differ by at most
    one; every item has exactly one owner)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))
