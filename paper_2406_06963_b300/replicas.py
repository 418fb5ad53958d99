"""Replica bookkeeping for runs on several GPUs of one node.

The hot path does not shard: every rank renders its own frames (its own
scene copy, camera path and SVGF history) and no data moves between ranks.
What is shared is only the measurement: a barrier on both sides of the
timed region, the slowest rank's time and the sum of the units all ranks
processed.  These helpers hold that logic so that it runs the same over
NCCL (one process per GPU) and over gloo (CPU processes, in tests).
"""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _device():
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def barrier(ws: int) -> None:
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(ws: int, x: float, op: str) -> float:
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(ws: int, x: float) -> float:
    """The largest x over all ranks (the slowest rank's time)."""
    return _reduce(ws, x, "max")


def sum_over_ranks(ws: int, x: float) -> float:
    """The sum of x over all ranks (units processed by the whole job)."""
    return _reduce(ws, x, "sum")


def job_throughput(ws: int, units: float, seconds: float) -> tuple[float, float, float]:
    """Whole-job throughput: units summed over ranks / the slowest rank's
    seconds.  Returns (throughput, total units, max seconds)."""
    total = sum_over_ranks(ws, units)
    tmax = max_over_ranks(ws, seconds)
    return total / tmax, total, tmax
