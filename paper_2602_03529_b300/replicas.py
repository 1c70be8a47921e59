"""Multi-GPU replicas: independent clips/streams per rank, no data-path collective.

The tokenizer's work units (clips of a batch, streams of a serving mix) are
independent, so N GPUs run N replicas. The only cross-rank traffic is
host-side bookkeeping: a barrier around the timed region and the maximum of
the ranks' elapsed times.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def init(backend: str | None = None) -> None:
    rank, local, ws = world()
    if ws > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)


def shard(n_units: int, rank: int, world_size: int) -> list[int]:
    """Units assigned to `rank`: round-robin, so every rank's share differs by at most one."""
    return list(range(rank, n_units, world_size))


def barrier() -> None:
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def _reduce(value: float, op) -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float) -> float:
    return _reduce(value, dist.ReduceOp.MAX)


def sum_over_ranks(value: float) -> float:
    return _reduce(value, dist.ReduceOp.SUM)


def finalize() -> None:
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
