"""Replica bookkeeping for runs over several GPUs of one node.

Views are independent units of the rasterizer, so N GPUs run N replicas with no
exchange on the data path: each rank renders its own camera pose of the same
workload, and only the timing is combined. The slowest rank sets the job's
time; the job's throughput is all ranks' units (in-mask pixels) over that time.
With one process (no process group) every function reduces to the local value.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import synth as S


def world() -> tuple[int, int]:
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def rank_rotation(rank: int, seed: int):
    """Camera rotation of a rank: the identity on rank 0 (the single-GPU
    workload itself), a seeded uniform rotation on every other rank."""
    if rank == 0:
        return None
    return S.random_rotation(np.random.default_rng(seed + 100 + rank))


def _reduce(x: float, op, dtype) -> torch.Tensor:
    ws, _ = world()
    t = torch.tensor([x], dtype=dtype)
    if ws > 1:
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=op)
    return t.cpu()


def job_time_ms(ms_local: float) -> float:
    """The job's time: the maximum over ranks."""
    return float(_reduce(ms_local, dist.ReduceOp.MAX, torch.float64).item())


def job_units(units_local: int) -> int:
    """Units processed by all ranks together."""
    return int(_reduce(units_local, dist.ReduceOp.SUM, torch.int64).item())


def throughput_per_s(units_local: int, ms_local: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return job_units(units_local) / (job_time_ms(ms_local) * 1e-3)
