"""The replica path of a multi-GPU run, as two gloo ranks on CPU: per-rank camera
poses, the job time as the maximum over ranks, and the whole-job throughput."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_29794_b300 import replicas as RP
from paper_2606_29794_b300 import synth as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert RP.world() == (world, rank)
        ms = 10.0 + 5.0 * rank                      # the slower rank sets the job time
        units = 1000 * (rank + 1)
        rot = RP.rank_rotation(rank, 7)
        view = S.make_view(5, S.CAM_FISHEYE, 190.0, R=rot)
        out[rank] = (RP.job_time_ms(ms), RP.job_units(units), RP.throughput_per_s(units, ms),
                     np.asarray(view["W"], np.float64).ravel().tolist())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:     # no fork: the parent may hold a CUDA context
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        t, u, thr, _ = res[r]
        assert t == 15.0 and u == 3000
        assert abs(thr - 3000 / 15e-3) < 1e-6
    W0, W1 = np.array(res[0][3]).reshape(3, 3), np.array(res[1][3]).reshape(3, 3)
    assert np.allclose(W0, np.eye(3))                 # rank 0 renders the single-GPU workload itself
    assert not np.allclose(W1, np.eye(3))
    assert np.allclose(W1 @ W1.T, np.eye(3), atol=1e-6)


def test_single_process_reduces_to_local():
    assert RP.world() == (1, 0)
    assert RP.job_time_ms(3.5) == 3.5 and RP.job_units(7) == 7
    assert RP.rank_rotation(0, 1) is None
