"""The multi-process path of bench.py on CPU: world_size 2 over gloo.  Each rank runs an
independent replica (or its shard of independent instances); the only cross-rank steps
are the barrier and the max of the step times, and the whole-job value counts every
rank's sites."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2011_00287_gb300 import workloads as WL


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 2.0 + rank  # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, dist, device="cpu")
    units = WL.shard(64, rank, world)
    total = bench.sum_over_ranks(len(units), dist, device="cpu")
    out[rank] = (ms, total, units[0], units[-1])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo_max_time_and_shards():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 3.0
    assert out[0][1] == out[1][1] == 64
    assert (out[0][2], out[0][3], out[1][2], out[1][3]) == (0, 31, 32, 63)
    assert bench.whole_job_mlups(sites=128 ** 3, world=2, ms=3.0) == pytest.approx(2 * 128 ** 3 / 3e-3 / 1e6)
