"""Multi-GPU runs are replicas (one camera stream per rank, no data-path
collective); the benchmark's rank logic is checked here with two gloo ranks
on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 * (rank + 1)            # rank 1 is the slower one
    ms, value = bench.combine_ranks(ms_local, 200, world, dist)
    out[rank] = (ms, value, bench.replica_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_frames():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        ms, value, seed = out[r]
        assert ms == 20.0                       # max over ranks
        assert abs(value - 200 * 2 / 0.020) < 1e-6   # all ranks' frames / slowest time
        assert seed == 1 + r                    # each rank its own stream
