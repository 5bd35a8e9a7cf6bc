"""Multi-GPU runs are independent replicas (one per GPU, launched by
torchrun).  The whole-job number is the units summed over ranks divided by
the slowest rank's time.  This checks that reduction with two gloo ranks on
the CPU (rendezvous on 127.0.0.1)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.replica_reduce(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world, dist, "cpu")
    dist.barrier()
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_replica_reduce_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, units = out[r]
        assert ms == 15.0            # slowest rank
        assert units == 3000.0       # 1000 + 2000
    assert 3000.0 / (15.0e-3) == pytest.approx(200000.0)


def test_replica_reduce_single_rank_is_identity():
    import bench
    assert bench.replica_reduce(3.5, 7.0, 1) == (3.5, 7.0)
