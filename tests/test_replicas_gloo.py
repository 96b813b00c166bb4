"""bench.py's multi-GPU path runs independent replicas: the only exchange is
the max over ranks of the timings.  World size 2 over gloo on CPU."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0 + 50.0 * rank, 300.0 - 10.0 * rank]  # per-rank (timed, e2e) milliseconds
    got = bench.max_over_ranks(ms, world, device="cpu")
    out[rank] = got + [bench.replica_throughput(10, world, got[0])]
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][:2] == [150.0, 300.0]
        assert abs(res[r][2] - 2 * 10 / 0.150) < 1e-9


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.0, 2.0], 1) == [1.0, 2.0]
    assert bench.replica_throughput(5, 1, 250.0) == 20.0
