"""The multi-GPU benchmark path runs independent replicas (the method has no
exchange step on one lattice): check its whole-job aggregation (slowest
rank's time, summed work) with two gloo ranks on the CPU."""
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
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 150.0][rank]
    cells = [1000, 3000][rank]
    res = bench.aggregate_replicas(ms, cells, 10, dist)
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms_max, cells, mlups = got[r]
        assert ms_max == 150.0 and cells == 4000.0
        assert abs(mlups - 4000 * 10 / 0.150 / 1e6) < 1e-12


def test_replica_aggregation_single_rank():
    import bench

    assert bench.aggregate_replicas(2.0, 500, 4) == (2.0, 500.0, 500 * 4 / 2e-3 / 1e6)
