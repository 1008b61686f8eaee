"""The N > 1 path of bench.py on CPU: two gloo ranks, each an independent
replica (weak scaling, no collective on the data path); the timing aggregate
takes the slowest rank and sums the points of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms_local = 2.0 + rank  # rank 1 is slower
    ms, value = bench.aggregate(ms_local, 1000, ws)
    bench.barrier(ws)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 3.0
        assert abs(value - 2 * 1000 / 3e-3) < 1e-6 * value
