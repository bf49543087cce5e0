"""The replica path of bench.py (one process per GPU, no data-path collective) on
CPU: two gloo ranks with different local times agree on the slowest rank's time,
and the job value counts the units of both ranks."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, q):
    import torch.distributed as tdist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_info() == (ws, rank, rank)
    local_ms = [100.0, 150.0][rank]
    max_ms, value = bench.job_throughput(local_ms, ws, 5, 1.0e9, "cpu", tdist)
    tdist.barrier()
    tdist.destroy_process_group()
    q.put((rank, max_ms, value))


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, max_ms, value in res:
        assert max_ms == 150.0
        assert abs(value - 2 * 5 * 1.0e9 / 0.150) <= 1e-6 * value
