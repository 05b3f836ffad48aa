"""The multi-rank bench path on the CPU (gloo, world size 2): ranks are
independent replicas, the timed region is the slowest rank's, and the metric
counts every rank's right-hand sides."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(1000.0 * (rank + 1))
    value = bench.seconds_per_rhs(ms, 3, 64, world)
    out.put((rank, ms, value))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_rhs():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2000.0, 2000.0]
    assert all(abs(r[2] - 2.0 / (3 * 64 * 2)) < 1e-15 for r in res)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.seconds_per_rhs(1000.0, 1, 64, 1) == 1.0 / 64
