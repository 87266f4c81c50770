"""Host logic of the multi-GPU bench (replicas only: no data-path collective).
Two gloo ranks on the CPU: the timing reduction returns the slowest rank's time on
every rank, and the whole-job value counts all ranks' units over that time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
    m = bench.reduce_max(dist, ms, "cpu")
    v = bench.replica_value(1000, ws, m)
    out.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 15.0
        assert v == pytest.approx(2 * 1000 / 15e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(None, 3.5, "cpu") == 3.5
    assert bench.replica_value(600, 1, 2.0) == pytest.approx(300000.0)
