"""Several GPUs run independent RT-DetMCD replicas (no data-path collective):
the whole-job throughput is the rows of every rank over the slowest rank's
time.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 200.0][rank]
    v, tot = bench.replica_throughput(local_ms, 1_000_000, 10, world, dist, None)
    q.put((rank, v, tot))
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, v, tot in res:
        assert tot == 200.0
        assert v == pytest.approx(10 * 1_000_000 * 2 / 0.2)


def test_single_rank_needs_no_process_group():
    import bench
    v, tot = bench.replica_throughput(50.0, 1000, 5, 1)
    assert tot == 50.0 and v == pytest.approx(5 * 1000 / 0.05)
