"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every rank
advances its own blocks, the reported time is the max over ranks and the value is
the whole-job aggregate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
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
    ms = 10.0 + 5.0 * rank                 # rank 1 is the slow one
    got = bench.max_over_ranks(ms, "cpu")
    val = bench.weak_scaling_value(1_000_000, 3, got, world)
    q.put((rank, got, val))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, got, val in res:
        assert got == 15.0
        assert abs(val - 2 * 1_000_000 * 3 / 15e-3 / 1e6) < 1e-9


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.weak_scaling_value(100, 3, 1.0, 1) == pytest.approx(0.3)
