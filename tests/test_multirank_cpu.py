"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): the batched workload
is split between the ranks by point count (each block on exactly one rank, loads balanced),
every rank steps with the smallest CFL step of all ranks, the reported time is the max over
ranks and the value is the whole-job aggregate."""
import os
import socket

import numpy as np
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
    from paper_2101_05886_gb300 import inputs as I
    ms = 10.0 + 5.0 * rank                 # rank 1 is the slow one
    got = bench.max_over_ranks(ms, "cpu")
    val = bench.weak_scaling_value(1_000_000, 3, got, world)
    sizes = I.batched_block_sizes(64 * world, 32, 128, 4)
    mine = bench.rank_share(sizes, world, rank)
    dt_local = 1e-3 * (1.0 + rank)          # rank 0 has the smallest CFL step
    dt = -bench.max_over_ranks(-dt_local, "cpu")
    q.put((rank, got, val, mine, dt))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_time_step_and_timing_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    from paper_2101_05886_gb300 import inputs as I
    sizes = I.batched_block_sizes(128, 32, 128, 4)
    shares = {}
    for rank, got, val, mine, dt in res:
        assert got == 15.0
        assert abs(val - 2 * 1_000_000 * 3 / 15e-3 / 1e6) < 1e-9
        assert dt == 1e-3                  # every rank steps with the global minimum
        shares[rank] = mine
    allb = sorted(shares[0] + shares[1])
    assert allb == list(range(128))        # each block on exactly one rank
    load = [sum(int(np.prod(sizes[k])) for k in shares[r]) for r in (0, 1)]
    heaviest = max(int(np.prod(n)) for n in sizes)
    assert abs(load[0] - load[1]) <= heaviest     # greedy heaviest-first bound


def test_single_process_identity():
    import bench
    from paper_2101_05886_gb300 import inputs as I
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.weak_scaling_value(100, 3, 1.0, 1) == pytest.approx(0.3)
    sizes = I.batched_block_sizes(64, 32, 128, 4)
    assert bench.rank_share(sizes, 1, 0) == list(range(64))
