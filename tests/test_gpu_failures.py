"""Failure paths on the GPU, injected on the host: allocation failures through the
library's failure hook (fp_debug_fail_allocation), swept over every allocation that
fp_init_grid, fp_batch_create and fp_pipe_create make.  Each must return FP_ERR_OOM,
hand back nothing and release whatever it had allocated; nothing here faults, traps or
hangs the GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2101_05886_gb300 import binding as B  # noqa: E402
from paper_2101_05886_gb300 import inputs as I  # noqa: E402
from paper_2101_05886_gb300.solver import Batch, Block, Pipe  # noqa: E402


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _sweep(make, limit=200):
    """Arm a failure at allocation k = 0, 1, ... until `make` succeeds; returns (the number
    of allocations that failed cleanly, the object made)."""
    for k in range(limit):
        B.fp_debug_fail_allocation(k)
        try:
            obj = make()
        except B.FPError as e:
            assert e.status == B.FP_ERR_OOM, (k, str(e))
            continue
        finally:
            B.fp_debug_fail_allocation(-1)
        return k, obj
    raise AssertionError("still failing after %d allocations" % limit)


def test_every_allocation_failure_returns_oom_and_releases_memory():
    M = 6
    Gn = O.node_ghost(M)
    qinf = I.uniform_qinf(0.8, 0.0)
    grids = [I.periodic_wavy_3d((20, 17, 13), L=10.0, amp=0.08, Gn=Gn), I.cylinder_ogrid((24, 18, 10), Lz=3.0, Gn=Gn),
             I.periodic_wavy_3d((16, 24, 12), L=10.0, amp=0.08, Gn=Gn)]
    warm = [Block(g, metric_order=M, precision=B.FP_F32_MIXED, q_inf=qinf) for g in grids]   # modules loaded
    states = [b.to_device(I.random_smooth_state(g, qinf, amp=0.03, seed=k)) for k, (b, g) in enumerate(zip(warm, grids))]
    hosts = [s.cpu().pin_memory() for s in states]
    w = Batch(warm, states, autotune=False)
    w.close()
    free0 = _free_bytes()

    n_init, blk = _sweep(lambda: Block(grids[1], metric_order=M, precision=B.FP_F32_MIXED, q_inf=qinf))
    assert n_init >= 20                       # every device buffer of a context was exercised
    blk.close()
    n_batch, bat = _sweep(lambda: Batch(warm, states, autotune=False))
    assert n_batch >= 8
    bat.rk3_step(1e-3)                        # the batch made after the failures works
    bat.close()
    n_pipe, pipe = _sweep(lambda: Pipe(warm, hosts, groups=2, autotune=False))
    assert n_pipe >= len(grids) + 8
    pipe.rk3_step(1e-3)
    pipe.close()
    assert all(b.status() == B.FP_OK for b in warm)
    # nothing the failed creations allocated is still held (a context of the middle grid
    # alone holds several MiB; allow the allocator's page rounding)
    free1 = _free_bytes()
    for b in warm:
        b.close()
    assert abs(free1 - free0) <= 8 << 20, (free0, free1)
