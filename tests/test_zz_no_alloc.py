"""Allocation-free residual entry point (fp_rhs_noalloc), called through the C ABI.

Some callers cannot allocate device memory where they evaluate a residual: a framework
that hands out device memory only from a pool reserved up front, a loop under a fixed
device-memory budget, a real-time loop that must not stall in the allocator.  For them
the residual accumulator lives in the library's static device scratch, which the
fp_init_grid of the context set up.  The result must be that of the regular fp_rhs
entry point bit for bit (same kernels, same data), on two calls in a row, with local
and global Lax-Friedrichs speeds, in 3-D and 2-D, in both precisions; blocks beyond the
scratch are refused.  This file is collected last on purpose, so that a run stopping at
the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2101_05886_gb300 import binding as B  # noqa: E402
from paper_2101_05886_gb300 import inputs as I  # noqa: E402
from paper_2101_05886_gb300.solver import Block  # noqa: E402


def _grid(dims, M):
    if dims == 3:
        g = I.periodic_wavy_3d((27, 21, 19), L=10.0, amp=0.08, Gn=O.node_ghost(M))
        return g, I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0), [I.vortex_3d(g, mach=0.8, eps=5.0, L=10.0)]
    g = I.periodic_wavy_2d(40, L=10.0, amp=0.1, Gn=O.node_ghost(M))
    qinf = I.uniform_qinf(0.5, 0.0, rho=1.0, p=1.0)
    return g, qinf, [I.shu_vortex(*g.interior_xyz(), 0.0, 5.0, 5.0, eps=5.0, mach=0.5, L=10.0)]


@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("global_lf", [0, 1])
@pytest.mark.parametrize("precision", [B.FP_F64, B.FP_F32_MIXED])
def test_noalloc_rhs_equals_fp_rhs_on_two_calls(precision, global_lf, dims):
    M = 6
    g, qinf, states = _grid(dims, M)
    states.append(I.random_smooth_state(g, qinf, amp=0.05, seed=11))
    blk = Block(g, metric_order=M, precision=precision, q_inf=qinf, global_lf=global_lf)
    stream = torch.cuda.current_stream().cuda_stream
    for q in states:                       # two calls in a row, different inputs
        qd = blk.to_device(q)
        ref = blk.rhs(qd)
        out = torch.full_like(qd, float("nan"))
        st = B.lib().fp_rhs_noalloc(blk.ctx, ctypes.c_void_p(qd.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == B.FP_OK, B.lib().fp_last_error(blk.ctx)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    blk.close()


def test_noalloc_rejects_blocks_beyond_the_static_scratch():
    M = 2
    g = I.periodic_wavy_3d((64, 64, 64), L=10.0, amp=0.08, Gn=O.node_ghost(M))   # 262,144 points
    blk = Block(g, metric_order=M, precision=B.FP_F64, q_inf=I.uniform_qinf(0.5, 0.0))
    q = blk.to_device(I.uniform_state(g, I.uniform_qinf(0.5, 0.0)))
    out = torch.empty_like(q)
    st = B.lib().fp_rhs_noalloc(blk.ctx, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == B.FP_ERR_ARG
    assert b"static scratch" in B.lib().fp_last_error(blk.ctx)
    blk.close()
