"""Allocation-free residual entry point (fp_rhs_noalloc), called through the C ABI.

For callers that cannot allocate device memory where they step: the residual
accumulator lives in the library's static device scratch.  Checked against the
regular fp_rhs entry point on two calls in a row, and for the size limit.  This
file is collected last on purpose."""
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
from tests.helpers import rel_err  # noqa: E402


@pytest.mark.parametrize("precision,tol", [(B.FP_F64, 1e-12), (B.FP_F32_MIXED, 1e-5)])
def test_noalloc_rhs_matches_fp_rhs_on_two_calls(precision, tol):
    M = 6
    g = I.periodic_wavy_3d((27, 21, 19), L=10.0, amp=0.08, Gn=O.node_ghost(M))
    qinf = I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0)
    blk = Block(g, metric_order=M, precision=precision, q_inf=qinf)
    stream = torch.cuda.current_stream().cuda_stream
    states = [I.vortex_3d(g, mach=0.8, eps=5.0, L=10.0),
              I.random_smooth_state(g, qinf, amp=0.05, seed=11)]
    for q in states:                       # two calls in a row, different inputs
        qd = blk.to_device(q)
        ref = blk.rhs(qd)
        out = torch.empty_like(qd)
        st = B.lib().fp_rhs_noalloc(blk.ctx, ctypes.c_void_p(qd.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == B.FP_OK, B.lib().fp_last_error(blk.ctx)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) <= tol
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
