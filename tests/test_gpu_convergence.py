"""Design order on the GPU: the 2-D isentropic vortex convected for one period over the periodic
wavy grid (amplitude 0.1, domain [0, 10]^2; vortex strength 5, Mach 0.5 mean flow), FP64, the
FP form, RK3 steps through the C ABI, the L2 density error against the closed form (the
initial vortex translated by one period, i.e. returned to its start).

Sec. 4.1.2 and Table 2: with metrics of the scheme's order (M6) the FP form converges at the
scheme's order (linear upwind: 5; WENO5-JS: high order, reduced by its nonlinear weights on
coarse grids), and 2nd-order metrics (M2) limit the order to 2.  The bounds are those claims;
no expected value comes from this code.  The time steps shrink with h^(5/3) between the M6
grids, so that the third-order time error falls by 2^5 with the spatial one; M2 takes the same
time step on both grids (its spatial error is far above the time error)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_2101_05886_gb300 import binding as B  # noqa: E402
from paper_2101_05886_gb300 import inputs as I  # noqa: E402
from paper_2101_05886_gb300.solver import Block  # noqa: E402

L_BOX = 10.0
PERIOD = L_BOX / (0.5 * math.sqrt(I.GAMMA))      # the mean flow crosses the box once


def _density_error(n, M, scheme, dt):
    g = I.periodic_wavy_2d(n, L=L_BOX, amp=0.1, Gn=I.node_ghost_width(M, scheme))
    x, y = g.interior_xyz()
    q0 = I.shu_vortex(x, y, 0.0, 5.0, 5.0, eps=5.0, mach=0.5, L=L_BOX)
    qinf = I.uniform_qinf(0.5, 0.0, rho=1.0, p=1.0)
    blk = Block(g, metric_order=M, scheme=scheme, precision=B.FP_F64, q_inf=qinf)
    q = blk.to_device(q0)
    steps = int(round(PERIOD / dt))
    h = PERIOD / steps
    assert blk.cfl_dt(q, 0.8) > h                 # a stable step at every resolution
    for _ in range(steps):
        blk.rk3_step(q, h)
    torch.cuda.synchronize()
    assert blk.status() == B.FP_OK
    rho = q.cpu().numpy()[0]
    blk.close()
    exact = I.shu_vortex(x, y, PERIOD, 5.0, 5.0, eps=5.0, mach=0.5, L=L_BOX)[0]
    return float(np.sqrt(np.mean((rho - exact) ** 2)))


def test_one_period_of_the_vortex_converges_at_design_order():
    dt64 = 0.01
    dt128 = dt64 / 2.0 ** (5.0 / 3.0)
    lu6 = [_density_error(64, 6, B.FP_LINEAR_UPWIND5, dt64), _density_error(128, 6, B.FP_LINEAR_UPWIND5, dt128)]
    w6 = [_density_error(64, 6, B.FP_WENO5_JS, dt64), _density_error(128, 6, B.FP_WENO5_JS, dt128)]
    dt2 = 0.0025                                  # CFL about 0.6 on the 256^2 wavy grid
    w2 = [_density_error(128, 2, B.FP_WENO5_JS, dt2), _density_error(256, 2, B.FP_WENO5_JS, dt2)]
    rate = lambda e: math.log2(e[0] / e[1])
    msg = {"LU5-M6": lu6, "WENO5-M6": w6, "WENO5-M2": w2}
    assert 4.0 < rate(lu6) < 6.0, msg
    assert rate(w6) > 3.0, msg
    assert 1.6 < rate(w2) < 2.4, msg
    assert w6[1] < w2[0] and lu6[1] < w2[0], msg     # consistent M6 metrics beat M2 at 128^2
