"""Shared helpers of the GPU tests: parity metric and sub-box oracle evaluation."""
import numpy as np

import oracle as O


FLOOR_FRAC = 1e-1


def rel_err(gpu, ora, floor_frac=FLOOR_FRAC, per_component=False):
    """Parity metric: per component c, max |gpu - oracle| / max(max |oracle_c|, tau) with
    tau = floor_frac * max over components of max |oracle| (10 % by default).  The
    characteristic projection mixes the components, so their round-off shares the
    scale of the largest one; a component whose residual is below 10 % of it is a
    cancellation remainder (rho w of a flow that is planar up to the grid's
    waviness falls like the truncation error as the grid is refined) and is
    judged against 10 % of the largest component instead of its own vanishing
    scale."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ora = np.asarray(ora, dtype=np.float64)
    tau = floor_frac * np.abs(ora).max()
    errs = []
    for c in range(ora.shape[0]):
        scale = max(np.abs(ora[c]).max(), tau)
        errs.append(np.abs(gpu[c] - ora[c]).max() / scale if scale > 0 else np.abs(gpu[c]).max())
    return errs if per_component else max(errs)


def ulp_sensitivity(cfg, met, q, draws=3, seed=0):
    """Conditioning of the residual at q: the largest parity metric between the
    oracle's dq/dt at q and at q with every entry moved by one unit in the last
    place (random sign), over a few draws.  Two correct FP64 evaluations that round
    differently can disagree by about this much; WENO7-JS, whose nonlinear weights
    react to smoothness indicators with coefficients up to 5188/240, is about a
    hundred times more sensitive than WENO5-JS on the same input."""
    _, d0 = O.rhs(cfg, met, q)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(draws):
        qp = q * (1.0 + np.finfo(np.float64).eps * rng.choice([-1.0, 1.0], size=q.shape))
        _, d1 = O.rhs(cfg, met, qp)
        worst = max(worst, rel_err(d1, d0))
    return worst


def oracle_subbox_dqdt(grid, q, M, lo, size, scheme=0, fp=1, charwise=1, gamma=1.4, qinf=None):
    """dQ/dt of the oracle on an interior sub-box [lo, lo+size) of a 3-D grid.

    The residual at a point depends only on states within G points and on node
    coordinates within G + 3M/2 points, so running the oracle on the sub-box grown
    by G (any boundary treatment) reproduces the full-grid values on the inner box.
    """
    G = O.ghost(M)
    Gn = O.node_ghost(M)
    lo = np.asarray(lo)
    size = np.asarray(size)
    a = lo - G
    b = lo + size + G
    n = np.asarray(grid.n)
    assert (a >= 0).all() and (b <= n).all(), "sub-box must be interior"
    assert grid.Gn >= Gn
    g0 = grid.Gn
    nodes = grid.nodes[:, a[2] - Gn + g0:b[2] + Gn + g0, a[1] - Gn + g0:b[1] + Gn + g0,
                       a[0] - Gn + g0:b[0] + Gn + g0]
    qs = np.ascontiguousarray(q[:, a[2]:b[2], a[1]:b[1], a[0]:b[0]], dtype=np.float64)
    sub_n = tuple(int(v) for v in (b - a))
    cfg = O.make_cfg(3, sub_n, M=M, scheme=scheme, fp=fp, charwise=charwise,
                     bc=((2, 2), (2, 2), (2, 2)), gamma=gamma,
                     qinf=qinf if qinf is not None else (1.4, 0, 0, 0, 2.5))
    met = O.metrics(cfg, np.ascontiguousarray(nodes), Gn)
    _, dq = O.rhs(cfg, met, qs)
    return dq[:, G:-G, G:-G, G:-G]
