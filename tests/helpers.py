"""Shared helpers of the GPU tests: the parity metric and sub-box oracle evaluation.

Parity metric (per residual component c, on the flux-difference residual
R = sum_d (F'_{d,i+1/2} - F'_{d,i-1/2}) of Eq. aderivative, Delta xi = 1):

    err_c = max_points |R_gpu,c - R_oracle,c| / max(max_points |R_oracle,c|, tau_c),
    tau_c = 1e-3 * max over points and swept directions of |F~_c|,

F~ = k . (F, G, H)(Q) the contravariant flux of Eq. FGH.  The floor tau_c only
matters for residual fields that are near zero (a free stream, a component that
a flow leaves untouched): there the error is judged against a thousandth of the
flux that the component carries.  The CUDA path returns dQ/dt = -J R, so its R is
recovered as -dQ/dt (1/J) with the oracle's 1/J.

FP32 inputs: the FP32 form holds its state, and with it the far-field state
q_inf that boundary ghosts take, as float values.  Parity of the FP32 form is
measured on inputs that are float-representable on both sides (state and q_inf,
see `f32`), so that both evaluate the same discrete problem.
"""
import numpy as np

import oracle as O


def f32(x):
    """The float-rounded value of x (array or sequence), as float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _interior(met, n, dims):
    """Interior view [..][nk][nj][ni] of a ghosted oracle array [..][nk+2G][nj+2G][ni+2G]."""
    ni, nj, nk = n
    G = (met.shape[-1] - ni) // 2
    ks = slice(None) if dims == 2 else slice(G, G + nk)
    return met[..., ks, G:G + nj, G:G + ni]


def flux_scale(met, q, dims, gamma=1.4):
    """Per component: max over interior points and swept directions d of |k_d . F(Q)|_c
    (the contravariant flux F~ of Eq. FGH with the oracle's cell metrics k_d)."""
    q = np.asarray(q, dtype=np.float64)
    n = (q.shape[3], q.shape[2], q.shape[1])
    m = _interior(met, n, dims)
    rho = q[0]
    u, v, w = q[1] / rho, q[2] / rho, q[3] / rho
    p = (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w))
    out = np.zeros(5)
    for d in range(dims):
        k = m[3 * d:3 * d + 3]
        U = u * k[0] + v * k[1] + w * k[2]
        F = (rho * U, q[1] * U + p * k[0], q[2] * U + p * k[1], q[3] * U + p * k[2], (q[4] + p) * U)
        out = np.maximum(out, [np.abs(f).max() for f in F])
    return out


def residual_err(R_gpu, R_ora, tau, per_component=False):
    """err_c = max |R_gpu,c - R_ora,c| / max(max |R_ora,c|, tau_c) (see the module docstring)."""
    R_gpu = np.asarray(R_gpu, dtype=np.float64)
    R_ora = np.asarray(R_ora, dtype=np.float64)
    errs = []
    for c in range(R_ora.shape[0]):
        scale = max(np.abs(R_ora[c]).max(), tau[c])
        diff = np.abs(R_gpu[c] - R_ora[c]).max()
        errs.append(diff / scale if scale > 0 else diff)   # a component that is zero on both sides
    return errs if per_component else max(errs)


class Parity:
    """The oracle's residual of one configuration, and the parity metric of a GPU dQ/dt
    against it."""

    def __init__(self, cfg, met, q, gamma=1.4):
        self.R, self.dq = O.rhs(cfg, met, q)
        self.invJ = _interior(met[9], tuple(cfg.n), cfg.dims)
        self.tau = 1e-3 * flux_scale(met, q, cfg.dims, gamma)

    def err(self, dq_gpu, per_component=False):
        R_gpu = -np.asarray(dq_gpu, dtype=np.float64) * self.invJ
        return residual_err(R_gpu, self.R, self.tau, per_component)


def rhs_err(dq_gpu, cfg, met, q, per_component=False):
    """Parity metric of a GPU dQ/dt against the oracle on the same inputs."""
    return Parity(cfg, met, q).err(dq_gpu, per_component)


def state_err(a, b, floor_frac=1e-3, per_component=False):
    """Per component max |a - b| / max(max |b_c|, floor_frac * max over components of max |b|):
    for comparing state increments (Q after steps minus Q before) of two evaluations."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    floor = floor_frac * np.abs(b).max()
    errs = []
    for c in range(b.shape[0]):
        scale = max(np.abs(b[c]).max(), floor)
        errs.append(np.abs(a[c] - b[c]).max() / scale if scale > 0 else np.abs(a[c]).max())
    return errs if per_component else max(errs)


def ulp_sensitivity(cfg, met, q, draws=3, seed=0):
    """Conditioning of the residual at q: the largest parity metric between the
    oracle's residual at q and at q with every entry moved by one unit in the last
    place (random sign), over a few draws.  Two correct FP64 evaluations that round
    differently can disagree by about this much; WENO7-JS, whose nonlinear weights
    react to smoothness indicators with coefficients up to 5188/240, is about a
    hundred times more sensitive than WENO5-JS on the same input."""
    P = Parity(cfg, met, q)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(draws):
        qp = q * (1.0 + np.finfo(np.float64).eps * rng.choice([-1.0, 1.0], size=q.shape))
        R1, _ = O.rhs(cfg, met, qp)
        worst = max(worst, residual_err(R1, P.R, P.tau))
    return worst


def oracle_subbox(grid, q, M, lo, size, scheme=0, fp=1, charwise=1, gamma=1.4, qinf=None):
    """The oracle on an interior sub-box [lo, lo+size) of a 3-D grid: returns (R, dQ/dt,
    1/J, tau) on the inner box, tau the parity floor of the sub-box's flux scale.

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
    R, dq = O.rhs(cfg, met, qs)
    inner = (slice(None), slice(G, -G), slice(G, -G), slice(G, -G))
    invJ = _interior(met[9], sub_n, 3)[G:-G, G:-G, G:-G]
    tau = 1e-3 * flux_scale(met[:, G:-G, G:-G, G:-G], qs[inner], 3, gamma)
    return R[inner], dq[inner], invJ, tau


def subbox_err(dq_gpu_box, grid, q, M, lo, size, qinf=None, **kw):
    """Parity metric of a GPU dQ/dt on a sub-box against the oracle on that sub-box."""
    R, _, invJ, tau = oracle_subbox(grid, q, M, lo, size, qinf=qinf, **kw)
    return residual_err(-np.asarray(dq_gpu_box, dtype=np.float64) * invJ, R, tau)


def subbox_sensitivity(grid, q, M, lo, size, qinf=None, draws=3, seed=0, **kw):
    """ulp_sensitivity of the oracle on a sub-box: the largest parity metric between its
    residual at q and at q with every entry moved by one unit in the last place."""
    R, _, _, tau = oracle_subbox(grid, q, M, lo, size, qinf=qinf, **kw)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(draws):
        qp = q * (1.0 + np.finfo(np.float64).eps * rng.choice([-1.0, 1.0], size=q.shape))
        R1, _, _, _ = oracle_subbox(grid, qp, M, lo, size, qinf=qinf, **kw)
        worst = max(worst, residual_err(R1, R, tau))
    return worst
