"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (Tables 1 and 2), closed forms (exact metrics on affine grids, the
closed-form time derivative of a translating vortex), invariants (the discrete
surface conservation law, telescoping of the flux difference, L R = I, A r = lambda r),
and identities the paper states (Remark 1, the linear-upwind / WENO relation of
the Appendix, the central-plus-dissipation form of Sec. 3.1).
"""
import numpy as np
import pytest

import oracle as O
from paper_2101_05886_gb300 import inputs as I
from tests.conftest import read_golden

GAMMA = 1.4


# ---------------------------------------------------------------- helpers
def euler_flux_k(Q, k, gamma=GAMMA):
    """(k_x F + k_y G + k_z H)(Q) from the definitions of Sec. 2.1 (test-side copy)."""
    rho = Q[0]
    u = Q[1] / rho
    v = Q[2] / rho
    w = Q[3] / rho
    p = (gamma - 1) * (Q[4] - 0.5 * rho * (u * u + v * v + w * w))
    U = k[0] * u + k[1] * v + k[2] * w
    return np.array([rho * U, Q[1] * U + p * k[0], Q[2] * U + p * k[1], Q[3] * U + p * k[2],
                     (Q[4] + p) * U])


def central_deriv(f, M, axis):
    """Order-M central derivative D = I(f)_{+1/2} - I(f)_{-1/2} along `axis`, valid
    on the points at least M/2 away from the array ends (returned array is cropped)."""
    c = O.interp_coef(M)
    h = M // 2
    n = f.shape[axis]
    # D_p = sum_m c_m (f_{p-h+1+m} - f_{p-h+m}), p = h .. n-h-1
    idx = np.arange(h, n - h)
    out = np.zeros(tuple(len(idx) if a == axis else f.shape[a] for a in range(f.ndim)))
    for m in range(M):
        out = out + c[m] * (np.take(f, idx - h + 1 + m, axis=axis) - np.take(f, idx - h + m, axis=axis))
    return out


def crop(a, axis, h):
    sl = [slice(None)] * a.ndim
    sl[axis] = slice(h, a.shape[axis] - h)
    return a[tuple(sl)]


# ---------------------------------------------------------------- stencils
@pytest.mark.parametrize("M", [2, 4, 6, 8])
def test_midpoint_weights_give_an_order_M_derivative(M):
    """Eq. (metric_discret): the weights sum to one and (dx/dxi)_i = x_{i+1/2} - x_{i-1/2}
    is an order-M central derivative.  Applied to cell averages the same weights give
    the face value of the primitive function at order M (they are not point
    interpolants of order M: on point values they are second order)."""
    c = O.interp_coef(M)
    assert abs(c.sum() - 1.0) < 1e-15
    errs_d, errs_a = [], []
    for n in (16, 32):
        h = 2 * np.pi / n
        x = np.arange(-M, n + M) * h
        f = np.sin(x)
        fbar = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h
        i = np.arange(M, n + M - M // 2)
        face = lambda g, j: sum(c[m] * g[j - M // 2 + 1 + m] for m in range(M))
        errs_d.append(np.abs(face(f, i) - face(f, i - 1) - h * np.cos(x[i])).max() / h)
        errs_a.append(np.abs(face(fbar, i) - np.sin(x[i] + 0.5 * h)).max())
    assert abs(np.log2(errs_d[0] / errs_d[1]) - M) < 0.3
    assert abs(np.log2(errs_a[0] / errs_a[1]) - M) < 0.3


def test_lu5_is_weno_with_optimal_weights_and_matches_the_printed_stencil():
    """Appendix (Eq. new_form_linear_upwind) and Eq. (linear_upwind): the optimal-weight
    WENO equals (2,-13,47,27,-3)/60.  This pins the first sub-stencil coefficients
    (1/3, -7/6, 11/6): the printed 7/6 for f_i would not reproduce it."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        v = rng.standard_normal(5)
        ref = (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60.0
        assert abs(O.lu5(v) - ref) <= 1e-15 * (1 + np.abs(v).sum())


def test_weno5_fifth_order_on_smooth_data_and_weights_tend_to_optimal():
    errs_w, errs_l = [], []
    for n in (32, 64, 128):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        cellavg = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h     # averages of sin
        e_w = e_l = 0.0
        for i in range(2, n - 2):
            v = cellavg[i - 2:i + 3]
            exact = np.sin(x[i] + h / 2)
            e_w = max(e_w, abs(O.weno5(v) - exact))
            e_l = max(e_l, abs(O.lu5(v) - exact))
        errs_w.append(e_w)
        errs_l.append(e_l)
    assert np.log2(errs_l[1] / errs_l[2]) > 4.7
    assert np.log2(errs_w[1] / errs_w[2]) > 4.5
    assert errs_w[2] < 10 * errs_l[2]      # WENO-JS loses some accuracy at critical points


def _parabola_through_cell_averages(vals, cells):
    """p(x) = a0 + a1 x + a2 x^2 whose averages over [c - 1/2, c + 1/2] are vals (h = 1)."""
    A = np.array([[((c + 0.5) ** (j + 1) - (c - 0.5) ** (j + 1)) / (j + 1) for j in range(3)] for c in cells])
    return np.polynomial.Polynomial(np.linalg.solve(A, vals))


def test_weno5_smoothness_indicators_and_face_values_follow_their_definitions():
    """Sec. 2.2.2, Eqs. weno and weno_wights: sub-stencil k covers the cells i-2+k .. i+k;
    q_k is the value at the face i+1/2 of the parabola whose cell averages there are the
    data, and beta_k = sum_{l=1,2} int_{cell i} h^(2l-1) (p_k^(l))^2 (Jiang & Shu's
    definition, h = 1).  Evaluated here by an independent least-squares-free solve and
    exact polynomial integration, so a swapped 1/4 <-> 13/12, a wrong sign inside a
    square or a shifted sub-stencil fails."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        v = rng.standard_normal(5)
        q, beta = O.weno5_parts(v)
        for k in range(3):
            cells = np.arange(k - 2, k + 1)
            p = _parabola_through_cell_averages(v[cells + 2], cells)
            b = 0.0
            for l in (1, 2):
                it = (p.deriv(l) ** 2).integ()
                b += it(0.5) - it(-0.5)
            assert abs(b - beta[k]) <= 1e-12 * (1 + abs(b)), (k, b, beta[k])
            assert abs(p(0.5) - q[k]) <= 1e-13 * (1 + np.abs(v).sum()), (k, p(0.5), q[k])


@pytest.mark.parametrize("s", [1.0, 1e-3])
def test_weno5_weights_use_epsilon_1e6_and_power_2(s):
    """A step in the last value, v = s (0, 0, 0, 0, 1): beta = (0, 0, 4/3 s^2) and
    q = (0, 0, -s/6), so the WENO5-JS value is -(s/6) w_2 with
    w_2 = [0.3/(4/3 s^2 + eps)^2] / [0.1/eps^2 + 0.6/eps^2 + 0.3/(4/3 s^2 + eps)^2].
    With s = 1 the value is about -4e-14 and scales with eps^2; with s = 1e-3 the indicator
    is of the size of eps and w_2 = 0.073.  Either fails for another eps or power."""
    eps = 1e-6
    a2 = 0.3 / (4.0 / 3.0 * s * s + eps) ** 2
    w2 = a2 / (0.7 / eps ** 2 + a2)
    ref = -(s / 6.0) * w2
    got = O.weno5([0.0, 0.0, 0.0, 0.0, s])
    assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
    for wrong_eps, power in ((1e-5, 2), (1e-7, 2), (1e-6, 1)):
        a2w = 0.3 / (4.0 / 3.0 * s * s + wrong_eps) ** power
        other = -(s / 6.0) * a2w / (0.7 / wrong_eps ** power + a2w)
        assert abs(other - ref) > 1e-3 * abs(ref)      # the pin discriminates


def test_weno5_is_non_oscillatory_across_a_step():
    # the upwind-biased reconstruction at i+1/2 with a jump between i and i+1 keeps the left value
    assert abs(O.weno5([0.0, 0.0, 0.0, 1.0, 1.0])) < 1e-10
    assert abs(O.weno5([1.0, 1.0, 1.0, 0.0, 0.0]) - 1.0) < 1e-10
    # linear upwind oscillates there
    assert abs(O.lu5([0.0, 0.0, 0.0, 1.0, 1.0]) - 0.4) < 1e-15


# ---------------------------------------------------------------- eigensystem
def _random_state(rng, mach=None):
    rho = rng.uniform(0.5, 2.0)
    p = rng.uniform(0.5, 2.0)
    u = rng.standard_normal(3) * (mach if mach is not None else 1.0)
    E = p / (GAMMA - 1) + 0.5 * rho * (u @ u)
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2], E])


@pytest.mark.parametrize("case", ["random", "z-normal", "2d-normal", "switch-boundary"])
def test_eigensystem_inverse_and_eigenpairs_of_the_flux_jacobian(case):
    rng = np.random.default_rng(hash(case) % 2**32)
    for _ in range(20):
        Q = _random_state(rng)
        if case == "random":
            k = rng.standard_normal(3) * rng.uniform(0.1, 10)
        elif case == "z-normal":
            k = np.array([1e-3, -2e-3, 1.0]) * rng.uniform(0.1, 10)
        elif case == "2d-normal":
            k = np.array([rng.standard_normal(), rng.standard_normal(), 0.0])
        else:
            t = rng.uniform(0, 2 * np.pi)
            k = np.array([np.cos(t) / np.sqrt(2), np.sin(t) / np.sqrt(2), 1 / np.sqrt(2) * (1 + 1e-12)])
        # equal left/right states: the Roe average is the state itself
        L, R = O.eigensystem(Q, Q, k)
        assert np.abs(L @ R - np.eye(5)).max() < 1e-12
        # A = d(F.n)/dQ by complex step, n = k/|k|; A r_s = lambda_s r_s
        n = k / np.linalg.norm(k)
        A = np.zeros((5, 5))
        for c in range(5):
            dq = np.zeros(5, dtype=complex)
            dq[c] = 1e-30j
            A[:, c] = np.imag(euler_flux_k(Q + dq, n)) / 1e-30
        rho = Q[0]
        u = Q[1:4] / rho
        p = (GAMMA - 1) * (Q[4] - 0.5 * rho * (u @ u))
        cs = np.sqrt(GAMMA * p / rho)
        U = u @ n
        lam = np.array([U - cs, U, U, U, U + cs])
        for s in range(5):
            r = R[:, s]
            assert np.abs(A @ r - lam[s] * r).max() < 1e-10 * (1 + np.abs(r).max() * (abs(U) + cs))
        if case == "2d-normal":
            # the second shear vector is the pure z-momentum field: 2-D flows keep w = 0
            assert np.abs(R[[0, 1, 2], 3]).max() == 0.0 and abs(R[3, 3] - 1) < 1e-15


# ---------------------------------------------------------------- metrics
@pytest.mark.parametrize("M", [2, 4, 6, 8])
def test_metrics_exact_on_power_of_two_cartesian_grid(M):
    Gn = O.node_ghost(M)
    g = I.cartesian_3d((6, 5, 7), 0.25, Gn)
    met = O.metrics(O.cfg_for(g, M=M), g.nodes, Gn)
    exp = np.zeros(10)
    exp[[0, 4, 8]] = 0.25 ** 2
    exp[9] = 0.25 ** 3
    for t in range(10):
        assert np.array_equal(met[t], np.full(met[t].shape, exp[t]))


@pytest.mark.parametrize("M", [2, 4, 6, 8])
def test_metrics_are_the_cofactor_matrix_on_an_affine_grid(M):
    """x = A xi + b: the metrics are the cofactors (xi_a/J = (adj A)_{d,a}) and 1/J = det A."""
    rng = np.random.default_rng(M)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    Gn = O.node_ghost(M)
    n = (5, 6, 4)
    KK, JJ, II = np.meshgrid(*[np.arange(-Gn, nn + Gn, dtype=float) for nn in n[::-1]], indexing="ij")
    xi = np.stack([II, JJ, KK])
    nodes = np.einsum("ab,b...->a...", A, xi) + b[:, None, None, None]
    g = I.Grid(3, n, Gn, np.ascontiguousarray(nodes), ((0, 0),) * 3)
    met = O.metrics(O.cfg_for(g, M=M), g.nodes, Gn)
    detA = np.linalg.det(A)
    adj = np.linalg.inv(A) * detA      # row d = grad(xi_d) * det
    for d in range(3):
        for a in range(3):
            assert np.abs(met[3 * d + a] - adj[d, a]).max() < 1e-12
    assert np.abs(met[9] - detA).max() < 1e-12


@pytest.mark.parametrize("M", [2, 4, 6, 8])
def test_surface_conservation_law_holds_to_round_off(M):
    """Sec. 2.1 Eq. (SCL): I_a = sum_d (d_a/J)_d = 0 with the same order-M operator."""
    Gn = O.node_ghost(M)
    g = I.periodic_wavy_3d((10, 9, 8), L=1.0, amp=0.08, Gn=Gn)
    met = O.metrics(O.cfg_for(g, M=M), g.nodes, Gn)
    h = M // 2
    scale = np.abs(met[:9]).max()
    for a in range(3):
        Ia = 0.0
        for d in range(3):
            dd = central_deriv(met[3 * d + a], M, axis=2 - d)
            for ax in range(3):
                if ax != 2 - d:
                    dd = crop(dd, ax, h)
            Ia = Ia + dd
        assert np.abs(Ia).max() < 3e-15 * scale


@pytest.mark.parametrize("M", [2, 4, 6])
def test_metrics_converge_at_order_M_to_the_analytic_cofactors(M):
    errs = []
    for n in (16, 32):
        Gn = O.node_ghost(M)
        g = I.periodic_wavy_3d((n, n, n), L=1.0, amp=0.05, Gn=Gn)
        met = O.metrics(O.cfg_for(g, M=M), g.nodes, Gn)
        G = O.ghost(M)
        # analytic Jacobian matrix of x_a = xi'_a + amp s(xi', eta', zeta'), xi' = i/n
        idx = np.arange(n) / n
        Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
        sx, sy, sz = np.sin(2 * np.pi * X), np.sin(2 * np.pi * Y), np.sin(2 * np.pi * Z)
        cx, cy, cz = np.cos(2 * np.pi * X), np.cos(2 * np.pi * Y), np.cos(2 * np.pi * Z)
        ds = 0.05 * 2 * np.pi * np.stack([cx * sy * sz, sx * cy * sz, sx * sy * cz]) / n  # d s / d index
        Jm = np.empty((3, 3) + X.shape)   # Jm[a, d] = d x_a / d index_d
        for a in range(3):
            for d in range(3):
                Jm[a, d] = (1.0 / n if a == d else 0.0) + ds[d]
        Jm = np.moveaxis(Jm, (0, 1), (-2, -1))
        det = np.linalg.det(Jm)
        adj = np.linalg.inv(Jm) * det[..., None, None]
        core = (slice(G, -G),) * 3
        e = max(np.abs(met[3 * d + a][core] - adj[..., d, a]).max() for d in range(3) for a in range(3))
        e = max(e, np.abs(met[9][core] - det).max() * n)
        errs.append(e * n * n)          # metrics scale like h^2
    rate = np.log2(errs[0] / errs[1])
    assert rate > M - 0.4


def test_2d_metrics_equal_the_3d_operators_on_an_extruded_grid():
    M = 6
    Gn = O.node_ghost(M)
    g2 = I.wavy_sinsin_2d(n=12, Gn=Gn)
    g3 = I.extrude_2d(g2, nk=6, dz=0.5)
    m2 = O.metrics(O.cfg_for(g2, M=M), g2.nodes, Gn)
    m3 = O.metrics(O.cfg_for(g3, M=M), g3.nodes, Gn)
    G = O.ghost(M)
    k = G + 2
    for t in (0, 1, 3, 4):
        assert np.abs(m3[t][k] - 0.5 * m2[t][0]).max() < 1e-14
    assert np.abs(m3[9][k] - 0.5 * m2[9][0]).max() < 1e-14
    assert np.abs(m3[8][k] - m2[9][0]).max() < 1e-14     # zeta_z/J = 2-D area


# ---------------------------------------------------------------- free stream (Table 1)
@pytest.mark.parametrize("kind", ["wavy", "random"])
def test_table1_free_stream_preserved_only_with_fp(kind):
    rows = {r[0]: [float(x) for x in r[1:]] for r in read_golden("table1_free_stream.txt")}
    M = 6
    Gn = O.node_ghost(M)
    g = I.paper_wavy_2d(Gn=Gn) if kind == "wavy" else I.paper_random_2d(Gn=Gn)
    qinf = I.uniform_qinf(0.5, 0.0)
    out = {}
    for fp in (1, 0):
        cfg = O.cfg_for(g, M=M, fp=fp, qinf=qinf)
        met = O.metrics(cfg, g.nodes, Gn)
        q = I.uniform_state(g, qinf)
        for _ in range(100):                       # t = 20 with dt = 0.2
            q = O.rk3_step(cfg, met, q, 0.2)
        v = q[2] / q[0]
        out[fp] = (np.sqrt(np.mean(v * v)), np.abs(v).max())
    col = 0 if kind == "wavy" else 2
    paper_fp = rows["WENO5-M6"][col:col + 2]
    paper_plain = rows["WENO5"][col:col + 2]
    # FP: round-off level, same decade as the paper's WENO5-M6 entry
    assert out[1][0] < 10 * paper_fp[0] and out[1][1] < 10 * paper_fp[1]
    # plain WENO5: O(1e-2) like the paper's WENO5 entry (within a factor 10)
    assert paper_plain[0] / 10 < out[0][0] < paper_plain[0] * 10


@pytest.mark.parametrize("M", [2, 4, 6, 8])
@pytest.mark.parametrize("scheme", [0, 1])
def test_config1_free_stream_ten_steps(M, scheme):
    Gn = O.node_ghost(M)
    g = I.wavy_sinsin_2d(n=33, amp=0.1, jitter=0.01, seed=1, Gn=Gn)
    qinf = I.uniform_qinf(0.5, 30.0)
    cfg = O.cfg_for(g, M=M, scheme=scheme, qinf=qinf)
    met = O.metrics(cfg, g.nodes, Gn)
    q = I.uniform_state(g, qinf)
    dt = O.cfl_dt(cfg, met, q, 0.5)
    for _ in range(10):
        q = O.rk3_step(cfg, met, q, dt)
    drift = np.abs(q - q.mean(axis=(1, 2, 3), keepdims=True)).max() / np.abs(qinf).max()
    assert drift < 1e-13


def test_3d_free_stream_on_wavy_grid_fp_vs_plain():
    M = 4
    Gn = O.node_ghost(M)
    g = I.periodic_wavy_3d((10, 8, 9), amp=0.08, Gn=Gn)
    qinf = I.uniform_qinf(0.8, 20.0, 10.0)
    res = {}
    for fp in (1, 0):
        cfg = O.cfg_for(g, M=M, fp=fp, qinf=qinf)
        met = O.metrics(cfg, g.nodes, Gn)
        R, _ = O.rhs(cfg, met, I.uniform_state(g, qinf))
        res[fp] = np.abs(R).max() / np.abs(met[:9]).max()
    assert res[1] < 1e-14
    assert res[0] > 1e-6


# ---------------------------------------------------------------- identities
@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("M", [2, 6, 8])
def test_remark1_fp_recovers_plain_scheme_bitwise_on_cartesian_grid(dims, scheme, M):
    Gn = O.node_ghost(M)
    if dims == 2:
        g = I.cartesian_2d((10, 9), 0.125, Gn)
    else:
        g = I.cartesian_3d((9, 8, 8), 0.125, Gn)
    q = I.random_smooth_state(g, I.uniform_qinf(0.7, 25.0, 10.0 if dims == 3 else 0.0), amp=0.1, seed=3)
    R = {}
    for fp in (1, 0):
        cfg = O.cfg_for(g, M=M, scheme=scheme, fp=fp)
        met = O.metrics(cfg, g.nodes, Gn)
        R[fp] = O.rhs(cfg, met, q)[0]
    assert np.array_equal(R[1], R[0])


def test_my_point1_and_my_point2_forms_agree():
    """Eq. (my_point1) and Eq. (my_point2) differ only by moving the constant face flux
    inside WENO; they agree to round-off."""
    M = 6
    Gn = O.node_ghost(M)
    g = I.periodic_wavy_3d((8, 8, 8), amp=0.08, Gn=Gn)
    q = I.random_smooth_state(g, I.uniform_qinf(0.8, 10.0, 5.0), amp=0.05, seed=2)
    R = {}
    for form in (1, 2):
        cfg = O.cfg_for(g, M=M, form=form)
        met = O.metrics(cfg, g.nodes, Gn)
        R[form] = O.rhs(cfg, met, q)[0]
    scale = np.abs(R[2]).max(axis=(1, 2, 3), keepdims=True)
    assert np.abs(R[1] - R[2]).max() / scale.min() < 1e-12


@pytest.mark.parametrize("charwise", [1, 0])
def test_appendix_fp_linear_upwind_equals_central_plus_reformulated_dissipation(charwise):
    """Sec. 3.1 Eq. (final_form_linear_upwind), first line, with M6 metrics: the FP
    linear-upwind face flux is the 6th-order central flux of F~ plus the 5th-order
    dissipation of (Q~ - Q*/J) in characteristic space (F^ of Eq. WENO_hatF is zero).
    Component-wise splitting (charwise = 0) is the same with one speed, the largest
    |U -+ c|grad|| over the stencil, for every component and no projection."""
    rng = np.random.default_rng(11)
    cfg = O.make_cfg(3, (8, 8, 8), M=6, scheme=1, fp=1, charwise=charwise)
    c6 = np.array([1, -8, 37, 37, -8, 1]) / 60.0
    d5 = np.array([1, -5, 10, -10, 5, -1]) / 60.0
    for _ in range(20):
        base = _random_state(rng, mach=0.5)
        q8 = np.array([base * (1 + 0.05 * rng.standard_normal(5)) for _ in range(8)])
        q8[:, 0] = np.abs(q8[:, 0])
        met8 = np.empty((8, 4))
        k0 = rng.standard_normal(3)
        for m in range(8):
            met8[m, :3] = k0 + 0.1 * rng.standard_normal(3)
            met8[m, 3] = rng.uniform(0.5, 1.5)
        got = O.face_flux(cfg, q8, met8)
        st = slice(1, 7)                          # cells i-2 .. i+3
        invJ = met8[:, 3]
        Ft = np.array([euler_flux_k(q8[m], met8[m, :3]) for m in range(8)])
        Qt = q8 * invJ[:, None]
        invJf = c6 @ invJ[st]
        Qs = (c6 @ Qt[st]) / invJf                # Eq. (Q_star) with Eqs. (QdJ_star), (1dJ)
        kf = c6 @ met8[st, :3]
        L, R = O.eigensystem(q8[3], q8[4], kf)
        # LLF speeds: max over the stencil of |eigenvalues of dF~/dQ~|
        lam = np.zeros(5)
        for m in range(1, 7):
            rho = q8[m, 0]
            u = q8[m, 1:4] / rho
            p = (GAMMA - 1) * (q8[m, 4] - 0.5 * rho * (u @ u))
            cs = np.sqrt(GAMMA * p / rho)
            gvec = met8[m, :3] / invJ[m]
            U = u @ gvec
            a = cs * np.linalg.norm(gvec)
            lam = np.maximum(lam, np.abs([U - a, U, U, U, U + a]))
        central = c6 @ Ft[st]
        diffQ = (Qt - Qs[None, :] * invJ[:, None])[st]      # Q~_m - Q~*_m
        if charwise:
            diss = R @ (lam * (L @ (d5 @ diffQ)))
        else:
            diss = max(lam[0], lam[4]) * (d5 @ diffQ)
        ref = central + diss
        assert np.abs(got - ref).max() < 1e-12 * (1 + np.abs(ref).max())


@pytest.mark.parametrize("M", [2, 6])
def test_flux_difference_telescopes_on_periodic_grid(M):
    Gn = O.node_ghost(M)
    g = I.periodic_wavy_3d((8, 9, 10), amp=0.08, Gn=Gn)
    q = I.random_smooth_state(g, I.uniform_qinf(0.6, 30.0, 20.0), amp=0.05, seed=5)
    cfg = O.cfg_for(g, M=M)
    met = O.metrics(cfg, g.nodes, Gn)
    R = O.rhs(cfg, met, q)[0]
    tot = R.sum(axis=(1, 2, 3))
    assert np.abs(tot).max() < 1e-13 * np.abs(R).sum()


def test_xi_eta_swap_symmetry():
    M = 6
    Gn = O.node_ghost(M)
    g = I.periodic_wavy_2d(12, L=10.0, amp=0.1, Gn=Gn)
    q = I.shu_vortex(*g.interior_xyz(), 0.0, 5.0, 5.0, eps=5.0, mach=0.5, L=10.0)
    cfg = O.cfg_for(g, M=M)
    R = O.rhs(cfg, O.metrics(cfg, g.nodes, Gn), q)[0]
    # swapped grid: x<->y and i<->j; swapped state: u<->v and i<->j
    nodes_s = np.ascontiguousarray(np.stack([g.nodes[1].T, g.nodes[0].T]))
    gs = I.Grid(2, g.n, Gn, nodes_s, g.bc)
    qs = np.ascontiguousarray(np.stack([q[0], q[2], q[1], q[3], q[4]]).transpose(0, 1, 3, 2))
    Rs = O.rhs(cfg, O.metrics(cfg, gs.nodes, Gn), qs)[0]
    # swapping x<->y together with i<->j keeps the orientation, so R maps back unchanged
    Rback = np.stack([Rs[0], Rs[2], Rs[1], Rs[3], Rs[4]]).transpose(0, 1, 3, 2)
    assert np.abs(Rback - R).max() < 1e-12 * np.abs(R).max()


def test_periodic_boundary_commutes_with_index_shift():
    M = 6
    Gn = O.node_ghost(M)
    g = I.cartesian_2d((12, 10), 0.5, Gn)
    q = I.random_smooth_state(g, I.uniform_qinf(0.5, 10.0), amp=0.1, seed=1)
    cfg = O.cfg_for(g, M=M)
    met = O.metrics(cfg, g.nodes, Gn)
    R = O.rhs(cfg, met, q)[0]
    Rs = O.rhs(cfg, met, np.ascontiguousarray(np.roll(q, 3, axis=3)))[0]
    assert np.abs(np.roll(R, 3, axis=3) - Rs).max() < 1e-13 * np.abs(R).max()


def test_farfield_boundary_sees_q_inf():
    """With far-field ghosts equal to the interior uniform state, the residual is
    round-off; with a different q_inf the boundary columns feel it."""
    M = 2
    Gn = O.node_ghost(M)
    g = I.wavy_sinsin_2d(n=16, Gn=Gn)
    qinf = I.uniform_qinf(0.5, 30.0)
    q = I.uniform_state(g, qinf)
    cfg = O.cfg_for(g, M=M, qinf=qinf)
    met = O.metrics(cfg, g.nodes, Gn)
    assert np.abs(O.rhs(cfg, met, q)[1]).max() < 1e-11
    cfg2 = O.cfg_for(g, M=M, qinf=qinf * 1.01)
    R2 = O.rhs(cfg2, met, q)[1]
    assert np.abs(R2[:, :, 4:-4, 4:-4]).max() < 1e-11 and np.abs(R2).max() > 1e-4


# ---------------------------------------------------------------- order of accuracy
def _vortex_complex(x, y, eps=5.0, mach=0.5, gamma=GAMMA, xc=5.0, yc=5.0):
    uinf = mach * np.sqrt(gamma)
    dx, dy = x - xc, y - yc
    r2 = dx * dx + dy * dy
    f = eps / (2 * np.pi) * np.exp(0.5 * (1 - r2))
    u, v = uinf - f * dy, f * dx
    T = 1 - (gamma - 1) * eps * eps / (8 * gamma * np.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1 / (gamma - 1))
    p = rho * T
    E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, 0 * rho, E])


def _rhs_error(n, M, scheme):
    Gn = O.node_ghost(M)
    g = I.periodic_wavy_2d(n, L=10.0, amp=0.1, Gn=Gn)
    x, y = g.interior_xyz()
    q = I.shu_vortex(x, y, 0.0, 5.0, 5.0, eps=5.0, mach=0.5, L=10.0)
    cfg = O.cfg_for(g, M=M, scheme=scheme)
    L = O.rhs(cfg, O.metrics(cfg, g.nodes, Gn), q)[1]
    # closed form: the vortex translates, dQ/dt = -u_inf dQ/dx (complex-step derivative)
    exact = -0.5 * np.sqrt(GAMMA) * np.imag(_vortex_complex(x + 1e-30j, y)) / 1e-30
    core = ((x - 5) ** 2 + (y - 5) ** 2 < 3.5 ** 2)[None]
    return np.abs((L - exact) * core).max()


def test_design_order_linear_upwind_m6_and_metric_limited_m2():
    """Sec. 4.1.2 / Table 2: consistent orders reach the scheme's order; M2 metrics
    limit the order to 2 as the grid is refined."""
    e6 = [_rhs_error(n, 6, 1) for n in (128, 256)]
    e2 = [_rhs_error(n, 2, 1) for n in (128, 256)]
    w2 = [_rhs_error(n, 2, 0) for n in (128, 256)]
    assert 4.6 < np.log2(e6[0] / e6[1]) < 5.4
    assert 1.8 < np.log2(e2[0] / e2[1]) < 2.2
    assert 1.8 < np.log2(w2[0] / w2[1]) < 2.2


def test_table2_vortex_paper_setup_loose():
    """Table 2 magnitudes at 21 and 41 points (the grid closure and time step are not
    fully specified, so the check is loose: linear upwind within 30 %, WENO within 3x)."""
    rows = read_golden("table2_vortex.txt")
    ref = {(r[0], int(r[1])): (float(r[2]), float(r[3])) for r in rows}
    qinf = I.uniform_qinf(0.5, 0.0)
    for name, scheme, M, npts, dt, tol in (("Linear-Upwind5-M6", 1, 6, 21, 0.1, 1.3),
                                           ("Linear-Upwind5-M6", 1, 6, 41, 0.05, 1.3),
                                           ("WENO5-M6", 0, 6, 21, 0.1, 3.0),
                                           ("WENO5-M2", 0, 2, 21, 0.1, 3.0)):
        Gn = O.node_ghost(M)
        g = I.paper_wavy_2d(npts=npts, Gn=Gn)
        x, y = g.interior_xyz()
        q = I.paper_vortex(x, y, 0.0)
        cfg = O.cfg_for(g, M=M, scheme=scheme, qinf=qinf)
        met = O.metrics(cfg, g.nodes, Gn)
        for _ in range(int(round(40.0 / dt))):
            q = O.rk3_step(cfg, met, q, dt)
        qe = I.paper_vortex(x, y, 40.0)
        e2 = np.sqrt(np.mean((q[2] / q[0] - qe[2] / qe[0]) ** 2))
        p2 = ref[(name, npts)][0]
        assert p2 / tol < e2 < p2 * tol, (name, npts, e2, p2)


def test_rk3_is_third_order_in_time():
    M = 6
    Gn = O.node_ghost(M)
    g = I.periodic_wavy_2d(24, L=10.0, amp=0.1, Gn=Gn)
    x, y = g.interior_xyz()
    q0 = I.shu_vortex(x, y, 0.0, 5.0, 5.0, eps=5.0, mach=0.5, L=10.0)
    cfg = O.cfg_for(g, M=M, scheme=1)
    met = O.metrics(cfg, g.nodes, Gn)
    T = 0.4
    sols = []
    for nst in (4, 8, 16):
        q = q0.copy()
        for _ in range(nst):
            q = O.rk3_step(cfg, met, q, T / nst)
        sols.append(q)
    ratio = np.abs(sols[0] - sols[1]).max() / np.abs(sols[1] - sols[2]).max()
    assert 6.5 < ratio < 9.5


def test_cfl_dt_closed_form_on_cartesian_grid():
    M = 2
    Gn = O.node_ghost(M)
    h = 0.25
    g = I.cartesian_3d((6, 6, 6), h, Gn)
    qinf = I.uniform_qinf(0.8, 30.0, 10.0)
    cfg = O.cfg_for(g, M=M, qinf=qinf)
    met = O.metrics(cfg, g.nodes, Gn)
    rho = qinf[0]
    u = qinf[1:4] / rho
    c = 1.0
    expected = 0.7 / sum((abs(u[d]) + c) / h for d in range(3))
    assert abs(O.cfl_dt(cfg, met, I.uniform_state(g, qinf), 0.7) - expected) < 1e-14


def test_global_speeds_enter_the_dissipation_linearly():
    """With given (global) Lax-Friedrichs speeds the FP linear-upwind face flux is still
    the central flux plus the dissipation of Sec. 3.1 with those speeds: doubling the
    speeds doubles the difference to the central flux."""
    rng = np.random.default_rng(21)
    cfg = O.make_cfg(3, (8, 8, 8), M=6, scheme=1, fp=1)
    c6 = np.array([1, -8, 37, 37, -8, 1]) / 60.0
    base = _random_state(rng, mach=0.5)
    q8 = np.array([base * (1 + 0.05 * rng.standard_normal(5)) for _ in range(8)])
    q8[:, 0] = np.abs(q8[:, 0])
    met8 = np.empty((8, 4))
    k0 = rng.standard_normal(3)
    for m in range(8):
        met8[m, :3] = k0 + 0.1 * rng.standard_normal(3)
        met8[m, 3] = rng.uniform(0.5, 1.5)
    st = slice(1, 7)
    Ft = np.array([euler_flux_k(q8[m], met8[m, :3]) for m in range(8)])
    central = c6 @ Ft[st]
    lam = np.array([3.0, 2.0, 2.0, 2.0, 4.0])
    f1 = O.face_flux_lam(cfg, q8, met8, lam)
    f2 = O.face_flux_lam(cfg, q8, met8, 2 * lam)
    assert np.abs((f2 - central) - 2 * (f1 - central)).max() < 1e-12 * np.abs(central).max()


# ---------------------------------------------------------------- WENO7 (Remark 2)
def test_weno7_optimal_weights_give_the_7th_order_upwind_stencil():
    C = np.array([1, 12, 18, 4]) / 35.0
    rng = np.random.default_rng(3)
    for _ in range(20):
        v = rng.standard_normal(7)
        q, _ = O.weno7_parts(v)
        ref = (-3 * v[0] + 25 * v[1] - 101 * v[2] + 319 * v[3] + 214 * v[4] - 38 * v[5] + 4 * v[6]) / 420.0
        assert abs(C @ q - ref) < 1e-14 * (1 + np.abs(v).sum())


def test_weno7_smoothness_indicators_follow_the_integral_definition():
    """beta_k = sum_{l=1..3} int_{-1/2}^{1/2} (p_k^(l))^2 dx for the cubic p_k whose cell
    averages over the sub-stencil are the data (h = 1)."""
    rng = np.random.default_rng(4)
    v = rng.standard_normal(7)
    _, beta = O.weno7_parts(v)
    for k in range(4):
        cells = np.arange(k - 3, k + 1)
        # cell average of x^j over [c - 1/2, c + 1/2]
        A = np.array([[((c + 0.5) ** (j + 1) - (c - 0.5) ** (j + 1)) / (j + 1) for j in range(4)] for c in cells])
        a = np.linalg.solve(A, v[cells + 3])
        p = np.polynomial.Polynomial(a)
        b = 0.0
        for l in range(1, 4):
            dl = p.deriv(l) ** 2
            it = dl.integ()
            b += it(0.5) - it(-0.5)
        assert abs(b - beta[k]) < 1e-10 * (1 + abs(b))


def test_weno7_seventh_order_and_non_oscillatory():
    errs = []
    for n in (32, 64):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        cellavg = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h
        e = 0.0
        for i in range(3, n - 3):
            e = max(e, abs(O.weno7(cellavg[i - 3:i + 4]) - np.sin(x[i] + h / 2)))
        errs.append(e)
    assert np.log2(errs[0] / errs[1]) > 6.0
    assert abs(O.weno7([0, 0, 0, 0, 1, 1, 1])) < 1e-9


def test_table1_weno7_rows():
    rows = {r[0]: [float(x) for x in r[1:]] for r in read_golden("table1_free_stream.txt")}
    qinf = I.uniform_qinf(0.5, 0.0)
    for M, fp, key in ((6, 1, "WENO7-M6"), (8, 1, "WENO7-M8"), (6, 0, "WENO7")):
        Gn = O.node_ghost(M, 2)
        g = I.paper_wavy_2d(Gn=Gn)
        cfg = O.cfg_for(g, M=M, scheme=2, fp=fp, qinf=qinf)
        met = O.metrics(cfg, g.nodes, Gn)
        q = I.uniform_state(g, qinf)
        for _ in range(100):
            q = O.rk3_step(cfg, met, q, 0.2)
        v = q[2] / q[0]
        l2 = np.sqrt(np.mean(v * v))
        paper = rows[key][0]
        if fp:
            assert l2 < 10 * paper
        else:
            assert paper / 10 < l2 < paper * 10


def test_table2_weno7_m8_at_21_and_41_points():
    ref = {(r[0], int(r[1])): float(r[2]) for r in read_golden("table2_vortex.txt")}
    qinf = I.uniform_qinf(0.5, 0.0)
    M = 8
    Gn = O.node_ghost(M, 2)
    for npts, dt in ((21, 0.1), (41, 0.05)):
        g = I.paper_wavy_2d(npts=npts, Gn=Gn)
        x, y = g.interior_xyz()
        q = I.paper_vortex(x, y, 0.0)
        cfg = O.cfg_for(g, M=M, scheme=2, qinf=qinf)
        met = O.metrics(cfg, g.nodes, Gn)
        for _ in range(int(round(40.0 / dt))):
            q = O.rk3_step(cfg, met, q, dt)
        qe = I.paper_vortex(x, y, 40.0)
        e2 = np.sqrt(np.mean((q[2] / q[0] - qe[2] / qe[0]) ** 2))
        p2 = ref[("WENO7-M8", npts)]
        assert p2 / 1.3 < e2 < p2 * 1.3, (npts, e2, p2)


def test_weno7_m8_design_order_on_the_vortex():
    errs = []
    for n in (64, 128):
        Gn = O.node_ghost(8, 2)
        g = I.periodic_wavy_2d(n, L=10.0, amp=0.1, Gn=Gn)
        x, y = g.interior_xyz()
        q = I.shu_vortex(x, y, 0.0, 5.0, 5.0, eps=5.0, mach=0.5, L=10.0)
        cfg = O.cfg_for(g, M=8, scheme=2)
        L = O.rhs(cfg, O.metrics(cfg, g.nodes, Gn), q)[1]
        exact = -0.5 * np.sqrt(GAMMA) * np.imag(_vortex_complex(x + 1e-30j, y)) / 1e-30
        core = ((x - 5) ** 2 + (y - 5) ** 2 < 3.5 ** 2)[None]
        errs.append(np.abs((L - exact) * core).max())
    assert np.log2(errs[0] / errs[1]) > 6.5


@pytest.mark.parametrize("M", [4, 8])
def test_remark1_weno7_bitwise_on_cartesian_grid(M):
    Gn = O.node_ghost(M, 2)
    g = I.cartesian_3d((9, 8, 10), 0.125, Gn)
    q = I.random_smooth_state(g, I.uniform_qinf(0.7, 25.0, 10.0), amp=0.1, seed=3)
    R = {}
    for fp in (1, 0):
        cfg = O.cfg_for(g, M=M, scheme=2, fp=fp)
        R[fp] = O.rhs(cfg, O.metrics(cfg, g.nodes, Gn), q)[0]
    assert np.array_equal(R[1], R[0])


# ---------------------------------------------------------------- WENOCU6 (Remark 2)
def test_wenocu6_linear_weights_give_the_m6_central_face_value():
    """The linear weights (1, 9, 9, 1)/20 of the four parabolic sub-stencil values make the
    6-point central face value whose weights are the paper's sixth-order midpoint
    formula (1, -8, 37, 37, -8, 1)/60 (Sec. 3, Eq. metric_discret at M = 6)."""
    d = np.array([1, 9, 9, 1]) / 20.0
    m6 = np.array([1, -8, 37, 37, -8, 1]) / 60.0
    for j in range(6):
        e = np.zeros(6)
        e[j] = 1.0
        q, _, _ = O.wenocu6_parts(e)
        assert abs(d @ q - m6[j]) < 1e-15


def test_wenocu6_beta6_is_the_integral_definition_on_six_cells():
    """The downwind stencil's indicator is beta6 = sum_{l=1..5} int_{-1/2}^{1/2} (p^(l))^2
    for the quintic p whose averages over cells -2..3 are the data (h = 1); the three
    upwind indicators are those of WENO5-JS."""
    rng = np.random.default_rng(8)
    for _ in range(5):
        v = rng.standard_normal(6)
        _, beta, tau = O.wenocu6_parts(v)
        cells = np.arange(-2, 4)
        A = np.array([[((c + 0.5) ** (j + 1) - (c - 0.5) ** (j + 1)) / (j + 1) for j in range(6)] for c in cells])
        p = np.polynomial.Polynomial(np.linalg.solve(A, v))
        b6 = 0.0
        for l in range(1, 6):
            it = (p.deriv(l) ** 2).integ()
            b6 += it(0.5) - it(-0.5)
        assert abs(b6 - beta[3]) < 1e-9 * (1 + abs(b6))
        assert abs(tau - abs(beta[3] - (beta[0] + 4 * beta[1] + beta[2]) / 6)) < 1e-12 * (1 + abs(tau))


def test_wenocu6_sixth_order_and_non_oscillatory():
    errs = []
    for n in (32, 64):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        cellavg = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h
        e = 0.0
        for i in range(2, n - 3):
            e = max(e, abs(O.wenocu6(cellavg[i - 2:i + 4]) - np.sin(x[i] + h / 2)))
        errs.append(e)
    assert 5.5 < np.log2(errs[0] / errs[1]) < 6.6
    # a step: the face value stays within the data (no overshoot), on either side of the jump
    for k in range(1, 6):
        v = np.r_[np.zeros(k), np.ones(6 - k)]
        r = O.wenocu6(v)
        assert -1e-6 < r < 1 + 1e-6, (k, r)


def test_wenocu6_free_stream_and_remark1():
    """Under the FP form WENOCU6-M6 keeps a uniform stream on the Table 1 wavy grid at
    rounding level while the plain scheme does not; on a uniform Cartesian grid the FP
    form is the plain scheme bit for bit (Remark 1)."""
    qinf = I.uniform_qinf(0.5, 0.0)
    Gn = O.node_ghost(6)
    g = I.paper_wavy_2d(Gn=Gn)
    res = {}
    for fp in (1, 0):
        cfg = O.cfg_for(g, M=6, scheme=3, fp=fp, qinf=qinf)
        met = O.metrics(cfg, g.nodes, Gn)
        q = I.uniform_state(g, qinf)
        for _ in range(50):
            q = O.rk3_step(cfg, met, q, 0.2)
        res[fp] = np.sqrt(np.mean((q[2] / q[0]) ** 2))
    assert res[1] < 1e-14 and res[0] > 1e-4
    gc = I.cartesian_3d((9, 8, 10), 0.125, Gn)
    q = I.random_smooth_state(gc, I.uniform_qinf(0.7, 25.0, 10.0), amp=0.1, seed=3)
    R = {}
    for fp in (1, 0):
        cfg = O.cfg_for(gc, M=6, scheme=3, fp=fp)
        R[fp] = O.rhs(cfg, O.metrics(cfg, gc.nodes, Gn), q)[0]
    assert np.array_equal(R[1], R[0])


def test_wenocu6_m6_converges_on_the_vortex_once_resolved():
    """With its scale-free epsilon (1e-40) the WENOCU6 weights adapt on the small FP
    difference values near critical points, so on the vortex the residual error converges
    slowly on coarse grids (order 1.8 from 128^2 to 256^2) and reaches third order between
    256^2 and 512^2 on the way to the linear limit's sixth order (the linear weights alone
    give order 5.7 here).  Pinned: the error falls at third order or better once resolved."""
    errs = []
    for n in (256, 512):
        Gn = O.node_ghost(6)
        g = I.periodic_wavy_2d(n, L=10.0, amp=0.1, Gn=Gn)
        x, y = g.interior_xyz()
        q = I.shu_vortex(x, y, 0.0, 5.0, 5.0, eps=5.0, mach=0.5, L=10.0)
        cfg = O.cfg_for(g, M=6, scheme=3)
        L = O.rhs(cfg, O.metrics(cfg, g.nodes, Gn), q)[1]
        exact = -0.5 * np.sqrt(GAMMA) * np.imag(_vortex_complex(x + 1e-30j, y)) / 1e-30
        core = ((x - 5) ** 2 + (y - 5) ** 2 < 3.5 ** 2)[None]
        errs.append(np.abs((L - exact) * core).max())
    assert np.log2(errs[0] / errs[1]) > 2.8, errs


# ------------------------------------------- boundary rules: slip wall and C-grid cut
# Sec. 4.2 imposes slip walls (cylinder, airfoils) and uses C-type grids around airfoils
# without stating the discrete rule.  Reading: the wall (and the cut) is the boundary
# face; wall ghosts mirror the interior with the momentum reflected about that face's
# unit normal; cut ghosts are the cells across the cut, taken as they are.
def _mirror_doubled_state(q):
    """State on the mirror-doubled channel: rows nj..2nj-1 are q, rows nj-1..0 are q
    mirrored with the y momentum negated."""
    low = q[:, :, ::-1, :].copy()
    low[2] *= -1.0
    return np.ascontiguousarray(np.concatenate([low, q], axis=2))


@pytest.mark.parametrize("M,scheme,charwise", [(2, 0, 1), (6, 0, 1), (6, 1, 0), (8, 2, 1)])
def test_slip_walls_equal_the_mirror_doubled_periodic_channel(M, scheme, charwise):
    """Walls on both sides of a wavy channel whose map is mirror symmetric about both
    walls give the same residual as the doubled channel (periodic, state mirrored with
    v -> -v) on its upper half, and the mirrored residual on its lower half: brute
    force against the wall rule, including the normal taken from the face metric."""
    Gn = O.node_ghost(M, scheme)
    g1 = I.mirror_channel_2d((24, 16), Gn=Gn)
    g2 = I.mirror_channel_2d((24, 16), Gn=Gn, doubled=True)
    qinf = I.uniform_qinf(0.6, 20.0)
    q1 = I.random_smooth_state(g1, qinf, amp=0.05, seed=3)
    q2 = _mirror_doubled_state(q1)
    c1 = O.cfg_for(g1, M=M, scheme=scheme, charwise=charwise, qinf=qinf)
    c2 = O.cfg_for(g2, M=M, scheme=scheme, charwise=charwise, qinf=qinf)
    _, d1 = O.rhs(c1, O.metrics(c1, g1.nodes, Gn), q1)
    _, d2 = O.rhs(c2, O.metrics(c2, g2.nodes, Gn), q2)
    scale = np.abs(d1).max()
    assert np.abs(d2[:, :, 16:, :] - d1).max() <= 1e-12 * scale
    assert np.abs(_mirror_doubled_state(d1) - d2).max() <= 1e-12 * scale
    # the rule matters: a zero-gradient side gives a different residual
    c0 = O.cfg_for(g1, M=M, scheme=scheme, charwise=charwise, qinf=qinf)
    c0.bc[1][0] = I.BC_EXTRAP
    _, d0 = O.rhs(c0, O.metrics(c0, g1.nodes, Gn), q1)
    assert np.abs(d0 - d1).max() > 1e-3 * scale


def _transpose_2d(g, q):
    """The same 2-D problem with i <-> j and x <-> y swapped (orientation kept)."""
    nodes = np.ascontiguousarray(np.stack([g.nodes[1].T, g.nodes[0].T]))
    qt = np.ascontiguousarray(q.transpose(0, 1, 3, 2)[[0, 2, 1, 3, 4]])
    bc = (g.bc[1], g.bc[0], g.bc[2])
    return I.Grid(2, (g.n[1], g.n[0], 1), g.Gn, nodes, bc, g.name + "_T", g.cut), qt


def test_slip_walls_in_the_xi_direction_and_in_3d():
    """The wall rule in the i direction (transposed channel) and in 3-D (the channel
    extruded in z, with spanwise momentum): both equal the wall-in-j 2-D result."""
    M = 6
    Gn = O.node_ghost(M)
    g = I.mirror_channel_2d((20, 14), Gn=Gn)
    qinf = I.uniform_qinf(0.6, 20.0)
    q = I.random_smooth_state(g, qinf, amp=0.05, seed=5)
    c = O.cfg_for(g, M=M, qinf=qinf)
    _, d = O.rhs(c, O.metrics(c, g.nodes, Gn), q)
    gt, qt = _transpose_2d(g, q)
    ct = O.cfg_for(gt, M=M, qinf=qinf)
    _, dt = O.rhs(ct, O.metrics(ct, gt.nodes, Gn), qt)
    assert np.abs(dt.transpose(0, 1, 3, 2)[[0, 2, 1, 3, 4]] - d).max() <= 1e-12 * np.abs(d).max()
    # 3-D: extruded channel, state uniform in z with a spanwise momentum added
    g3 = I.extrude_2d(g, 6, dz=0.05)
    q3 = np.repeat(q, 6, axis=1)
    w = 0.1 * q3[0]
    q3[4] += 0.5 * w * w / q3[0]
    q3[3] = w
    g3d = I.mirror_channel_2d((20, 14), Gn=Gn, doubled=True)
    g3d = I.extrude_2d(g3d, 6, dz=0.05)
    c3 = O.cfg_for(g3, M=M, qinf=qinf)
    c3d = O.cfg_for(g3d, M=M, qinf=qinf)
    _, d3 = O.rhs(c3, O.metrics(c3, g3.nodes, Gn), np.ascontiguousarray(q3))
    _, d3d = O.rhs(c3d, O.metrics(c3d, g3d.nodes, Gn), _mirror_doubled_state(q3))
    assert np.abs(d3d[:, :, 14:, :] - d3).max() <= 1e-12 * np.abs(d3).max()


def test_slip_wall_keeps_a_tangent_uniform_stream_and_rejects_a_crossing_one():
    """A uniform stream along a straight wall is an exact solution (zero residual to
    rounding); one that crosses the wall is not."""
    M = 6
    Gn = O.node_ghost(M)
    g = I.mirror_channel_2d((20, 14), Gn=Gn)
    q_along = I.uniform_state(g, I.uniform_qinf(0.7, 0.0))
    q_cross = I.uniform_state(g, I.uniform_qinf(0.7, 30.0))
    c = O.cfg_for(g, M=M)
    met = O.metrics(c, g.nodes, Gn)
    assert np.abs(O.rhs(c, met, q_along)[1]).max() < 1e-12
    assert np.abs(O.rhs(c, met, q_cross)[1]).max() > 1e-2


def _cut_vortex_error(ni, bc_lo=I.BC_CUT):
    M, scheme = 6, 1
    Gn = O.node_ghost(M)
    g = I.parabolic_cgrid_2d((ni, ni // 2), a=3.0, b=3.0, Gn=Gn)
    bc = list(map(list, g.bc))
    bc[1][0] = bc_lo
    g.bc = tuple(map(tuple, bc))
    x, y = g.interior_xyz()
    xc, yc = 4.0, 0.3
    q = I.shu_vortex(x, y, 0.0, xc, yc, eps=5.0, mach=0.5)
    c = O.cfg_for(g, M=M, scheme=scheme, qinf=I.uniform_qinf(0.5, 0.0, rho=1.0, p=1.0))
    L = O.rhs(c, O.metrics(c, g.nodes, Gn), q)[1]
    exact = -0.5 * np.sqrt(GAMMA) * np.imag(_vortex_complex(x + 1e-30j, y, xc=xc, yc=yc)) / 1e-30
    # cells whose stencils reach through the cut, in the vortex core
    rows = np.zeros_like(x, dtype=bool)
    rows[:, :O.ghost(M), :] = True
    sel = (rows & ((x - xc) ** 2 + (y - yc) ** 2 < 1.5 ** 2))[None]
    assert sel.sum() > 0
    return np.abs((L - exact) * sel).max()


def test_cgrid_cut_is_design_order_through_the_cut():
    """A translating vortex sitting on the cut of a parabolic C-grid: the residual of
    the cells whose stencils cross the cut converges to the closed-form time derivative
    at the scheme's order (linear upwind, M6), while a wall or zero-gradient rule there
    leaves an O(1) error."""
    e = [_cut_vortex_error(n) for n in (128, 256)]
    assert 4.3 < np.log2(e[0] / e[1]) < 5.7, e
    assert _cut_vortex_error(256, I.BC_SLIP_WALL) > 100 * e[1]
    assert _cut_vortex_error(256, I.BC_EXTRAP) > 100 * e[1]


def test_cgrid_cut_preserves_a_uniform_stream_at_incidence():
    """The cut connects the block to itself: a uniform stream at 30 degrees is kept to
    rounding (a wall there would deflect it)."""
    M = 6
    Gn = O.node_ghost(M)
    g = I.parabolic_cgrid_2d((32, 16), a=2.0, b=2.0, Gn=Gn)
    qinf = I.uniform_qinf(0.7, 30.0)
    q = I.uniform_state(g, qinf)
    c = O.cfg_for(g, M=M, qinf=qinf)
    met = O.metrics(c, g.nodes, Gn)
    assert np.abs(O.rhs(c, met, q)[1]).max() < 1e-12
    c.cut = 6                                       # middle of the slit becomes a flat-plate wall
    assert np.abs(O.rhs(c, met, q)[1]).max() > 1e-2
    q0inf = I.uniform_qinf(0.7, 0.0)                  # ... which a stream along it does not see
    c0 = O.cfg_for(g, M=M, qinf=q0inf)
    c0.cut = 6
    assert np.abs(O.rhs(c0, met, I.uniform_state(g, q0inf))[1]).max() < 1e-12
