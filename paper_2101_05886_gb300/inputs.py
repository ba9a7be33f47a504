"""Seeded synthetic inputs: curvilinear node grids and initial flow states.

This module is shared by the oracle tests and the CUDA path. It holds no
arithmetic of the numerical method (no metrics, no fluxes, no reconstruction):
only node coordinates produced by analytic mappings, seeded perturbations of
those nodes, and closed-form initial states.

Conventions
-----------
* Solution points are grid nodes (finite-difference convention, Sec. 2.2.1):
  a block of ``n = (ni, nj, nk)`` points carries ``ni*nj*nk`` unknowns.
* Node arrays carry ``Gn`` ghost layers on every side of every swept direction
  and are laid out C-contiguous as ``[3][nk+2Gn][nj+2Gn][ni+2Gn]`` (3-D) or
  ``[2][nj+2Gn][ni+2Gn]`` (2-D), i fastest.  Ghost nodes come from the analytic
  mapping evaluated outside the index range (which is the periodic image with
  its coordinate offset for periodic mappings).
* States are conserved variables ``[5][nk][nj][ni]`` = (rho, rho u, rho v,
  rho w, rho E), float64, interior points only.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 1.4

# Boundary codes (same numbering as the C header).
BC_PERIODIC = 0
BC_FARFIELD = 1
BC_EXTRAP = 2
BC_SLIP_WALL = 3
BC_CUT = 4
BC_BLOCK = 5
BC_HALO = 6


def ghost_width(metric_order: int, scheme: int = 0) -> int:
    """State/metric ghost width G = max(3, M/2): the five-point upwind stencils
    reach three points and the order-M face interpolation M/2 points past a
    face.  The seven-point WENO stencil (scheme 2) reaches four points."""
    return max(4 if scheme == 2 else 3, metric_order // 2)


def node_ghost_width(metric_order: int, scheme: int = 0) -> int:
    """Node ghost width needed to evaluate metrics and Jacobian by the same
    central operators in every state ghost cell: G + 3M/2 (inner derivative,
    outer derivative of the metric products, derivative in the Jacobian)."""
    return ghost_width(metric_order, scheme) + 3 * (metric_order // 2)


@dataclasses.dataclass
class Grid:
    """One structured block: node coordinates with ghosts plus its boundary codes."""
    dims: int
    n: tuple            # (ni, nj, nk); nk == 1 in 2-D
    Gn: int
    nodes: np.ndarray   # [dims][..][..] float64 with Gn ghosts
    bc: tuple           # ((lo,hi) for i, (lo,hi) for j, (lo,hi) for k)
    name: str = ""
    cut: int = 0        # BC_CUT sides: cells t < cut and t >= n_t - cut meet across the cut

    def interior_xyz(self):
        """Coordinates of the solution points, each shaped like one state component."""
        g = self.Gn
        if self.dims == 2:
            return tuple(self.nodes[c, g:-g, g:-g][None] for c in range(2))
        return tuple(self.nodes[c, g:-g, g:-g, g:-g] for c in range(3))


def _index_range(n, Gn):
    return np.arange(-Gn, n + Gn, dtype=np.float64)


# --------------------------------------------------------------------------
# 2-D grids
# --------------------------------------------------------------------------
def cartesian_2d(n, h, Gn, origin=(0.0, 0.0), periodic=True):
    """Uniform Cartesian grid with spacing h (use a power of two for exact metrics)."""
    ni, nj = n
    I = _index_range(ni, Gn)
    J = _index_range(nj, Gn)
    JJ, II = np.meshgrid(J, I, indexing="ij")
    nodes = np.stack([origin[0] + h * II, origin[1] + h * JJ])
    bc = (BC_PERIODIC, BC_PERIODIC) if periodic else (BC_FARFIELD, BC_FARFIELD)
    return Grid(2, (ni, nj, 1), Gn, np.ascontiguousarray(nodes), (bc, bc, (0, 0)), "cartesian_2d")


def wavy_sinsin_2d(n=33, amp=0.1, jitter=0.01, seed=1, Gn=6):
    """Free-stream grid on [0,1]^2: x = xi + amp sin(2 pi xi) sin(2 pi eta), y likewise,
    with a seeded uniform jitter of +-jitter*h on every node that is not on the
    boundary ring.  n points per direction, far-field boundaries."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (n - 1)
    I = _index_range(n, Gn)
    JJ, II = np.meshgrid(I, I, indexing="ij")
    xi, eta = II * h, JJ * h
    s = amp * np.sin(2 * np.pi * xi) * np.sin(2 * np.pi * eta)
    x = xi + s
    y = eta + s
    inner = slice(Gn + 1, Gn + n - 1)
    d = rng.uniform(-jitter * h, jitter * h, size=(2, n - 2, n - 2))
    x[inner, inner] += d[0]
    y[inner, inner] += d[1]
    nodes = np.ascontiguousarray(np.stack([x, y]))
    bc = (BC_FARFIELD, BC_FARFIELD)
    return Grid(2, (n, n, 1), Gn, nodes, (bc, bc, (0, 0)), "wavy_sinsin_2d")


def periodic_wavy_2d(n, L=10.0, amp=0.1, Gn=6):
    """Periodic wavy grid on [0,L)^2: x = L(xi' + amp sin 2pi xi' sin 2pi eta'), y likewise,
    xi' = i/n.  The mapping is periodic with offset L, so ghost nodes are images."""
    I = _index_range(n, Gn) / n
    JJ, II = np.meshgrid(I, I, indexing="ij")
    s = amp * np.sin(2 * np.pi * II) * np.sin(2 * np.pi * JJ)
    nodes = np.ascontiguousarray(np.stack([L * (II + s), L * (JJ + s)]))
    bc = (BC_PERIODIC, BC_PERIODIC)
    return Grid(2, (n, n, 1), Gn, nodes, (bc, bc, (0, 0)), "periodic_wavy_2d")


def paper_wavy_2d(npts=21, L=20.0, A_dx=0.6, nwave=8, Gn=6):
    """Wavy grid of the free-stream and vortex tests (Sec. 4.1.1, wavy-grid equation):
    domain [-L/2, L/2]^2 with npts points per direction, the last point the periodic
    image of the first, so npts-1 unique periodic points."""
    n = npts - 1
    d0 = L / n
    I = _index_range(n, Gn)
    JJ, II = np.meshgrid(I, I, indexing="ij")
    x = -L / 2 + d0 * (II + (A_dx / d0) * np.sin(nwave * np.pi * JJ * d0 / L))
    y = -L / 2 + d0 * (JJ + (A_dx / d0) * np.sin(nwave * np.pi * II * d0 / L))
    nodes = np.ascontiguousarray(np.stack([x, y]))
    bc = (BC_PERIODIC, BC_PERIODIC)
    return Grid(2, (n, n, 1), Gn, nodes, (bc, bc, (0, 0)), "paper_wavy_2d")


def paper_random_2d(npts=21, L=20.0, frac=0.2, seed=7, Gn=6):
    """Random grid of the free-stream test: every unique node of the periodic
    Cartesian grid moved by frac*spacing in a seeded random direction; ghost nodes
    are periodic images (with offset L) of the moved nodes."""
    n = npts - 1
    d0 = L / n
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0.0, 2 * np.pi, size=(n, n))
    dx = frac * d0 * np.cos(ang)
    dy = frac * d0 * np.sin(ang)
    idx = np.arange(-Gn, n + Gn)
    JJ, II = np.meshgrid(idx, idx, indexing="ij")
    wj, wi = JJ % n, II % n
    x = -L / 2 + d0 * II + dx[wj, wi]
    y = -L / 2 + d0 * JJ + dy[wj, wi]
    nodes = np.ascontiguousarray(np.stack([x.astype(np.float64), y.astype(np.float64)]))
    bc = (BC_PERIODIC, BC_PERIODIC)
    return Grid(2, (n, n, 1), Gn, nodes, (bc, bc, (0, 0)), "paper_random_2d")


def random_grid_2d(n, L=1.0, frac=0.2, seed=5, Gn=6):
    """Cartesian grid of n x n points on [0,L]^2 with every node (ghosts included)
    moved by frac*spacing in a seeded random direction (the randomised grids of the
    shock tests of Sec. 4.2); zero-gradient boundaries."""
    rng = np.random.default_rng(seed)
    h = L / (n - 1)
    I = _index_range(n, Gn)
    JJ, II = np.meshgrid(I, I, indexing="ij")
    ang = rng.uniform(0.0, 2 * np.pi, size=II.shape)
    x = h * II + frac * h * np.cos(ang)
    y = h * JJ + frac * h * np.sin(ang)
    nodes = np.ascontiguousarray(np.stack([x, y]))
    bc = (BC_EXTRAP, BC_EXTRAP)
    return Grid(2, (n, n, 1), Gn, nodes, (bc, bc, (0, 0)), "random_grid_2d")


def extrude_2d(g2: Grid, nk: int, dz: float = 1.0):
    """Extrude a 2-D grid into 3-D with z = dz*k (periodic in k): used to check that
    the 3-D operators reduce to the 2-D ones."""
    Gn = g2.Gn
    K = _index_range(nk, Gn)
    shp = (nk + 2 * Gn,) + g2.nodes.shape[1:]
    x = np.broadcast_to(g2.nodes[0][None], shp)
    y = np.broadcast_to(g2.nodes[1][None], shp)
    z = np.broadcast_to((dz * K)[:, None, None], shp)
    nodes = np.ascontiguousarray(np.stack([x, y, z]))
    bc = (g2.bc[0], g2.bc[1], (BC_PERIODIC, BC_PERIODIC))
    return Grid(3, (g2.n[0], g2.n[1], nk), Gn, nodes, bc, g2.name + "_extruded")


# --------------------------------------------------------------------------
# 3-D grids
# --------------------------------------------------------------------------
def _mesh3(ni, nj, nk, Gn):
    K = _index_range(nk, Gn)
    J = _index_range(nj, Gn)
    I = _index_range(ni, Gn)
    return np.meshgrid(K, J, I, indexing="ij")  # KK, JJ, II each [nk+2G][nj+2G][ni+2G]


def cartesian_3d(n, h, Gn, periodic=True):
    ni, nj, nk = n
    KK, JJ, II = _mesh3(ni, nj, nk, Gn)
    nodes = np.ascontiguousarray(np.stack([h * II, h * JJ, h * KK]))
    b = (BC_PERIODIC, BC_PERIODIC) if periodic else (BC_FARFIELD, BC_FARFIELD)
    return Grid(3, (ni, nj, nk), Gn, nodes, (b, b, b), "cartesian_3d")


def periodic_wavy_3d(n, L=10.0, amp=0.08, Gn=6, dtype=np.float64, k_range=None):
    """Periodic 3-D wavy grid on [0,L)^3: each coordinate x_a = L(xi'_a + amp
    sin 2pi xi' sin 2pi eta' sin 2pi zeta'), xi'_a = index/n_a.
    k_range=(k0, k1): only the points k0 <= k < k1 of that grid (any integers: the mapping
    is evaluated there, with Gn ghost layers around the range), as a block of
    (ni, nj, k1 - k0) points whose nodes equal the full grid's bit for bit."""
    ni, nj, nk = n
    if k_range is None:
        KK, JJ, II = _mesh3(ni, nj, nk, Gn)
        nb = nk
    else:
        k0, k1 = k_range
        nb = k1 - k0
        KK, JJ, II = np.meshgrid(np.arange(k0 - Gn, k1 + Gn, dtype=np.float64), _index_range(nj, Gn),
                                 _index_range(ni, Gn), indexing="ij")
    xi, eta, zeta = II / ni, JJ / nj, KK / nk
    s = amp * np.sin(2 * np.pi * xi) * np.sin(2 * np.pi * eta) * np.sin(2 * np.pi * zeta)
    nodes = np.empty((3,) + KK.shape, dtype=dtype)
    nodes[0] = L * (xi + s)
    nodes[1] = L * (eta + s)
    nodes[2] = L * (zeta + s)
    b = (BC_PERIODIC, BC_PERIODIC)
    return Grid(3, (ni, nj, nb), Gn, nodes, (b, b, b), "periodic_wavy_3d")


def cylinder_ogrid(n, r0=0.5, r1=20.0, beta=3.0, Lz=4.0, Gn=6, wall=False):
    """Cylinder O-grid: i runs around the cylinder (periodic), j is radial with a
    tanh stretch r = r0 + (r1-r0)[1 - tanh(beta(1-eta'))/tanh(beta)], k is spanwise
    (periodic with offset Lz); the outer side (j=nj-1) is far field.
    wall=False: eta' = j/(nj-1), the first points lie on r = r0, zero-gradient there.
    wall=True: eta' = (j+1/2)/(nj-1/2), so r = r0 is the face j = -1/2, a slip wall."""
    ni, nj, nk = n
    KK, JJ, II = _mesh3(ni, nj, nk, Gn)
    th = 2 * np.pi * II / ni
    ep = (JJ + 0.5) / (nj - 0.5) if wall else JJ / (nj - 1)
    r = r0 + (r1 - r0) * (1.0 - np.tanh(beta * (1.0 - ep)) / np.tanh(beta))
    nodes = np.ascontiguousarray(np.stack([r * np.cos(th), r * np.sin(th), Lz * KK / nk]))
    bc = ((BC_PERIODIC, BC_PERIODIC), (BC_SLIP_WALL if wall else BC_EXTRAP, BC_FARFIELD),
          (BC_PERIODIC, BC_PERIODIC))
    return Grid(3, (ni, nj, nk), Gn, nodes, bc, "cylinder_ogrid_wall" if wall else "cylinder_ogrid")


def mirror_channel_2d(n, amp=0.06, Gn=6, doubled=False):
    """Wavy channel for the slip-wall checks: xi' = i/ni periodic in i (x offset 1),
    eta'_j = (j + 1/2)/nj, x = xi' + amp sin(2 pi xi') cos(2 pi eta'),
    y = eta' + amp sin(2 pi xi') sin(2 pi eta').  The map is mirror symmetric about
    eta' = 0 and eta' = 1 (x even, y odd), the faces j = -1/2 and j = nj - 1/2, so the
    ghost nodes are the mirror images of the interior nodes.
    doubled=False: walls on both j sides.  doubled=True: the mirror-doubled channel
    eta' in [-1, 1) (2 nj points, j - nj in place of j), periodic in j with y offset 2."""
    ni, nj = n
    nj2 = 2 * nj if doubled else nj
    I = _index_range(ni, Gn)
    J = _index_range(nj2, Gn)
    JJ, II = np.meshgrid(J, I, indexing="ij")
    xi = II / ni
    eta = ((JJ - nj) if doubled else JJ) / nj + 0.5 / nj
    sx = amp * np.sin(2 * np.pi * xi)
    nodes = np.ascontiguousarray(np.stack([xi + sx * np.cos(2 * np.pi * eta), eta + sx * np.sin(2 * np.pi * eta)]))
    bj = (BC_PERIODIC, BC_PERIODIC) if doubled else (BC_SLIP_WALL, BC_SLIP_WALL)
    return Grid(2, (ni, nj2, 1), Gn, nodes, ((BC_PERIODIC, BC_PERIODIC), bj, (BC_PERIODIC, BC_PERIODIC)),
                "mirror_channel_2d")


def parabolic_cgrid_2d(n, a=1.0, b=1.0, Gn=6):
    """C-grid of the parabolic map x + i y = (xi' + i eta')^2 with xi'_i = a(2(i+1/2)/ni - 1)
    (i runs from the lower side of the slit y = 0, x > 0 around the origin to its upper
    side) and eta'_j = b (j + 1/2)/nj.  The face j = -1/2 is the slit, which the grid meets
    from both sides: (xi', -eta') and (-xi', eta') are the same point, so the analytic ghost
    nodes j < 0 are the nodes across the cut (index ni-1-i, -1-j), as the C-grid cut rule
    expects.  The whole j-lo side is a cut (cut = ni/2, ni even); other sides far field."""
    ni, nj = n
    assert ni % 2 == 0
    I = _index_range(ni, Gn)
    J = _index_range(nj, Gn)
    JJ, II = np.meshgrid(J, I, indexing="ij")
    xs = a * (2.0 * (II + 0.5) / ni - 1.0)
    es = b * (JJ + 0.5) / nj
    nodes = np.ascontiguousarray(np.stack([xs * xs - es * es, 2.0 * xs * es]))
    bc = ((BC_FARFIELD, BC_FARFIELD), (BC_CUT, BC_FARFIELD), (BC_PERIODIC, BC_PERIODIC))
    return Grid(2, (ni, nj, 1), Gn, nodes, bc, "parabolic_cgrid_2d", cut=ni // 2)


def _stretch_beta(first, npts):
    """beta such that 1 - tanh(beta(1 - 1/(npts-1)))/tanh(beta) == first (bisection)."""
    lo, hi = 1e-3, 30.0
    for _ in range(200):
        b = 0.5 * (lo + hi)
        s1 = 1.0 - math.tanh(b * (1.0 - 1.0 / (npts - 1))) / math.tanh(b)
        if s1 > first:
            lo = b
        else:
            hi = b
    return 0.5 * (lo + hi)


def _growth_ratio(first, total, steps):
    """r such that first * (r**steps - 1)/(r - 1) == total (bisection, r > 1)."""
    lo, hi = 1.0 + 1e-9, 2.0
    while first * (hi ** steps - 1.0) / (hi - 1.0) < total:
        hi *= 1.5
    for _ in range(200):
        r = 0.5 * (lo + hi)
        if first * (r ** steps - 1.0) / (r - 1.0) < total:
            lo = r
        else:
            hi = r
    return 0.5 * (lo + hi)


def cgrid_wing(n=(512, 384, 512), tc=0.15, taper=0.5, sweep_deg=30.0, span=3.0,
               far=20.0, first_cell=1e-4, wake_frac=0.25, Gn=6, dtype=np.float64, physical=True):
    """Single-block C-grid around a swept, tapered, extruded thick wing-like body.

    i wraps from the lower wake outflow, around the body (trailing edge -> leading
    edge -> trailing edge) to the upper wake outflow; j runs from the body/wake
    line to a far field `far` chords away with tanh stretching (first node offset
    `first_cell` chords); k runs along the span.  At span station z the chord is
    c(z) = 1 - (1-taper) z/span and the leading edge is swept back by z*tan(sweep).
    The section, with body parameter t in [-1, 1] (1 lower trailing edge, 0 leading
    edge), is x = c t^2, y = -K c t (1 - t^2): round-nosed (y ~ sqrt(x) at the
    leading edge, like an ellipse), thickness tc*c, and a finite trailing-edge wedge
    so the wake lines leave it without a kink.  Wake points are spaced geometrically
    from the body's trailing-edge spacing out to `far` chords.  Grid lines leave the
    inner curve along a direction that turns continuously from -y (lower wake)
    through -x (leading edge) to +y (upper wake).  Ghost nodes are the same formulas
    evaluated outside the index ranges.
    physical=True: the body surface and the wake line are the face j = -1/2 (the wall
    normal parameter is taken at j + 1/2); the j-lo side is a C-grid cut over the wake
    cells (i < cut, i >= ni - cut, whose ghost nodes are set to their partners across
    the cut) and a slip wall over the body, and the root plane k-lo is zero-gradient.
    physical=False: the first nodes lie on the body and wake line, every j-lo ghost is
    zero-gradient.
    """
    ni, nj, nk = n
    beta = _stretch_beta(first_cell / far, nj)
    i = _index_range(ni, Gn)
    j = _index_range(nj, Gn)
    k = _index_range(nk, Gn)
    s = i / (ni - 1)                                   # wrap parameter
    z = span * k / (nk - 1)                            # span coordinate
    ej = (j + 0.5) / (nj - 0.5) if physical else j / (nj - 1)
    sj = 1.0 - np.tanh(beta * (1.0 - ej)) / np.tanh(beta)  # 0 wall, 1 far
    chord = 1.0 - (1.0 - taper) * z / span
    xle = z * math.tan(math.radians(sweep_deg))
    wf = wake_frac
    sb = np.clip((s - wf) / (1.0 - 2 * wf), 0.0, 1.0)  # body fraction
    t = 1.0 - 2.0 * sb
    kth = tc / (2.0 * (2.0 / 3.0) * math.sqrt(1.0 / 3.0))   # max of t(1-t^2) is (2/3)sqrt(1/3)
    sig = np.maximum((wf - s) / wf, 0.0) + np.maximum((s - (1.0 - wf)) / wf, 0.0)  # wake fraction
    steps = wf * (ni - 1)                              # wake intervals on each side
    first = 4.0 / ((1.0 - 2 * wf) * (ni - 1))          # body trailing-edge step in chords
    psi = -0.5 * np.pi - np.pi * sb                    # outward direction angle
    dx, dy = np.cos(psi), np.sin(psi)
    nodes = np.empty((3, k.size, j.size, i.size), dtype=dtype)
    for kk in range(k.size):
        c = chord[kk]
        r = _growth_ratio(first, far / c, steps)
        wl = c * first * (r ** (sig * steps) - 1.0) / (r - 1.0)
        xin = xle[kk] + c * t * t + wl
        yin = -kth * c * t * (1.0 - t * t)
        nodes[0, kk] = xin[None, :] + far * sj[:, None] * dx[None, :]
        nodes[1, kk] = yin[None, :] + far * sj[:, None] * dy[None, :]
        nodes[2, kk] = z[kk]
    if not physical:
        bc = ((BC_EXTRAP, BC_EXTRAP), (BC_EXTRAP, BC_FARFIELD), (BC_EXTRAP, BC_EXTRAP))
        return Grid(3, (ni, nj, nk), Gn, nodes, bc, "cgrid_wing")
    cut = int(np.count_nonzero(np.arange(ni) / (ni - 1) < wf))
    # wake ghost nodes (j < 0, i < cut or i >= ni - cut, ghost i included) are the nodes
    # across the cut: (i, -1-m) -> (ni-1-i, m)
    iw = np.concatenate([np.arange(-Gn, cut), np.arange(ni - cut, ni + Gn)])
    for m in range(Gn):
        nodes[:, :, Gn - 1 - m, iw + Gn] = nodes[:, :, Gn + m, ni - 1 - iw + Gn]
    bc = ((BC_EXTRAP, BC_EXTRAP), (BC_CUT, BC_FARFIELD), (BC_EXTRAP, BC_EXTRAP))
    return Grid(3, (ni, nj, nk), Gn, nodes, bc, "cgrid_wing", cut=cut)


def batched_block_sizes(nblocks=64, lo=32, hi=128, seed=4):
    """Seeded uneven block sizes: each of ni, nj, nk drawn from U{lo..hi}."""
    rng = np.random.default_rng(seed)
    return [tuple(int(v) for v in rng.integers(lo, hi + 1, size=3)) for _ in range(nblocks)]


def batched_blocks(nblocks=64, lo=32, hi=128, seed=4, Gn=12):
    """Multi-block set: first half cylinder O-grids (random spanwise extent
    U(1,8)), second half periodic 3-D wavy grids (amplitude 0.08)."""
    rng = np.random.default_rng(seed + 1000)
    sizes = batched_block_sizes(nblocks, lo, hi, seed)
    grids = []
    for b, n in enumerate(sizes):
        if b < nblocks // 2:
            grids.append(cylinder_ogrid(n, Lz=float(rng.uniform(1.0, 8.0)), Gn=Gn))
        else:
            grids.append(periodic_wavy_3d(n, L=10.0, amp=0.08, Gn=Gn))
    return grids


# --------------------------------------------------------------------------
# Initial states
# --------------------------------------------------------------------------
def primitive_to_conserved(rho, u, v, w, p, gamma=GAMMA):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, E]).astype(np.float64))


def uniform_qinf(mach, alpha_deg=0.0, beta_deg=0.0, rho=GAMMA, p=1.0, gamma=GAMMA):
    """Uniform state of Mach `mach`, flow angle alpha in the x-y plane (and beta
    towards z); with rho = gamma and p = 1 the sound speed is 1."""
    c = math.sqrt(gamma * p / rho)
    a, b = math.radians(alpha_deg), math.radians(beta_deg)
    u = mach * c * math.cos(a) * math.cos(b)
    v = mach * c * math.sin(a) * math.cos(b)
    w = mach * c * math.sin(b)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.array([rho, rho * u, rho * v, rho * w, E], dtype=np.float64)


def uniform_state(grid: Grid, qinf):
    ni, nj, nk = grid.n
    q = np.empty((5, nk, nj, ni), dtype=np.float64)
    q[:] = np.asarray(qinf, dtype=np.float64)[:, None, None, None]
    return q


def shu_vortex(x, y, t=0.0, xc=5.0, yc=5.0, eps=5.0, mach=0.5, L=None, gamma=GAMMA):
    """Isentropic vortex of strength eps on a rho=p=1 background moving with Mach
    `mach` along x; closed form at time t is the initial field translated by u t
    (wrapped into a periodic box of size L when L is given)."""
    uinf = mach * math.sqrt(gamma)
    cx = xc + uinf * t
    dx = x - cx
    dy = y - yc
    if L is not None:
        dx = (dx + 0.5 * L) % L - 0.5 * L
        dy = (dy + 0.5 * L) % L - 0.5 * L
    r2 = dx * dx + dy * dy
    f = eps / (2 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = uinf - f * dy
    v = f * dx
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return primitive_to_conserved(rho, u, v, np.zeros_like(u), p, gamma)


def paper_vortex(x, y, t=0.0, eps=0.02, alpha=0.204, rc=1.0, mach=0.5, L=20.0, gamma=GAMMA):
    """Vortex of Sec. 4.1.2 on the rho=gamma, p=1 background at Mach `mach` along x,
    centred at the origin at t=0 of a periodic box [-L/2, L/2)^2."""
    uinf = mach  # sound speed is 1 for rho=gamma, p=1
    dx = x - uinf * t
    dy = np.asarray(y, dtype=np.float64) + 0.0
    dx = (dx + 0.5 * L) % L - 0.5 * L
    dy = (dy + 0.5 * L) % L - 0.5 * L
    r = np.sqrt(dx * dx + dy * dy)
    tau = r / rc
    e = np.exp(alpha * (1.0 - tau * tau))
    # eps*tau*e^{..}*(sin th, -cos th) with (sin th, -cos th) = (dy/r, -dx/r)
    u = uinf + eps * e * dy / rc
    v = -eps * e * dx / rc
    Tinf = 1.0 / gamma
    T = Tinf - (gamma - 1.0) * eps * eps / (4.0 * alpha * gamma) * e * e
    rho = gamma * (T / Tinf) ** (1.0 / (gamma - 1.0))
    p = rho * T
    return primitive_to_conserved(rho, u, v, np.zeros_like(u), p, gamma)


def vortex_3d(grid: Grid, mach=0.8, eps=5.0, L=10.0, gamma=GAMMA):
    """Mach `mach` stream along x plus a z-extruded isentropic vortex of strength eps
    centred in the x-y plane of the box."""
    x, y, _ = grid.interior_xyz()
    return shu_vortex(x, y, 0.0, 0.5 * L, 0.5 * L, eps=eps, mach=mach, L=L, gamma=gamma)


def normal_shock_state(grid: Grid, x0, mach=2.0, gamma=GAMMA):
    """Planar shock at x = x0 moving into still gas (rho = gamma, p = 1, c = 1) with
    shock Mach number `mach`; the Rankine-Hugoniot post-shock state is behind it
    (x < x0)."""
    x = grid.interior_xyz()[0]
    r1, p1 = gamma, 1.0
    m2 = mach * mach
    r2 = r1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    u2 = mach * 1.0 * (1.0 - r1 / r2)
    behind = x < x0
    rho = np.where(behind, r2, r1)
    u = np.where(behind, u2, 0.0)
    p = np.where(behind, p2, p1)
    z = np.zeros_like(rho)
    return primitive_to_conserved(rho, u, z, z, p, gamma)


def perturbed_state(grid: Grid, qinf, amp=1e-3, seed=0):
    """Uniform state times (1 + amp * smooth seeded field): three random Fourier
    modes in the index space, so the perturbation is smooth and periodic."""
    rng = np.random.default_rng(seed)
    ni, nj, nk = grid.n
    K, J, I = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    q = uniform_state(grid, qinf)
    for c in range(5):
        f = np.zeros(I.shape)
        for _ in range(3):
            kx, ky, kz = rng.integers(1, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            f += np.sin(2 * np.pi * kx * I / ni + ph[0]) * np.sin(2 * np.pi * ky * J / nj + ph[1]) \
                * np.cos(2 * np.pi * kz * K / max(nk, 1) + ph[2])
        if c in (1, 2, 3):
            q[c] += amp * f * max(abs(qinf[0]), 1.0)
        else:
            q[c] *= 1.0 + amp * f / 3.0
    return q


def random_smooth_state(grid: Grid, qinf, amp=0.05, seed=0):
    """A non-trivial smooth state for parity checks (larger perturbation)."""
    return perturbed_state(grid, qinf, amp=amp, seed=seed)


def fade_to_farfield(grid: Grid, q, qinf, width=8):
    """q blended into the uniform far-field state over the `width` points next to every
    far-field side (weight cos^2 from 1, `width` points inside, to 0 at the last two
    points), so that the state meets its far-field ghosts without a jump."""
    q = np.array(q, dtype=np.float64, copy=True)
    qu = uniform_state(grid, qinf)
    w = np.ones(q.shape[1:])
    for d in range(grid.dims):
        n = grid.n[d]
        ax = 2 - d                                   # axis of direction d in [k][j][i]
        x = np.arange(n, dtype=np.float64)
        for side in (0, 1):
            if grid.bc[d][side] != BC_FARFIELD:
                continue
            dist = x if side == 0 else (n - 1 - x)
            t = np.clip((width - 1 - dist) / (width - 2.0), 0.0, 1.0)
            wd = np.cos(0.5 * np.pi * t) ** 2
            shape = [1, 1, 1]
            shape[ax] = n
            w = w * wd.reshape(shape)
    return qu + (q - qu) * w[None]


# --------------------------------------------------------------------------
# Multi-block splits
# --------------------------------------------------------------------------
def split_grid(grid: Grid, direction: int, sizes, side_bc: int = BC_BLOCK):
    """Split a block into consecutive blocks of the given extents along `direction`.

    Returns (blocks, links): each block's ghost nodes are the neighbouring blocks' nodes
    (sliced from the parent, whose own ghosts serve the outer sides); the inner sides get
    `side_bc` (BC_BLOCK for blocks of one batch, BC_HALO for slabs held by different
    processes) and a link (a, direction, side, b); a periodic parent's outer sides are
    linked around (last block's high side to the first block's low side).  States are
    split with `split_state`."""
    assert sum(sizes) == grid.n[direction] and min(sizes) >= 1
    Gn = grid.Gn
    ax = grid.nodes.ndim - 1 - direction          # array axis of `direction` in the node array
    nb = len(sizes)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)
    periodic = grid.bc[direction] == (BC_PERIODIC, BC_PERIODIC)
    blocks, links = [], []
    for b, (a0, nloc) in enumerate(zip(starts, sizes)):
        sl = [slice(None)] * grid.nodes.ndim
        sl[ax] = slice(a0, a0 + nloc + 2 * Gn)
        nodes = np.ascontiguousarray(grid.nodes[tuple(sl)])
        n = list(grid.n)
        n[direction] = int(nloc)
        bc = [list(p) for p in grid.bc]
        if b > 0 or periodic:
            bc[direction][0] = side_bc
            links.append((b, direction, 0, (b - 1) % nb))
        if b < nb - 1 or periodic:
            bc[direction][1] = side_bc
            links.append((b, direction, 1, (b + 1) % nb))
        blocks.append(Grid(grid.dims, tuple(n), Gn, nodes, tuple(map(tuple, bc)),
                           f"{grid.name}_part{b}", grid.cut))
    return blocks, links


def split_state(q: np.ndarray, direction: int, sizes):
    """Split a state [5][nk][nj][ni] into the parts of `split_grid`."""
    ax = q.ndim - 1 - direction
    cuts = np.cumsum(sizes)[:-1]
    return [np.ascontiguousarray(p) for p in np.split(q, cuts, axis=ax)]
