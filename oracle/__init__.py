"""ctypes front end of the serial FP64 oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The product path never imports it.

The oracle follows the paper (arXiv 2101.05886) equation by equation: the
symmetric conservative metrics and Jacobian (Eqs. JBabc, JB, metric_discret),
WENO5-JS / linear upwind (Eqs. weno, weno_wights, linear_upwind,
new_form_linear_upwind), characteristic Lax-Friedrichs splitting (Sec. 2.2.2),
the free-stream-preserving face flux (Eqs. Q_star, QdJ_star, 1dJ, xidJ,
my_point1/2/3, Linear_upwind_LFspliting), the flux difference (Eq. aderivative)
and third-order TVD Runge-Kutta.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                               "-o", _LIB_PATH, src, "-lm"])
    return _LIB_PATH


class Cfg(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", ctypes.c_int * 3), ("M", ctypes.c_int),
                ("scheme", ctypes.c_int), ("fp", ctypes.c_int), ("charwise", ctypes.c_int),
                ("form", ctypes.c_int), ("global_lf", ctypes.c_int), ("bc", (ctypes.c_int * 2) * 3),
                ("gamma", ctypes.c_double),
                ("qinf", ctypes.c_double * 5), ("cut", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.or_ghost.restype = ctypes.c_int
        L.or_node_ghost.restype = ctypes.c_int
        L.or_ghost_s.restype = ctypes.c_int
        L.or_node_ghost_s.restype = ctypes.c_int
        L.or_weno7.argtypes = [_D]
        L.or_weno7.restype = ctypes.c_double
        L.or_weno7_parts.argtypes = [_D, _D, _D]
        L.or_wenocu6.argtypes = [_D]
        L.or_wenocu6.restype = ctypes.c_double
        L.or_wenocu6_parts.argtypes = [_D, _D, _D, _D]
        L.or_interp_coef.argtypes = [ctypes.c_int, _D]
        L.or_weno5.argtypes = [_D]
        L.or_weno5_parts.argtypes = [_D, _D, _D]
        L.or_weno5.restype = ctypes.c_double
        L.or_lu5.argtypes = [_D]
        L.or_lu5.restype = ctypes.c_double
        L.or_eigensystem.argtypes = [_D, _D, _D, ctypes.c_double, _D, _D]
        L.or_metrics.argtypes = [ctypes.POINTER(Cfg), _D, ctypes.c_int, _D]
        L.or_metrics.restype = ctypes.c_int
        L.or_face_flux.argtypes = [ctypes.POINTER(Cfg), _D, _D, _D]
        L.or_face_flux_lam.argtypes = [ctypes.POINTER(Cfg), _D, _D, _D, _D]
        L.or_rhs.argtypes = [ctypes.POINTER(Cfg), _D, _D, _D, _D]
        L.or_rhs.restype = ctypes.c_int
        L.or_rk3_step.argtypes = [ctypes.POINTER(Cfg), _D, _D, ctypes.c_double]
        L.or_rk3_step.restype = ctypes.c_int
        L.or_cfl_dt.argtypes = [ctypes.POINTER(Cfg), _D, _D, ctypes.c_double]
        L.or_cfl_dt.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def make_cfg(dims, n, M=6, scheme=0, fp=1, charwise=1, form=2, bc=((0, 0), (0, 0), (0, 0)),
             gamma=1.4, qinf=(1.4, 0.0, 0.0, 0.0, 2.5), global_lf=0, cut=0) -> Cfg:
    c = Cfg()
    c.dims = dims
    for d in range(3):
        c.n[d] = int(n[d])
        c.bc[d][0] = int(bc[d][0])
        c.bc[d][1] = int(bc[d][1])
    c.M, c.scheme, c.fp, c.charwise, c.form = M, scheme, fp, charwise, form
    c.global_lf = global_lf
    c.cut = int(cut)
    c.gamma = gamma
    for v in range(5):
        c.qinf[v] = float(qinf[v])
    return c


def cfg_for(grid, M=6, scheme=0, fp=1, charwise=1, form=2, gamma=1.4, qinf=None, global_lf=0) -> Cfg:
    if qinf is None:
        qinf = (1.4, 0.0, 0.0, 0.0, 2.5)
    return make_cfg(grid.dims, grid.n, M, scheme, fp, charwise, form, grid.bc, gamma, qinf, global_lf,
                    getattr(grid, "cut", 0))


def ghost(M: int, scheme: int = 0) -> int:
    return lib().or_ghost_s(M, scheme)


def node_ghost(M: int, scheme: int = 0) -> int:
    return lib().or_node_ghost_s(M, scheme)


def met_shape(cfg: Cfg):
    G = ghost(cfg.M, cfg.scheme)
    ni, nj, nk = cfg.n[0], cfg.n[1], cfg.n[2]
    if cfg.dims == 2:
        return (10, 1, nj + 2 * G, ni + 2 * G)
    return (10, nk + 2 * G, nj + 2 * G, ni + 2 * G)


def metrics(cfg: Cfg, nodes: np.ndarray, Gn: int) -> np.ndarray:
    met = np.zeros(met_shape(cfg), dtype=np.float64)
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    rc = lib().or_metrics(ctypes.byref(cfg), _p(nodes), int(Gn), _p(met))
    if rc:
        raise ValueError("or_metrics rejected its arguments")
    return met


def rhs(cfg: Cfg, met: np.ndarray, q: np.ndarray):
    """Returns (R, dq/dt): R = sum_d (F'_{i+1/2} - F'_{i-1/2}) and dq/dt = -J R."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros_like(q)
    L = np.zeros_like(q)
    rc = lib().or_rhs(ctypes.byref(cfg), _p(met), _p(q), _p(R), _p(L))
    if rc:
        raise ValueError("or_rhs rejected its arguments")
    return R, L


def rk3_step(cfg: Cfg, met: np.ndarray, q: np.ndarray, dt: float) -> np.ndarray:
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    rc = lib().or_rk3_step(ctypes.byref(cfg), _p(met), _p(q), float(dt))
    if rc:
        raise ValueError("or_rk3_step rejected its arguments")
    return q


def cfl_dt(cfg: Cfg, met: np.ndarray, q: np.ndarray, cfl: float) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().or_cfl_dt(ctypes.byref(cfg), _p(met), _p(q), float(cfl))


def weno5(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().or_weno5(_p(v))


def weno7(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().or_weno7(_p(v))


def weno5_parts(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    q = np.zeros(3)
    b = np.zeros(3)
    lib().or_weno5_parts(_p(v), _p(q), _p(b))
    return q, b


def weno7_parts(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    q = np.zeros(4)
    b = np.zeros(4)
    lib().or_weno7_parts(_p(v), _p(q), _p(b))
    return q, b


def wenocu6(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().or_wenocu6(_p(v))


def wenocu6_parts(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    q = np.zeros(4)
    b = np.zeros(4)
    t = np.zeros(1)
    lib().or_wenocu6_parts(_p(v), _p(q), _p(b), _p(t))
    return q, b, float(t[0])


def lu5(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().or_lu5(_p(v))


def interp_coef(M: int) -> np.ndarray:
    c = np.zeros(8)
    lib().or_interp_coef(M, _p(c))
    return c[:M]


def eigensystem(qL, qR, k, gamma=1.4):
    L = np.zeros(25)
    R = np.zeros(25)
    lib().or_eigensystem(_p(np.ascontiguousarray(qL, dtype=np.float64)),
                         _p(np.ascontiguousarray(qR, dtype=np.float64)),
                         _p(np.ascontiguousarray(k, dtype=np.float64)), gamma, _p(L), _p(R))
    return L.reshape(5, 5), R.reshape(5, 5)


def face_flux(cfg: Cfg, q8: np.ndarray, met8: np.ndarray) -> np.ndarray:
    out = np.zeros(5)
    lib().or_face_flux(ctypes.byref(cfg), _p(np.ascontiguousarray(q8, dtype=np.float64)),
                       _p(np.ascontiguousarray(met8, dtype=np.float64)), _p(out))
    return out


def face_flux_lam(cfg: Cfg, q8: np.ndarray, met8: np.ndarray, lam) -> np.ndarray:
    """Face flux with given (global) Lax-Friedrichs speeds per characteristic field."""
    out = np.zeros(5)
    lib().or_face_flux_lam(ctypes.byref(cfg), _p(np.ascontiguousarray(q8, dtype=np.float64)),
                           _p(np.ascontiguousarray(met8, dtype=np.float64)),
                           _p(np.ascontiguousarray(lam, dtype=np.float64)), _p(out))
    return out
