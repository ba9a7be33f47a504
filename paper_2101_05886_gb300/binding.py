"""Thin ctypes binding of libfpgb300.so (include/fp.h): argument marshalling only.

Every entry point keeps its C name.  Device buffers are passed as raw pointers
(``tensor.data_ptr()``) and streams as ``torch.cuda.Stream.cuda_stream`` values;
torch is used by the callers only for device memory and streams.  There is no
fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# FPGB300_LIBRARY selects another build of the library, e.g. the bounds-checking build
# libfpgb300_check.so (build.build(check=True)); it must be set before the first call.
LIB_PATH = os.environ.get("FPGB300_LIBRARY") or os.path.join(HERE, "libfpgb300.so")

(FP_OK, FP_ERR_ARG, FP_ERR_CUDA, FP_ERR_OOM, FP_ERR_NONFINITE, FP_ERR_TIMEOUT, FP_ERR_UNSUPPORTED,
 FP_ERR_BOUNDS) = range(8)
FP_WENO5_JS, FP_LINEAR_UPWIND5, FP_WENO7_JS, FP_WENOCU6 = 0, 1, 2, 3
FP_F64, FP_F32_MIXED = 0, 1
FP_BC_PERIODIC, FP_BC_FARFIELD, FP_BC_EXTRAP, FP_BC_SLIP_WALL, FP_BC_CUT, FP_BC_BLOCK, FP_BC_HALO = 0, 1, 2, 3, 4, 5, 6

# every symbol include/fp.h declares
EXPORTS = [
    "fp_ghost_width", "fp_node_ghost_width", "fp_init_grid", "fp_rhs", "fp_rhs_noalloc", "fp_rk3_step", "fp_cfl_dt",
    "fp_get_metrics", "fp_get_face_metrics", "fp_get_device_status", "fp_launches_per_rhs",
    "fp_launches_per_step", "fp_get_cta_sizes", "fp_get_tile", "fp_set_tile", "fp_last_error", "fp_status_string",
    "fp_free", "fp_batch_create", "fp_batch_create_linked", "fp_batch_rk3_step", "fp_batch_rhs", "fp_batch_launches_per_step", "fp_batch_get_tile",
    "fp_batch_last_error", "fp_batch_free", "fp_state_bytes", "fp_pipe_create", "fp_pipe_rk3_step_host",
    "fp_pipe_set_ordered", "fp_pipe_groups", "fp_pipe_launches_per_step", "fp_pipe_last_error", "fp_pipe_free",
    "fp_balanced_groups", "fp_debug_fail_allocation", "fp_probe_peaks", "fp_rk3_stage", "fp_set_halo",
    "fp_halo_bytes", "fp_pack_halo", "fp_bounds_checking",
]


class fp_block_link(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int), ("dir", ctypes.c_int), ("side", ctypes.c_int), ("b", ctypes.c_int)]


class fp_grid_desc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", ctypes.c_int * 3), ("metric_order", ctypes.c_int),
                ("scheme", ctypes.c_int), ("free_stream_preserving", ctypes.c_int),
                ("characteristic", ctypes.c_int), ("precision", ctypes.c_int),
                ("bc", (ctypes.c_int * 2) * 3), ("gamma", ctypes.c_double),
                ("q_inf", ctypes.c_double * 5), ("global_lf", ctypes.c_int), ("cut_width", ctypes.c_int)]


_lib = None
_VP = ctypes.c_void_p


def lib():
    """Load libfpgb300.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        L.fp_ghost_width.argtypes = [ctypes.c_int, ctypes.c_int]
        L.fp_node_ghost_width.argtypes = [ctypes.c_int, ctypes.c_int]
        L.fp_init_grid.argtypes = [ctypes.POINTER(fp_grid_desc), _VP, ctypes.c_int, _VP, ctypes.POINTER(_VP)]
        L.fp_rhs.argtypes = [_VP, _VP, _VP, _VP]
        L.fp_rhs_noalloc.argtypes = [_VP, _VP, _VP, _VP]
        L.fp_rk3_step.argtypes = [_VP, _VP, ctypes.c_double, _VP]
        L.fp_cfl_dt.argtypes = [_VP, _VP, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _VP]
        L.fp_get_metrics.argtypes = [_VP, _VP]
        L.fp_get_face_metrics.argtypes = [_VP, ctypes.c_int, _VP]
        L.fp_get_device_status.argtypes = [_VP, _VP]
        L.fp_launches_per_rhs.argtypes = [_VP]
        L.fp_launches_per_step.argtypes = [_VP]
        L.fp_get_cta_sizes.argtypes = [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.fp_get_tile.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.fp_set_tile.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.fp_last_error.argtypes = [_VP]
        L.fp_last_error.restype = ctypes.c_char_p
        L.fp_status_string.argtypes = [ctypes.c_int]
        L.fp_status_string.restype = ctypes.c_char_p
        L.fp_free.argtypes = [_VP]
        L.fp_free.restype = None
        L.fp_batch_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP), ctypes.c_int,
                                      _VP, ctypes.POINTER(_VP)]
        L.fp_batch_create_linked.argtypes = [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP),
                                             ctypes.POINTER(fp_block_link), ctypes.c_int, ctypes.c_int,
                                             _VP, ctypes.POINTER(_VP)]
        L.fp_batch_rk3_step.argtypes = [_VP, ctypes.c_double, _VP]
        L.fp_batch_rhs.argtypes = [_VP, ctypes.POINTER(_VP), _VP]
        L.fp_batch_launches_per_step.argtypes = [_VP]
        L.fp_batch_get_tile.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]
        L.fp_batch_last_error.argtypes = [_VP]
        L.fp_batch_last_error.restype = ctypes.c_char_p
        L.fp_batch_free.argtypes = [_VP]
        L.fp_batch_free.restype = None
        L.fp_state_bytes.argtypes = [_VP]
        L.fp_state_bytes.restype = ctypes.c_size_t
        L.fp_pipe_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP), ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(_VP)]
        L.fp_pipe_rk3_step_host.argtypes = [_VP, ctypes.POINTER(_VP), ctypes.c_double, _VP]
        L.fp_pipe_set_ordered.argtypes = [_VP, ctypes.c_int]
        L.fp_pipe_groups.argtypes = [_VP]
        L.fp_pipe_launches_per_step.argtypes = [_VP]
        L.fp_pipe_last_error.argtypes = [_VP]
        L.fp_pipe_last_error.restype = ctypes.c_char_p
        L.fp_pipe_free.argtypes = [_VP]
        L.fp_pipe_free.restype = None
        L.fp_balanced_groups.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]
        L.fp_debug_fail_allocation.argtypes = [ctypes.c_int]
        L.fp_bounds_checking.argtypes = []
        L.fp_probe_peaks.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3 + [_VP]
        L.fp_rk3_stage.argtypes = [_VP, _VP, ctypes.c_double, ctypes.c_int, _VP]
        L.fp_set_halo.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP]
        L.fp_halo_bytes.argtypes = [_VP, ctypes.c_int]
        L.fp_halo_bytes.restype = ctypes.c_size_t
        L.fp_pack_halo.argtypes = [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]
        _lib = L
    return _lib


class FPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{lib().fp_status_string(status).decode()}: {msg}")
        self.status = status


def _check(st, ctx=None, batch=None):
    if st != FP_OK:
        msg = ""
        if ctx:
            msg = lib().fp_last_error(ctx).decode()
        elif batch:
            msg = lib().fp_batch_last_error(batch).decode()
        raise FPError(st, msg)


def make_desc(dims, n, metric_order=6, scheme=FP_WENO5_JS, fp=1, characteristic=1,
              precision=FP_F64, bc=((0, 0), (0, 0), (0, 0)), gamma=1.4,
              q_inf=(1.4, 0.0, 0.0, 0.0, 2.5), global_lf=0, cut_width=0) -> fp_grid_desc:
    d = fp_grid_desc()
    d.dims = dims
    for k in range(3):
        d.n[k] = int(n[k])
        d.bc[k][0] = int(bc[k][0])
        d.bc[k][1] = int(bc[k][1])
    d.metric_order = metric_order
    d.scheme = scheme
    d.free_stream_preserving = fp
    d.characteristic = characteristic
    d.precision = precision
    d.gamma = gamma
    for v in range(5):
        d.q_inf[v] = float(q_inf[v])
    d.global_lf = int(global_lf)
    d.cut_width = int(cut_width)
    return d


def fp_ghost_width(M, scheme=FP_WENO5_JS):
    return lib().fp_ghost_width(M, scheme)


def fp_node_ghost_width(M, scheme=FP_WENO5_JS):
    return lib().fp_node_ghost_width(M, scheme)


def fp_init_grid(desc, nodes_host_ptr, ghost_nodes, stream=0):
    ctx = _VP()
    st = lib().fp_init_grid(ctypes.byref(desc), nodes_host_ptr, ghost_nodes, stream, ctypes.byref(ctx))
    if st != FP_OK:
        raise FPError(st, "fp_init_grid")
    return ctx


def fp_rhs(ctx, q_ptr, dqdt_ptr, stream=0):
    _check(lib().fp_rhs(ctx, q_ptr, dqdt_ptr, stream), ctx)


def fp_rhs_noalloc(ctx, q_ptr, dqdt_ptr, stream=0):
    """fp_rhs with its residual accumulator in the library's static device scratch."""
    _check(lib().fp_rhs_noalloc(ctx, q_ptr, dqdt_ptr, stream), ctx)


def fp_rk3_step(ctx, q_ptr, dt, stream=0):
    _check(lib().fp_rk3_step(ctx, q_ptr, float(dt), stream), ctx)


def fp_rk3_stage(ctx, q_ptr, dt, stage, stream=0):
    _check(lib().fp_rk3_stage(ctx, q_ptr, float(dt), int(stage), stream), ctx)


def fp_set_halo(ctx, direction, side, halo_ptr):
    _check(lib().fp_set_halo(ctx, int(direction), int(side), halo_ptr), ctx)


def fp_halo_bytes(ctx, direction):
    return lib().fp_halo_bytes(ctx, int(direction))


def fp_pack_halo(ctx, q_ptr, stage, direction, side, out_ptr, stream=0):
    _check(lib().fp_pack_halo(ctx, q_ptr, int(stage), int(direction), int(side), out_ptr, stream), ctx)


def fp_cfl_dt(ctx, q_ptr, cfl, stream=0):
    out = ctypes.c_double()
    _check(lib().fp_cfl_dt(ctx, q_ptr, float(cfl), ctypes.byref(out), stream), ctx)
    return out.value


def fp_get_metrics(ctx, host_ptr):
    _check(lib().fp_get_metrics(ctx, host_ptr), ctx)


def fp_get_face_metrics(ctx, direction, host_ptr):
    _check(lib().fp_get_face_metrics(ctx, direction, host_ptr), ctx)


def fp_get_device_status(ctx, stream=0):
    return lib().fp_get_device_status(ctx, stream)


def fp_launches_per_rhs(ctx):
    return lib().fp_launches_per_rhs(ctx)


def fp_launches_per_step(ctx):
    return lib().fp_launches_per_step(ctx)


def fp_get_cta_sizes(ctx):
    """(primary, alternative) threads per CTA of the context's sweep; alternative 0 if none."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().fp_get_cta_sizes(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def fp_get_tile(ctx, direction):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().fp_get_tile(ctx, direction, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def fp_set_tile(ctx, direction, faces, lines):
    _check(lib().fp_set_tile(ctx, direction, faces, lines), ctx)


def fp_free(ctx):
    lib().fp_free(ctx)


def fp_batch_create(ctxs, q_ptrs, autotune=1, stream=0):
    n = len(ctxs)
    arr = (_VP * n)(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    qs = (_VP * n)(*q_ptrs)
    out = _VP()
    st = lib().fp_batch_create(arr, n, qs, int(autotune), stream, ctypes.byref(out))
    if st != FP_OK:
        raise FPError(st, "fp_batch_create")
    return out


def fp_batch_create_linked(ctxs, q_ptrs, links, autotune=1, stream=0):
    """links: iterable of (a, dir, side, b): side `side` of direction `dir` of block a takes
    its ghost cells from block b."""
    n = len(ctxs)
    arr = (_VP * n)(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    qs = (_VP * n)(*q_ptrs)
    links = list(links)
    la = (fp_block_link * max(1, len(links)))(*[fp_block_link(*l) for l in links])
    out = _VP()
    st = lib().fp_batch_create_linked(arr, n, qs, la, len(links), int(autotune), stream, ctypes.byref(out))
    if st != FP_OK:
        raise FPError(st, "fp_batch_create_linked")
    return out


def fp_batch_rk3_step(batch, dt, stream=0):
    _check(lib().fp_batch_rk3_step(batch, float(dt), stream), batch=batch)


def fp_batch_rhs(batch, dqdt_ptrs, stream=0):
    arr = (_VP * len(dqdt_ptrs))(*dqdt_ptrs)
    _check(lib().fp_batch_rhs(batch, arr, stream), batch=batch)


def fp_batch_launches_per_step(batch):
    return lib().fp_batch_launches_per_step(batch)


def fp_batch_get_tile(batch, block, direction):
    """(faces, lines) the batch runs block `block` with in `direction`."""
    a, b = ctypes.c_int(), ctypes.c_int()
    st = lib().fp_batch_get_tile(batch, int(block), int(direction), ctypes.byref(a), ctypes.byref(b))
    if st != FP_OK:
        raise FPError(st, "fp_batch_get_tile")
    return a.value, b.value


def fp_batch_free(batch):
    lib().fp_batch_free(batch)


def fp_state_bytes(ctx):
    return lib().fp_state_bytes(ctx)


def fp_pipe_create(ctxs, q_host_ptrs, ngroups=4, autotune=1):
    n = len(ctxs)
    arr = (_VP * n)(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    qs = (_VP * n)(*q_host_ptrs)
    out = _VP()
    st = lib().fp_pipe_create(arr, n, qs, int(ngroups), int(autotune), ctypes.byref(out))
    if st != FP_OK:
        raise FPError(st, "fp_pipe_create")
    return out


def fp_pipe_rk3_step_host(pipe, q_host_ptrs, dt, stream=0):
    qs = (_VP * len(q_host_ptrs))(*q_host_ptrs)
    st = lib().fp_pipe_rk3_step_host(pipe, qs, float(dt), stream)
    if st != FP_OK:
        raise FPError(st, lib().fp_pipe_last_error(pipe).decode())


def fp_pipe_set_ordered(pipe, ordered):
    st = lib().fp_pipe_set_ordered(pipe, int(ordered))
    if st != FP_OK:
        raise FPError(st, "fp_pipe_set_ordered")


def fp_pipe_groups(pipe):
    return lib().fp_pipe_groups(pipe)


def fp_pipe_launches_per_step(pipe):
    return lib().fp_pipe_launches_per_step(pipe)


def fp_pipe_free(pipe):
    lib().fp_pipe_free(pipe)


def fp_balanced_groups(weights, ngroups):
    """Group index of each weighted item (the partition of batch branches and pipe groups)."""
    n = len(weights)
    w = (ctypes.c_longlong * max(n, 1))(*[int(x) for x in weights])
    out = (ctypes.c_int * max(n, 1))()
    st = lib().fp_balanced_groups(w, n, int(ngroups), out)
    if st != FP_OK:
        raise FPError(st, "fp_balanced_groups: invalid arguments")
    return list(out[:n])


def fp_debug_fail_allocation(n):
    """Make the n-th library allocation from now fail as out of memory (n < 0: cancel)."""
    return lib().fp_debug_fail_allocation(int(n))


def fp_bounds_checking():
    """1 when the loaded library is the bounds-checking build, else 0."""
    return lib().fp_bounds_checking()


def fp_probe_peaks(stream=0):
    """Measured FP32 (FFMA), FP32x2 (FFMA2) and FP64 (DFMA) TFLOP/s of the current device."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib().fp_probe_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), stream)
    if st != FP_OK:
        raise FPError(st, "fp_probe_peaks")
    return a.value, b.value, c.value
