"""The C-ABI library loads and exports every symbol include/fp.h declares, and
rejects invalid arguments before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2101_05886_gb300 import binding as B
from paper_2101_05886_gb300 import build as BUILD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.lib()


def test_header_and_binding_list_the_same_entry_points():
    hdr = open(os.path.join(ROOT, "include", "fp.h")).read()
    declared = set(re.findall(r"\b(fp_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(B.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in B.EXPORTS:
        assert hasattr(lib, name), name


def test_ghost_widths(lib):
    assert [B.fp_ghost_width(m) for m in (2, 4, 6, 8)] == [3, 3, 3, 4]
    assert [B.fp_node_ghost_width(m) for m in (2, 4, 6, 8)] == [6, 9, 12, 16]
    assert [B.fp_ghost_width(m, B.FP_WENO7_JS) for m in (2, 4, 6, 8)] == [4, 4, 4, 4]
    assert [B.fp_node_ghost_width(m, B.FP_WENO7_JS) for m in (2, 4, 6, 8)] == [7, 10, 13, 16]


def test_status_strings(lib):
    for st in range(8):
        assert lib.fp_status_string(st) != b"unknown status"
    assert lib.fp_status_string(8) == b"unknown status"


def test_the_normal_build_does_not_check_bounds():
    assert B.fp_bounds_checking() == 0


@pytest.mark.parametrize("field,value", [("dims", 4), ("metric_order", 5), ("scheme", 4), ("precision", 3),
                                         ("gamma", 0.9), ("characteristic", 2), ("free_stream_preserving", -1)])
def test_invalid_descriptor_is_rejected_before_any_gpu_work(lib, field, value):
    d = B.make_desc(3, (8, 8, 8), metric_order=6)
    setattr(d, field, value)
    nodes = np.zeros(3 * 32 ** 3)
    ctx = ctypes.c_void_p()
    st = lib.fp_init_grid(ctypes.byref(d), nodes.ctypes.data, 12, None, ctypes.byref(ctx))
    assert st == B.FP_ERR_ARG and not ctx.value


def test_other_invalid_arguments(lib):
    d = B.make_desc(3, (8, 8, 8), metric_order=6)
    nodes = np.zeros(3 * 32 ** 3)
    ctx = ctypes.c_void_p()
    # too few node ghost layers, extent below the ghost width, bad boundary code, 2-D with nk != 1
    assert lib.fp_init_grid(ctypes.byref(d), nodes.ctypes.data, 11, None, ctypes.byref(ctx)) == B.FP_ERR_ARG
    d2 = B.make_desc(3, (2, 8, 8), metric_order=6)
    assert lib.fp_init_grid(ctypes.byref(d2), nodes.ctypes.data, 12, None, ctypes.byref(ctx)) == B.FP_ERR_ARG
    d3 = B.make_desc(3, (8, 8, 8), metric_order=6, bc=((0, 7), (0, 0), (0, 0)))
    assert lib.fp_init_grid(ctypes.byref(d3), nodes.ctypes.data, 12, None, ctypes.byref(ctx)) == B.FP_ERR_ARG
    # global Lax-Friedrichs speeds would be per slab on a block with halo sides
    d6 = B.make_desc(3, (8, 8, 8), metric_order=6, bc=((0, 0), (0, 0), (B.FP_BC_HALO, B.FP_BC_HALO)), global_lf=1)
    assert lib.fp_init_grid(ctypes.byref(d6), nodes.ctypes.data, 12, None, ctypes.byref(ctx)) == B.FP_ERR_ARG
    d4 = B.make_desc(2, (8, 8, 3), metric_order=2)
    assert lib.fp_init_grid(ctypes.byref(d4), nodes.ctypes.data, 6, None, ctypes.byref(ctx)) == B.FP_ERR_ARG
    d5 = B.make_desc(3, (8, 8, 8), metric_order=6, q_inf=(1.0, 0, 0, 0, -1.0))
    assert lib.fp_init_grid(ctypes.byref(d5), nodes.ctypes.data, 12, None, ctypes.byref(ctx)) == B.FP_ERR_ARG
    assert lib.fp_init_grid(ctypes.byref(d), None, 12, None, ctypes.byref(ctx)) == B.FP_ERR_ARG
    assert lib.fp_init_grid(ctypes.byref(d), nodes.ctypes.data, 12, None, None) == B.FP_ERR_ARG
    # null contexts and buffers
    assert lib.fp_rhs(None, None, None, None) == B.FP_ERR_ARG
    assert lib.fp_rk3_step(None, None, 0.1, None) == B.FP_ERR_ARG
    out = ctypes.c_double()
    assert lib.fp_cfl_dt(None, None, 0.5, ctypes.byref(out), None) == B.FP_ERR_ARG
    assert lib.fp_get_metrics(None, None) == B.FP_ERR_ARG
    assert lib.fp_get_device_status(None, None) == B.FP_ERR_ARG
    assert lib.fp_batch_rk3_step(None, 0.1, None) == B.FP_ERR_ARG
    bo = ctypes.c_void_p()
    assert lib.fp_batch_create(None, 0, None, 0, None, ctypes.byref(bo)) == B.FP_ERR_ARG
    lib.fp_free(None)
    lib.fp_batch_free(None)


def test_pipe_and_link_calls_reject_null_arguments(lib):
    """The pipe and linked-batch entry points reject missing arguments before any GPU work."""
    out = ctypes.c_void_p()
    assert lib.fp_state_bytes(None) == 0
    assert lib.fp_pipe_create(None, 1, None, 4, 0, ctypes.byref(out)) == B.FP_ERR_ARG
    assert lib.fp_pipe_create(None, 0, None, 4, 0, None) == B.FP_ERR_ARG
    assert lib.fp_pipe_rk3_step_host(None, None, 1e-3, None) == B.FP_ERR_ARG
    assert lib.fp_pipe_set_ordered(None, 1) == B.FP_ERR_ARG
    a, b = ctypes.c_int(), ctypes.c_int()
    assert lib.fp_get_cta_sizes(None, ctypes.byref(a), ctypes.byref(b)) == B.FP_ERR_ARG
    assert lib.fp_batch_get_tile(None, 0, 0, ctypes.byref(a), ctypes.byref(b)) == B.FP_ERR_ARG
    assert lib.fp_pipe_groups(None) == 0
    assert lib.fp_pipe_launches_per_step(None) == 0
    lib.fp_pipe_free(None)
    links = (B.fp_block_link * 1)(B.fp_block_link(0, 0, 1, 0))
    assert lib.fp_batch_create_linked(None, 1, None, links, 1, 0, None, ctypes.byref(out)) == B.FP_ERR_ARG
    assert lib.fp_batch_create_linked(None, 1, None, None, 1, 0, None, ctypes.byref(out)) == B.FP_ERR_ARG


def test_balanced_groups_rule(lib):
    """Heaviest first, each into the lightest group; ties in index order and to the lower group."""
    assert B.fp_balanced_groups([5, 5, 5, 5], 2) == [0, 1, 0, 1]
    assert B.fp_balanced_groups([1, 9, 3], 2) == [1, 0, 1]
    assert B.fp_balanced_groups([7, 2, 2, 3], 3) == [0, 2, 2, 1]   # 7, 3, then both 2s into the third
    assert B.fp_balanced_groups([4, 1], 5) == [0, 1]
    assert B.fp_balanced_groups([], 2) == []


def test_balanced_groups_lpt_bound_by_brute_force(lib):
    """Graham's bound for longest-processing-time-first scheduling on m groups: the heaviest
    group is at most (4/3 - 1/(3m)) of the optimum, found here by enumerating every partition;
    and no group is heavier than the lightest by more than the heaviest item."""
    import itertools
    rng = np.random.default_rng(11)
    for trial in range(60):
        m = 2 + trial % 2
        n = int(rng.integers(1, 9))
        w = [int(x) for x in rng.integers(1, 1000, size=n)]
        g = B.fp_balanced_groups(w, m)
        load = [sum(wk for wk, gk in zip(w, g) if gk == j) for j in range(m)]
        best = min(max(sum(wk for wk, gk in zip(w, a) if gk == j) for j in range(m))
                   for a in itertools.product(range(m), repeat=n))
        assert max(load) * 3 * m <= best * (4 * m - 1)
        assert max(load) - min(load) <= max(w)


def test_balanced_groups_on_the_batched_workload_subset(lib):
    """The 16-block subset of the batched workload splits 5,608,608 / 5,683,224 points."""
    from paper_2101_05886_gb300 import inputs as I
    sizes = I.batched_block_sizes(64, 32, 128, 4)[:16]
    w = [int(np.prod(n)) for n in sizes]
    g = B.fp_balanced_groups(w, 2)
    assert [sum(wk for wk, gk in zip(w, g) if gk == j) for j in range(2)] == [5608608, 5683224]


def test_balanced_groups_rejects_invalid_arguments(lib):
    one = (ctypes.c_longlong * 1)(1)
    out = (ctypes.c_int * 1)()
    assert lib.fp_balanced_groups(None, 1, 2, out) == B.FP_ERR_ARG
    assert lib.fp_balanced_groups(one, 1, 2, None) == B.FP_ERR_ARG
    assert lib.fp_balanced_groups(one, -1, 2, out) == B.FP_ERR_ARG
    assert lib.fp_balanced_groups(one, 1, 0, out) == B.FP_ERR_ARG
    neg = (ctypes.c_longlong * 1)(-1)
    assert lib.fp_balanced_groups(neg, 1, 2, out) == B.FP_ERR_ARG
    assert lib.fp_balanced_groups(None, 0, 2, None) == B.FP_OK


def test_scheduled_allocation_failure_returns_oom_before_any_gpu_work(lib):
    """The host-side failure hook: with the next allocation scheduled to fail, fp_init_grid
    returns FP_ERR_OOM (its first allocation is the node array, made before any other CUDA
    call) and hands back no context; the hook disarms itself after firing, and a pending
    failure can be cancelled."""
    d = B.make_desc(3, (8, 8, 8), metric_order=6)
    nodes = np.zeros(3 * 32 ** 3)
    ctx = ctypes.c_void_p()
    assert B.fp_debug_fail_allocation(0) == B.FP_OK
    st = lib.fp_init_grid(ctypes.byref(d), nodes.ctypes.data, 12, None, ctypes.byref(ctx))
    assert st == B.FP_ERR_OOM and not ctx.value
    assert B.fp_debug_fail_allocation(5) == B.FP_OK
    assert B.fp_debug_fail_allocation(-1) == B.FP_OK
    # invalid arguments are still rejected first, whatever is armed
    B.fp_debug_fail_allocation(0)
    d.metric_order = 5
    assert lib.fp_init_grid(ctypes.byref(d), nodes.ctypes.data, 12, None, ctypes.byref(ctx)) == B.FP_ERR_ARG
    B.fp_debug_fail_allocation(-1)
