"""Benchmark of the free-stream-preserving residual sweep on GB300.

Default workload: 64 blocks of seeded uneven sizes (each side U{32..128}; half
cylinder O-grids, half periodic wavy grids), Mach 3 stream with a 1e-3 smooth
perturbation, WENO5-JS FP form, 6th-order metrics, FP32 state and arithmetic on
FP64-built metrics, all blocks advanced by one CUDA-graph replay per SSP-RK3
step (two independent chains of the graph, each with half of the blocks and one
persistent launch per direction pass), autotuned tiles.  Under torchrun every
rank advances its own share of a batch of 64 x N blocks (the same family,
assigned by point count with fp_balanced_groups) with one time step, the
minimum over ranks of the CFL steps: weak scaling, no data-path collective.

Metric: Mcell-RHS/s per RK stage = interior points x RK stages / second.
Prints one JSON line (rank 0).  Beside the headline: the measured FP32/FP64
arithmetic peaks the roofline divides by, the linear-upwind scheme on the same
batched workload, an end-to-end run through the C ABI with host states, the
plain FP64 single block, scheme variants, slip walls, the 100M-point C-grid
and the oracle timed on the host cores.  --impl reference times the serial
FP64 oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-RHS/s per RK stage"
WORKLOAD = "batched multi-block: 64 blocks U{32..128}^3 (32 cylinder O-grids, 32 wavy), Mach 3 + 1e-3 perturbation, WENO5-JS FP, M6 metrics"
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

# Algorithmic bytes per interior point per RK stage of the FP32 form:
# state: read Q^(s) 20 + read Q^n (stages 2,3 only: 2/3 * 20) + write Q^(s+1) 20;
# cell metrics 9 + 1/J as float 40; face metrics 3 directions x 3 floats 36; per-point
# face-metric differences 3 directions x 3 floats 36.
BYTES_PER_CELL_STAGE_F32 = 20 + 20 * 2.0 / 3.0 + 20 + 40 + 36 + 36
BYTES_PER_CELL_STAGE_F64 = 2 * BYTES_PER_CELL_STAGE_F32
# Algorithmic FP32 operations per point per direction pass (one face per point and pass),
# counted from the steps of the face flux: characteristic WENO5-JS FP about 2,000
# (projection of the stencil differences 720, reconstruction 600, reference-state
# differences 270, eigensystem 140, reference state / face flux / back-projection 250);
# linear upwind projected after the (linear) reconstruction about 700 (reference-state
# differences 270, central and dissipation sums 120, eigensystem 140, one projection and
# back-projection 60, reference state and speeds 110).
ALG_FLOPS_PER_POINT_PASS = {"weno5_char": 2000.0, "lu5_char": 700.0}
# FP32 operations the kernels execute per point and pass, counted by ncu on the 16-block
# subset (FFMA 2, FFMA2 4, FADD/FMUL 1, FADD2/FMUL2 2): reported beside the algorithmic count.
EXEC_FLOPS_PER_POINT_PASS = {"weno5_char": 2145.0, "lu5_char": 1132.0}
# DRAM bytes per point per direction pass measured by ncu (16-block capture, mean over an RK
# step: 96.4 B), scaled to a pass over the workload.  The linear-upwind sweep makes the same
# loads and stores (78.0 / 99.4 / 100.8 B per point in its captured passes against 77.9 /
# 99.8 / 101.1 B for WENO5).
TRAFFIC_BYTES_PER_POINT_PASS = {"weno5_char": 96.4, "lu5_char": 96.4}
ORACLE_SAMPLE_N = 32           # side of the O-grid block each host core advances (both CPU arms)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names[1:], p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(x, device="cpu"):
    """Max of a per-rank scalar over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(points_per_rank, stages, ms_max, world):
    """Whole-job Mcell-RHS/s per RK stage: every rank advances its own blocks, the job
    takes as long as the slowest rank."""
    return world * points_per_rank * stages / (ms_max * 1e-3) / 1e6


def residual_error(dq32, dq64, met64, q, dims=3, gamma=1.4):
    """FP32 against FP64 in the parity metric of the tests: per component c, on the residual
    R = -dQ/dt (1/J), max |R32 - R64| / max(max |R64_c|, 1e-3 max |F~_c|), F~ = k . (F, G, H)
    the contravariant flux over the swept directions.  dq32, dq64, q: host arrays [5, nk, nj, ni];
    met64: the FP64 block's metrics [10, nk+2G, nj+2G, ni+2G]."""
    n = q.shape[1:]
    G = (met64.shape[-1] - n[2]) // 2
    m = met64[:, G:G + n[0], G:G + n[1], G:G + n[2]]
    invJ = m[9]
    rho = q[0]
    u, v, w = q[1] / rho, q[2] / rho, q[3] / rho
    p = (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w))
    scale = np.zeros(5)
    for d in range(dims):
        k = m[3 * d:3 * d + 3]
        U = u * k[0] + v * k[1] + w * k[2]
        for c, f in enumerate((rho * U, q[1] * U + p * k[0], q[2] * U + p * k[1], q[3] * U + p * k[2],
                               (q[4] + p) * U)):
            scale[c] = max(scale[c], np.abs(f).max())
    e = 0.0
    for c in range(5):
        r32, r64 = -dq32[c] * invJ, -dq64[c] * invJ
        e = max(e, np.abs(r32 - r64).max() / max(np.abs(r64).max(), 1e-3 * scale[c]))
    return e


def pipe_groups_used(pipe):
    from paper_2101_05886_gb300 import binding as B
    return B.fp_pipe_groups(pipe.pipe)


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json: STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def rank_share(sizes, world, rank):
    """Block indices of this rank: the blocks are assigned to ranks by point count with the
    library's heaviest-first partition (fp_balanced_groups), so every rank gets about the
    same work."""
    from paper_2101_05886_gb300 import binding as B
    if world == 1:
        return list(range(len(sizes)))
    group = B.fp_balanced_groups([int(np.prod(n)) for n in sizes], world)
    return [k for k, g in enumerate(group) if g == rank]


def workload_grids(I, Gn, nblocks, world, rank):
    """This rank's grids of the batched workload: nblocks x world blocks of the seeded family
    (block k a cylinder O-grid when k % 64 < 32, else a periodic wavy grid), the rank's share
    by rank_share.  Returns (indices, sizes of all blocks, grids of the rank's blocks)."""
    total = nblocks * world
    sizes = I.batched_block_sizes(max(64, total), 32, 128, 4)[:total]
    mine = set(rank_share(sizes, world, rank))
    rng = np.random.default_rng(1004)
    idx, grids = [], []
    for k, n in enumerate(sizes):
        cyl = k % 64 < 32
        lz = float(rng.uniform(1.0, 8.0)) if cyl else None     # drawn for every cylinder, owned or not
        if k not in mine:
            continue
        idx.append(k)
        grids.append(I.cylinder_ogrid(n, Lz=lz, Gn=Gn) if cyl else I.periodic_wavy_3d(n, L=10.0, amp=0.08, Gn=Gn))
    return idx, sizes, grids


def time_batch(torch, batch, dt, steps, warmup, stream, label="timed_leg"):
    """CUDA-event time of `steps` graph replays after `warmup` (ms, total) and the sum of the
    per-replay times (ms); the replays sit in an NVTX range named `label`."""
    for _ in range(warmup):
        batch.rk3_step(dt)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push(label)
    gs = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ge = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(steps):
        gs[s].record(stream)
        batch.rk3_step(dt)
        ge[s].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return e0.elapsed_time(e1), sum(a.elapsed_time(b) for a, b in zip(gs, ge))


def roofline(kind, ncells, pass_ms, launches_per_pass, fp32_peak, peak_src, full_workload):
    """ALU roofline of one direction pass over the batch (the unit the graph runs as
    `launches_per_pass` concurrent persistent launches), with the HBM fraction beside it."""
    hbm, hsrc = hbm_peak()
    alg = ALG_FLOPS_PER_POINT_PASS[kind] * ncells
    tf = alg / (pass_ms * 1e-3) / 1e12
    gbs = BYTES_PER_CELL_STAGE_F32 * ncells / 3.0 / (pass_ms * 1e-3) / 1e9
    ex = EXEC_FLOPS_PER_POINT_PASS.get(kind)
    tr = TRAFFIC_BYTES_PER_POINT_PASS.get(kind)
    return {"bound": "alu", "achieved": round(tf, 2), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
            "frac": round(tf / fp32_peak, 4),
            "traffic": round(tr * ncells) if (tr is not None and full_workload) else None,
            "peak_source": peak_src, "pass_ms": round(pass_ms, 4), "launches_per_pass": launches_per_pass,
            "algorithmic_flops_per_point_pass": ALG_FLOPS_PER_POINT_PASS[kind],
            "executed_flops_per_point_pass": ex,
            "executed_tflops": round(ex * ncells / (pass_ms * 1e-3) / 1e12, 2) if ex else None,
            "hbm": {"achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
                    "peak_source": hsrc, "algorithmic_bytes_per_point_stage": round(BYTES_PER_CELL_STAGE_F32, 1)}}


def run_gpu(args):
    import torch
    from paper_2101_05886_gb300 import binding as B
    from paper_2101_05886_gb300 import inputs as I
    from paper_2101_05886_gb300.solver import Batch, Block, Pipe

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    # measured arithmetic peaks of this GPU (the roofline's denominators)
    p32, p32x2, p64 = B.fp_probe_peaks(stream.cuda_stream)
    props = torch.cuda.get_device_properties(local)
    fp32_peak = max(p32, p32x2)
    peak_src = (f"measured on this GPU by fp_probe_peaks: FFMA {p32:.1f}, FFMA2 {p32x2:.1f} TFLOP/s "
                f"(FMA chains on all {props.multi_processor_count} SMs, best of 3)")
    M = 6
    Gn = B.fp_node_ghost_width(M, B.FP_WENO5_JS)
    qinf = I.uniform_qinf(3.0, 0.0)
    prec = B.FP_F32_MIXED
    idx, sizes, grids = workload_grids(I, Gn, args.blocks, world, rank)
    blocks, states = [], []
    for k, g in zip(idx, grids):
        blk = Block(g, metric_order=M, precision=prec, q_inf=qinf)
        states.append(blk.to_device(I.perturbed_state(g, qinf, amp=1e-3, seed=k)))
        blocks.append(blk)
    ncells = sum(int(np.prod(sizes[k])) for k in idx)
    batch = Batch(blocks, states, autotune=True)
    # one time step for every rank: the smallest CFL step of all blocks of all ranks
    dt = -max_over_ranks(-min(b.cfl_dt(q, 0.5) for b, q in zip(blocks, states)), "cuda")
    for _ in range(args.warmup):
        batch.rk3_step(dt)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gstart = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    gend = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for s in range(args.steps):
            gstart[s].record(stream)
            batch.rk3_step(dt)
            gend[s].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if world > 1:
            torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    graph_ms = sum(a.elapsed_time(b) for a, b in zip(gstart, gend))
    ms = max_over_ranks(ms, "cuda")
    stages = 3 * args.steps
    value = weak_scaling_value(ncells, stages, ms, world)
    launches_per_step = batch.launches_per_step()
    st = [b.status() for b in blocks]
    assert all(s == B.FP_OK for s in st), "non-finite state during the benchmark"

    # ---- end-to-end through the public API with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        # host-resident states (page-locked) advanced through the pipelined public API
        # (fp_pipe_*): every step copies each block's state in, advances it and copies it back
        hosts = [torch.empty(q.shape, dtype=q.dtype, pin_memory=True) for q in states]
        for h, q in zip(hosts, states):
            h.copy_(q)
        h2d = sum(h.numel() * h.element_size() for h in hosts)
        pipe = Pipe(blocks, hosts, groups=args.pipe_groups, autotune=True)
        pipe.rk3_step(dt)                             # warm-up
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            pipe.rk3_step(dt)
        f1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(f0.elapsed_time(f1), "cuda")
        e2e = {"value": weak_scaling_value(ncells, stages, ems, world), "unit": "Mcell/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
               "api": f"fp_pipe_rk3_step_host, {pipe_groups_used(pipe)} groups, pinned host states"}
        pipe.close()
        del hosts

    # ---- roofline of the dominant kernel (the sweep; every launch in the graph is one).  A
    # direction pass over all blocks is `launches_per_pass` concurrent launches (one per graph
    # branch, each on its share of the blocks), so the unit is the pass: its algorithmic work
    # over the pass time (graph time / passes)
    passes_per_step = 3 * 3
    launches_per_pass = launches_per_step // passes_per_step
    pass_ms = graph_ms / (args.steps * passes_per_step)
    full = args.blocks == 64 and world == 1
    roof = roofline("weno5_char", ncells, pass_ms, launches_per_pass, fp32_peak, peak_src, full)
    roof["kernel"] = "fpk::fp_sweep<float,6,0,false,1> (characteristic WENO5-JS, switches folded, 64-thread CTAs)"

    # ---- the FP32 residual's error against the FP64 sweep (itself within 1e-12 of the FP64
    # oracle in the parity tests), on the rank's first block at its current state
    def fp32_error(blk32, grid, q32, **kw):
        # the FP64 sweep takes the far-field state as the FP32 one holds it (float values)
        b64 = Block(grid, metric_order=M, precision=B.FP_F64, q_inf=np.float32(qinf).astype(np.float64), **kw)
        r32 = blk32.rhs(q32).double().cpu().numpy()
        r64 = b64.rhs(q32.double()).cpu().numpy()
        e = residual_error(r32, r64, b64.metrics(), q32.double().cpu().numpy())
        b64.close()
        return e

    err32 = None
    if rank == 0:
        err32 = {"case": f"block {idx[0]} of the workload ({'x'.join(map(str, sizes[idx[0]]))}), dQ/dt after "
                         "the timed steps, against the FP64 sweep on the same float inputs",
                 "max_rel": fp32_error(blocks[0], grids[0], states[0]), "bound": 1e-5}

    # ---- the linear-upwind scheme (projection after the linear reconstruction) on the same
    # batched workload, with the same states, tiles autotuned for it
    lu5 = None
    if args.lu5:
        lblocks = [Block(g, metric_order=M, scheme=B.FP_LINEAR_UPWIND5, precision=prec, q_inf=qinf) for g in grids]
        lstates = [q.clone() for q in states]
        lbatch = Batch(lblocks, lstates, autotune=True)
        lsteps = max(10, args.steps // 2)
        lms, lgraph = time_batch(torch, lbatch, dt, lsteps, 3, stream, "timed_lu5")
        lms = max_over_ranks(lms, "cuda")
        lpass = lgraph / (lsteps * passes_per_step)
        lu5 = {"workload": "the headline's batched workload with linear upwind (Eq. linear_upwind) in the FP form, "
                           "characteristic, M6, FP32",
               "value": round(weak_scaling_value(ncells, 3 * lsteps, lms, world), 2), "unit": "Mcell/s",
               "ms_per_step": round(lms / lsteps, 4), "steps": lsteps,
               "roofline": roofline("lu5_char", ncells, lpass, lbatch.launches_per_step() // passes_per_step,
                                    fp32_peak, peak_src, full),
               "finite": all(b.status() == B.FP_OK for b in lblocks)}
        lu5["roofline"]["kernel"] = "fpk::fp_sweep<float,6,1,false,2> (characteristic linear upwind, switches folded, 64-thread CTAs of a batch)"
        if rank == 0:
            lu5["fp32_error_vs_fp64"] = {"max_rel": fp32_error(lblocks[0], grids[0], lstates[0],
                                                               scheme=B.FP_LINEAR_UPWIND5), "bound": 1e-5}
        lbatch.close()
        for b in lblocks:
            b.close()
        del lstates
    grids = None

    # ---- FP64 plain single block (256^3 wavy grid + vortex) on the same GPU
    fp64 = None
    if not args.no_fp64 and rank == 0:
        g = I.periodic_wavy_3d((256, 256, 256), L=10.0, amp=0.08, Gn=Gn)
        b64 = Block(g, metric_order=M, precision=B.FP_F64, q_inf=I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0))
        q64 = b64.to_device(I.vortex_3d(g, mach=0.8, eps=5.0, L=10.0))
        # FP32 sweep on the same grid and (float-rounded) state: its residual error
        b32 = Block(g, metric_order=M, precision=B.FP_F32_MIXED, q_inf=I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0))
        qr = q64.float()
        vortex_err = residual_error(b32.rhs(qr).double().cpu().numpy(), b64.rhs(qr.double()).cpu().numpy(),
                                    b64.metrics(), qr.double().cpu().numpy())
        b32.close()
        del qr
        del g
        dt64 = b64.cfl_dt(q64, 0.5)
        b64.rk3_step(q64, dt64)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n64 = 2
        h0.record(stream)
        for _ in range(n64):
            b64.rk3_step(q64, dt64)
        h1.record(stream)
        torch.cuda.synchronize()
        ms64 = h0.elapsed_time(h1)
        tf64 = ALG_FLOPS_PER_POINT_PASS["weno5_char"] * 3 * 256 ** 3 * 3 * n64 / (ms64 * 1e-3) / 1e12
        fp64 = {"workload": "single block 256^3 wavy grid, Mach 0.8 + vortex, WENO5-JS FP, M6",
                "fp32_rhs_max_rel_error_vs_fp64": vortex_err,
                "value": 256 ** 3 * 3 * n64 / (ms64 * 1e-3) / 1e6, "unit": "Mcell/s",
                "ms_per_step": ms64 / n64, "dtype": "f64",
                "roofline": {"bound": "alu", "achieved": round(tf64, 3), "peak": round(p64, 3), "unit": "TFLOP/s",
                             "frac": round(tf64 / p64, 4),
                             "peak_source": "measured FP64 DFMA chain on this GPU (fp_probe_peaks)",
                             "algorithmic_flops_per_point_pass": ALG_FLOPS_PER_POINT_PASS["weno5_char"]}}
        b64.close()

    # ---- scheme variants on one 256^3 FP32 block: where each sits between the ALU and HBM bounds
    variants = None
    if args.variants and rank == 0:
        variants = run_variants(I, B, Block, Gn, M, torch, stream)

    # ---- the batch with slip walls on the cylinders
    walls = None
    if args.variants and rank == 0:
        walls = run_c4_walls(I, B, Block, Batch, Gn, M, torch, stream)

    # ---- single large C-grid (512 x 384 x 512, about 100M points), FP32 and FP64 plain
    c5 = None
    if args.c5 and rank == 0:
        for b in blocks:
            b.close()
        batch.close()
        blocks, states = [], []
        torch.cuda.empty_cache()
        c5 = run_c5(args, I, B, Block, Gn, M, torch, stream)

    result = None
    if rank == 0:
        cpu = None if args.no_cpu else cpu_baseline(args)
        oc3 = None if (args.no_cpu or not args.oracle_c3) else oracle_c3_rhs(args)
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": "Mcell/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded grids and states)",
            "config": {"workload": WORKLOAD if args.blocks == 64 else WORKLOAD + f" (first {args.blocks} blocks only)",
                       "blocks": args.blocks * world, "blocks_per_gpu": len(idx), "cells_per_gpu": ncells,
                       "rk_stages_per_step": 3, "precision": "FP32 sweep on FP64-built metrics",
                       "parallelism": f"blocks assigned to {world} GPU(s) by point count, one CFL step for all",
                       "l2": "inputs larger than L2 (state %.0f MB)" % (ncells * 20 / 1e6)},
            "device": {"name": props.name, "sm_count": props.multi_processor_count,
                       "fp32_ffma_tflops": round(p32, 2), "fp32_ffma2_tflops": round(p32x2, 2),
                       "fp64_dfma_tflops": round(p64, 3)},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "fp64_plain_single_block": fp64,
            "lu5_batched": lu5, "c5_single_large": c5, "variants_256cubed_f32": variants, "c4_slip_walls": walls,
            "fp32_error_vs_fp64": err32, "oracle_c3_full_rhs": oc3,
        }
        print(json.dumps(result))
    for b in blocks:
        b.close()
    batch.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_variants(I, B, Block, Gn, M, torch, stream, nsteps=5):
    """FP32 RK3 steps on one 256^3 wavy block (Mach 0.8 + vortex) for the paper's
    characteristic WENO5-JS, the linear-upwind scheme, component-wise WENO5-JS,
    characteristic WENO7-JS and characteristic WENOCU6 (all under the free-stream-preserving
    form, metric order M)."""
    Gn = max(Gn, B.fp_node_ghost_width(M, B.FP_WENO7_JS))
    g = I.periodic_wavy_3d((256, 256, 256), L=10.0, amp=0.08, Gn=Gn)
    qinf = I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0)
    q0 = I.vortex_3d(g, mach=0.8, eps=5.0, L=10.0)
    ncell = 256 ** 3
    out = {}
    for name, scheme, charw in (("weno5_char", B.FP_WENO5_JS, 1), ("lu5_char", B.FP_LINEAR_UPWIND5, 1),
                                ("weno5_comp", B.FP_WENO5_JS, 0), ("weno7_char", B.FP_WENO7_JS, 1),
                                ("wenocu6_char", B.FP_WENOCU6, 1)):
        blk = Block(g, metric_order=M, scheme=scheme, characteristic=charw, precision=B.FP_F32_MIXED,
                    q_inf=qinf)
        q = blk.to_device(q0)
        dt = blk.cfl_dt(q, 0.5)
        blk.rk3_step(q, dt)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(nsteps):
            blk.rk3_step(q, dt)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        v = ncell * 3 * nsteps / (ms * 1e-3) / 1e6
        gbs = v * 1e6 * BYTES_PER_CELL_STAGE_F32 / 1e9
        out[name] = {"value": round(v, 1), "unit": "Mcell/s", "hbm_algorithmic_gbs": round(gbs, 1),
                     "hbm_frac": round(gbs / hbm_peak()[0], 4)}
        blk.close()
    return out


def run_c4_walls(I, B, Block, Batch, Gn, M, torch, stream, nsteps=10):
    """The batched workload's 64 grids with slip walls on the 32 cylinders, Mach 0.8
    (local Lax-Friedrichs, as the headline): FP32, timed over nsteps RK3 steps.  The
    headline's Mach 3 cannot start impulsively at a wall: the rarefaction behind the
    cylinder drops the wall pressure to ~2e-3 of the stream and WENO-JS without a
    positivity limiter goes negative there (the FP64 oracle fails the same way)."""
    qinf = I.uniform_qinf(0.8, 0.0)
    sizes = I.batched_block_sizes(64, 32, 128, 4)
    rng = np.random.default_rng(1004)
    blocks, states = [], []
    for k, n in enumerate(sizes):
        g = (I.cylinder_ogrid(n, Lz=float(rng.uniform(1.0, 8.0)), Gn=Gn, wall=True) if k < 32
             else I.periodic_wavy_3d(n, L=10.0, amp=0.08, Gn=Gn))
        blk = Block(g, metric_order=M, precision=B.FP_F32_MIXED, q_inf=qinf)
        states.append(blk.to_device(I.perturbed_state(g, qinf, amp=1e-3, seed=k)))
        blk.grid = None
        blocks.append(blk)
    ncells = sum(int(np.prod(n)) for n in sizes)
    batch = Batch(blocks, states, autotune=True)
    dt = min(b.cfl_dt(q, 0.5) for b, q in zip(blocks, states))
    for _ in range(3):
        batch.rk3_step(dt)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(nsteps):
        batch.rk3_step(dt)
    e.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(e)
    ok = all(b.status() == B.FP_OK for b in blocks)
    out = {"workload": "the headline's 64 grids, cylinder O-grids with slip walls, Mach 0.8 + 1e-3 perturbation, "
                       "impulsive start, WENO5-JS FP, M6, local LF",
           "value": round(ncells * 3 * nsteps / (ms * 1e-3) / 1e6, 1), "unit": "Mcell/s",
           "ms_per_step": round(ms / nsteps, 3), "steps": nsteps,
           "launches_per_step": batch.launches_per_step(), "finite": ok}
    batch.close()
    for b in blocks:
        b.close()
    return out


def run_c5(args, I, B, Block, Gn, M, torch, stream):
    """C-grid 512x384x512 around a swept tapered wing-like body (slip wall, wake cut),
    Mach 0.84 at 3 degrees, impulsive start from the uniform stream.  FP32: ten untimed steps
    (the first is the warm-up), a copy of the state, then args.c5_steps timed steps.  FP64:
    args.c5_f64_steps timed steps from the same float start with the same dt.  Reported: the
    throughputs; positivity (minimum density and pressure) at the end of each run; where the
    largest density change is (i around the C, j away from the wall, k along the span); and
    how closely the FP32 steps track the FP64 steps after the same number of steps: per
    component max |dQ32 - dQ64| / max(max |dQ64_c|, 1e-3 max |dQ64|), dQ the change since the
    start."""
    g = I.cgrid_wing(n=(512, 384, 512), Gn=Gn)
    qinf = np.float32(I.uniform_qinf(0.84, 3.0)).astype(np.float64)
    ncell = 512 * 384 * 512
    out = {"workload": "C-grid 512x384x512 (100.7M points), swept tapered thick wing-like body with a "
                       "slip wall and a C-grid wake cut, tanh wall spacing 1e-4 chord, Mach 0.84 at 3 deg, "
                       "impulsive start, WENO5-JS FP, M6"}

    def summary(q, q0):
        rho = q[0]
        u2 = (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / rho
        p = 0.4 * (q[4] - 0.5 * u2)
        d = (rho - q0[0]).abs()
        flat = int(torch.argmax(d).item())
        k, rem = divmod(flat, 384 * 512)
        j, i = divmod(rem, 512)
        return {"min_density": float(rho.min().item()), "min_pressure": float(p.min().item()),
                "max_density_change": float(d.max().item()),
                "max_density_change_at": {"i": i, "j": j, "k": k, "density": float(rho[k, j, i].item())}}

    q0 = None
    snap32 = None
    dt = None
    for prec, key, nsteps in ((B.FP_F32_MIXED, "fp32", args.c5_steps), (B.FP_F64, "fp64", args.c5_f64_steps)):
        blk = Block(g, metric_order=M, precision=prec, q_inf=qinf)
        q = blk.to_device(I.uniform_state(g, qinf))
        if q0 is None:
            q0 = q.clone()
            dt = blk.cfl_dt(q, 0.5)
        if prec == B.FP_F32_MIXED:
            for _ in range(10):
                blk.rk3_step(q, dt)
            snap32 = q.clone()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(nsteps):
            blk.rk3_step(q, dt)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out[key] = {"value": round(ncell * 3 * nsteps / (ms * 1e-3) / 1e6, 2), "unit": "Mcell/s",
                    "ms_per_step": round(ms / nsteps, 3), "steps": nsteps,
                    "state_after": summary(q, q0.to(q.dtype)),
                    "finite": blk.status() == B.FP_OK}
        if prec == B.FP_F32_MIXED:
            out[key]["state_after_10_steps"] = summary(snap32, q0)
            out[key]["steps_before_timing"] = 10
        elif nsteps == 10:
            d32 = snap32.double() - q0.double()
            d64 = q - q0.double()
            floor = 1e-3 * d64.abs().max().item()
            errs = [((d32[c] - d64[c]).abs().max().item() / max(d64[c].abs().max().item(), floor)) for c in range(5)]
            out["fp32_vs_fp64_after_10_steps"] = {"max_rel": max(errs), "per_component": errs}
            del d32, d64
        blk.close()
        del q
        torch.cuda.empty_cache()
    out["dt"] = dt
    del g, q0, snap32
    return out


def _oracle_sample(n=ORACLE_SAMPLE_N, seed=0):
    """The oracle on a bounded sample of the workload: one cylinder O-grid block of n^3
    points from the batch's family (Mach 3 + 1e-3 perturbation, WENO5-JS FP, M6)."""
    import oracle as O
    from paper_2101_05886_gb300 import inputs as I
    M = 6
    g = I.cylinder_ogrid((n, n, n), Lz=4.0, Gn=O.node_ghost(M))
    qinf = I.uniform_qinf(3.0, 0.0)
    cfg = O.cfg_for(g, M=M, qinf=qinf)
    met = O.metrics(cfg, g.nodes, g.Gn)
    q = I.perturbed_state(g, qinf, amp=1e-3, seed=seed)
    dt = O.cfl_dt(cfg, met, q, 0.5)
    return cfg, met, q, dt, n ** 3


def _oracle_worker(job):
    """One host core's share: RK3 steps of the oracle on its own sample block, either for
    `seconds` (steps = 0) or for `warmup` + `steps` steps; returns (cell-stages, seconds, steps)."""
    n, seed, seconds, warmup, steps = job
    import oracle as O
    cfg, met, q, dt, ncell = _oracle_sample(n=n, seed=seed)
    for _ in range(warmup):
        q = O.rk3_step(cfg, met, q, dt)
    t0 = time.perf_counter()
    done = 0
    while (steps and done < steps) or (not steps and (done == 0 or time.perf_counter() - t0 < seconds)):
        q = O.rk3_step(cfg, met, q, dt)
        done += 1
    return ncell * 3 * done, time.perf_counter() - t0, done


def _oracle_c3_worker(job):
    """One host core's slab of the 256^3 wavy-grid vortex case (k0 <= k < k1): the oracle's
    residual on the slab grown by G points in k (zero-gradient there; i and j periodic),
    which reproduces the full-grid residual on the slab.  Returns (points, rhs seconds,
    metric seconds)."""
    k0, k1 = job
    import oracle as O
    from paper_2101_05886_gb300 import inputs as I
    M = 6
    G = O.ghost(M)
    g = I.periodic_wavy_3d((256, 256, 256), L=10.0, amp=0.08, Gn=O.node_ghost(M), k_range=(k0 - G, k1 + G))
    q = I.vortex_3d(g, mach=0.8, eps=5.0, L=10.0)
    cfg = O.make_cfg(3, g.n, M=M, bc=((0, 0), (0, 0), (2, 2)), qinf=I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0))
    t0 = time.perf_counter()
    met = O.metrics(cfg, g.nodes, g.Gn)
    t1 = time.perf_counter()
    O.rhs(cfg, met, q)
    t2 = time.perf_counter()
    return 256 * 256 * (k1 - k0), t2 - t1, t1 - t0


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_pool(jobs, fn=_oracle_worker):
    """Run the oracle jobs one process per host core (spawned interpreters: safe after CUDA
    has been initialised in this process)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        return pool.map(fn, jobs)


def _sample_text(cores):
    n = ORACLE_SAMPLE_N
    return (f"{cores} processes, one per host core, each advancing its own {n}^3 cylinder O-grid block of the "
            f"workload's family (Mach 3 + 1e-3 perturbation, WENO5-JS FP, M6) by RK3 steps; serial FP64 C oracle; "
            f"value = cell-stages of all processes / the slowest process's time")


def cpu_baseline(args):
    cores = _host_cores()
    res = _oracle_pool([(ORACLE_SAMPLE_N, k, 10.0, 1, 0) for k in range(cores)])
    el = max(r[1] for r in res)
    value = sum(r[0] for r in res) / el / 1e6
    steps = sum(r[2] for r in res)
    return {"value": round(value, 4), "unit": "Mcell/s", "cores": cores, "kind": "oracle",
            "sample": _sample_text(cores) + f" (about 10 s each after one untimed step; {steps} steps in all)"}


def oracle_c3_rhs(args):
    """The oracle's residual of the full 256^3 wavy-grid vortex case (C3), split into k-slabs,
    one per host core (the oracle itself stays serial)."""
    cores = _host_cores()
    bounds = np.linspace(0, 256, cores + 1).astype(int)
    jobs = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    res = _oracle_pool(jobs, _oracle_c3_worker)
    t_rhs = max(r[1] for r in res)
    return {"workload": "single block 256^3 wavy grid, Mach 0.8 + vortex, WENO5-JS FP, M6 (one residual)",
            "value": round(256 ** 3 / t_rhs / 1e6, 4), "unit": "Mcell/s", "cores": cores,
            "rhs_seconds": round(t_rhs, 2), "metric_seconds": round(max(r[2] for r in res), 2),
            "how": f"{len(jobs)} k-slabs, one oracle process per host core, each on its slab grown by 3 points"}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    cores = _host_cores()
    res = _oracle_pool([(ORACLE_SAMPLE_N, k, 0.0, args.warmup, args.steps) for k in range(cores)])
    el = max(r[1] for r in res)
    v = sum(r[0] for r in res) / el / 1e6
    sample = _sample_text(cores) + f" ({args.warmup} untimed and {args.steps} timed steps each)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Mcell/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded grids and states)", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": round(v, 4), "unit": "Mcell/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "Mcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--blocks", type=int, default=64, help="blocks of the workload (64 = the full workload)")
    ap.add_argument("--c5", type=int, default=1, help="also time the single 100M-point C-grid (1/0)")
    ap.add_argument("--c5-steps", type=int, default=100, help="timed FP32 RK3 steps of the C-grid")
    ap.add_argument("--c5-f64-steps", type=int, default=10, help="timed FP64 RK3 steps of the C-grid")
    ap.add_argument("--lu5", type=int, default=1, help="also time linear upwind on the batched workload (1/0)")
    ap.add_argument("--oracle-c3", type=int, default=1, help="also time the oracle's full 256^3 residual (1/0)")
    ap.add_argument("--variants", type=int, default=1, help="also time scheme variants on a 256^3 block (1/0)")
    ap.add_argument("--pipe-groups", type=int, default=4, help="groups of the pipelined host-state e2e run")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
