"""Benchmark of the free-stream-preserving residual sweep on GB300.

Default workload: 64 blocks of seeded uneven sizes (each side U{32..128}; half
cylinder O-grids, half periodic wavy grids), Mach 3 stream with a 1e-3 smooth
perturbation, WENO5-JS FP form, 6th-order metrics, FP32 state and arithmetic on
FP64-built metrics, all blocks advanced by one CUDA-graph replay per SSP-RK3
step (two independent chains of the graph, each with half of the blocks and one
persistent launch per direction pass), autotuned tiles.

Metric: Mcell-RHS/s per RK stage = interior points x RK stages / second.
Prints one JSON line (rank 0).  --impl reference times the serial FP64 oracle
on the host cores instead.
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
# FP32 floating-point operations per point per direction pass of the WENO5-JS FP sweep
# (FFMA counted as 2), counted by ncu on the 16-block subset of the workload
# (an ncu capture of the FP32 sweep).  The pass is bound by FP32 instruction issue.
FLOPS_PER_POINT_PASS_F32 = 2280.0
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes per point per direction pass measured by ncu for the current kernel (16-block
# capture of two RK stages of one graph branch; mean over an RK step, whose second and third
# stages also read Q^n in the last pass: 95.7-97.0 B depending on the branch captured), scaled
# to a pass over the 64-block workload.
TRAFFIC_BYTES_PER_POINT_PASS = 96.4


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


def relative_error(a, b, floor_frac=0.1):
    """Largest per-component max |a - b| / max(max |b_c|, 10 % of the largest component's max),
    the parity metric of the tests, on device tensors [5, ...]."""
    tau = floor_frac * b.abs().max().item()
    e = 0.0
    for c in range(b.shape[0]):
        scale = max(b[c].abs().max().item(), tau)
        e = max(e, (a[c] - b[c]).abs().max().item() / scale if scale > 0 else 0.0)
    return e


def pipe_groups_used(pipe):
    from paper_2101_05886_gb300 import binding as B
    return B.fp_pipe_groups(pipe.pipe)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


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
    M = 6
    Gn = B.fp_node_ghost_width(M, B.FP_WENO5_JS)
    qinf = I.uniform_qinf(3.0, 0.0)
    prec = B.FP_F32_MIXED
    sizes = I.batched_block_sizes(64, 32, 128, 4)[:args.blocks]
    rng = np.random.default_rng(1004)
    blocks, states = [], []
    grid0 = None
    for k, n in enumerate(sizes):
        g = (I.cylinder_ogrid(n, Lz=float(rng.uniform(1.0, 8.0)), Gn=Gn) if k < 32
             else I.periodic_wavy_3d(n, L=10.0, amp=0.08, Gn=Gn))
        blk = Block(g, metric_order=M, precision=prec, q_inf=qinf)
        q = blk.to_device(I.perturbed_state(g, qinf, amp=1e-3, seed=k))
        if k == 0:
            grid0 = g
        blk.grid = None
        blocks.append(blk)
        states.append(q)
    ncells = sum(int(np.prod(n)) for n in sizes)
    batch = Batch(blocks, states, autotune=True)
    dt = min(b.cfl_dt(q, 0.5) for b, q in zip(blocks, states))
    stream = torch.cuda.current_stream()
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
    hbm, src = peaks()
    passes_per_step = 3 * 3
    launches_per_pass = launches_per_step // passes_per_step
    per_launch_ms = graph_ms / (args.steps * passes_per_step)
    alg_bytes_per_launch = BYTES_PER_CELL_STAGE_F32 * ncells / 3.0     # one of the 3 direction passes
    achieved_gbs = alg_bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    flops_per_launch = FLOPS_PER_POINT_PASS_F32 * ncells
    achieved_tf = flops_per_launch / (per_launch_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": round(achieved_tf, 2), "peak": round(FP32_PEAK_TFLOPS, 1),
            "unit": "TFLOP/s", "frac": round(achieved_tf / FP32_PEAK_TFLOPS, 4),
            "traffic": round(TRAFFIC_BYTES_PER_POINT_PASS * ncells) if args.blocks == 64 else None,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (maximum SM clock)",
            "kernel": "fpk::fp_sweep<float,6,0>", "pass_ms": round(per_launch_ms, 4),
            "launches_per_pass": launches_per_pass,
            "algorithmic_flops_per_pass": flops_per_launch,
            "hbm": {"achieved": round(achieved_gbs, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(achieved_gbs / hbm, 4), "peak_source": src,
                    "algorithmic_bytes_per_point_stage": round(BYTES_PER_CELL_STAGE_F32, 1)}}

    # ---- the FP32 residual's error against the FP64 sweep (itself within 1e-12 of the FP64
    # oracle in the parity tests), on block 0 of the workload at its current state
    err32 = None
    if rank == 0:
        b64 = Block(grid0, metric_order=M, precision=B.FP_F64, q_inf=qinf)
        q32 = states[0]
        r32 = blocks[0].rhs(q32).double()
        r64 = b64.rhs(q32.double())
        err32 = {"case": f"block 0 of the workload ({'x'.join(map(str, sizes[0]))} cylinder O-grid), "
                         "dQ/dt after the timed steps",
                 "max_rel": relative_error(r32, r64), "bound": 3e-5}
        b64.close()
        del r32, r64
    grid0 = None

    # ---- FP64 plain single block (256^3 wavy grid + vortex) on the same GPU
    fp64 = None
    if not args.no_fp64 and rank == 0:
        g = I.periodic_wavy_3d((256, 256, 256), L=10.0, amp=0.08, Gn=Gn)
        b64 = Block(g, metric_order=M, precision=B.FP_F64, q_inf=I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0))
        q64 = b64.to_device(I.vortex_3d(g, mach=0.8, eps=5.0, L=10.0))
        # FP32 sweep on the same grid and (float-rounded) state: its residual error
        b32 = Block(g, metric_order=M, precision=B.FP_F32_MIXED, q_inf=I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0))
        qr = q64.float()
        vortex_err = relative_error(b32.rhs(qr).double(), b64.rhs(qr.double()))
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
        fp64 = {"workload": "single block 256^3 wavy grid, Mach 0.8 + vortex, WENO5-JS FP, M6",
                "fp32_rhs_max_rel_error_vs_fp64": vortex_err,
                "value": 256 ** 3 * 3 * n64 / (ms64 * 1e-3) / 1e6, "unit": "Mcell/s",
                "ms_per_step": ms64 / n64, "dtype": "f64"}
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
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": "Mcell/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded grids and states)",
            "config": {"workload": WORKLOAD if args.blocks == 64 else WORKLOAD + f" (first {args.blocks} blocks only)",
                       "blocks": args.blocks, "cells_per_gpu": ncells,
                       "rk_stages_per_step": 3, "precision": "FP32 sweep on FP64-built metrics",
                       "parallelism": f"independent block batches per GPU x{world}",
                       "l2": "inputs larger than L2 (state %.0f MB)" % (ncells * 20 / 1e6)},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "fp64_plain_single_block": fp64,
            "c5_single_large": c5, "variants_256cubed_f32": variants, "c4_slip_walls": walls,
            "fp32_error_vs_fp64": err32,
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
                     "hbm_frac": round(gbs / peaks()[0], 4)}
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
    Mach 0.84 at 3 degrees, impulsive start from the uniform stream: FP32 sweep timed
    over args.c5_steps RK3 steps, FP64 plain over 1."""
    g = I.cgrid_wing(n=(512, 384, 512), Gn=Gn)
    qinf = I.uniform_qinf(0.84, 3.0)
    ncell = 512 * 384 * 512
    out = {"workload": "C-grid 512x384x512 (100.7M points), swept tapered thick wing-like body with a "
                       "slip wall and a C-grid wake cut, tanh wall spacing 1e-4 chord, Mach 0.84 at 3 deg, "
                       "impulsive start, WENO5-JS FP, M6"}
    for prec, key, nsteps in ((B.FP_F32_MIXED, "fp32", args.c5_steps), (B.FP_F64, "fp64", 1)):
        blk = Block(g, metric_order=M, precision=prec, q_inf=qinf)
        q = blk.to_device(I.uniform_state(g, qinf))
        rho0 = q[0].clone()
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
        out[key] = {"value": round(ncell * 3 * nsteps / (ms * 1e-3) / 1e6, 2), "unit": "Mcell/s",
                    "ms_per_step": round(ms / nsteps, 3), "steps": nsteps}
        out[key]["max_density_change"] = float((q[0] - rho0).abs().max().item())
        assert blk.status() == B.FP_OK
        blk.close()
        del q, rho0
        torch.cuda.empty_cache()
    del g
    return out


def _oracle_sample(n=40, seed=0):
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


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_pool(jobs):
    """Run the oracle jobs one process per host core (spawned interpreters: safe after CUDA
    has been initialised in this process)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        return pool.map(_oracle_worker, jobs)


def cpu_baseline(args):
    cores = _host_cores()
    res = _oracle_pool([(40, k, 10.0, 0, 0) for k in range(cores)])
    value = sum(r[0] / r[1] for r in res) / 1e6
    steps = sum(r[2] for r in res)
    return {"value": round(value, 4), "unit": "Mcell/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, one per host core, each RK3 steps of its own 40^3 cylinder O-grid "
                      f"block for 10 s ({steps} steps in all; Mach 3 + 1e-3 perturbation, WENO5-JS FP, M6), "
                      "serial FP64 C oracle"}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    cores = _host_cores()
    res = _oracle_pool([(24, k, 0.0, args.warmup, args.steps) for k in range(cores)])
    el = max(r[1] for r in res)
    v = sum(r[0] for r in res) / el / 1e6
    sample = (f"each step one RK3 step of one 24^3 cylinder O-grid block of the workload's family in each of "
              f"{cores} processes (one per host core), serial FP64 C oracle")
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
    ap.add_argument("--c5-steps", type=int, default=10)
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
