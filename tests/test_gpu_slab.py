"""Slabs of one block with FP_BC_HALO sides on the GPU (several slabs in one process, their
halos refreshed by copies before every RK stage): the residual and RK3 steps of the split
block equal those of the unsplit block, up to the rounding of the separately compiled
boundary-rule sweep the split direction runs, and the FP64 residual equals the oracle's.
The exchange between processes (NCCL on GPUs) is the same code with another transport; it
is tested with gloo ranks on CPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2101_05886_gb300 import binding as B  # noqa: E402
from paper_2101_05886_gb300 import inputs as I  # noqa: E402
from paper_2101_05886_gb300 import slab as S  # noqa: E402
from paper_2101_05886_gb300.solver import Batch, Block  # noqa: E402
from tests.helpers import Parity, f32, residual_err, state_err, ulp_sensitivity  # noqa: E402

F64, F32 = B.FP_F64, B.FP_F32_MIXED


def _case(name, precision):
    M = 6
    Gn = O.node_ghost(M)
    if name == "wavy_k3":
        g = I.periodic_wavy_3d((24, 18, 20), L=10.0, amp=0.08, Gn=Gn)
        qinf = I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0)
        q, d, parts = I.vortex_3d(g, mach=0.8, eps=5.0, L=10.0), 2, 3
    elif name == "ogrid_i2":
        g = I.cylinder_ogrid((28, 18, 10), Lz=3.0, Gn=Gn, wall=True)
        qinf = I.uniform_qinf(0.8, 0.0)
        q, d, parts = I.random_smooth_state(g, qinf, amp=0.05, seed=7), 0, 2
    elif name == "cgrid_k2":
        g = I.cgrid_wing(n=(48, 24, 16), Gn=Gn)
        qinf = I.uniform_qinf(0.84, 3.0)
        q = I.fade_to_farfield(g, I.random_smooth_state(g, qinf, amp=0.03, seed=2), qinf)
        d, parts = 2, 2
    else:
        raise KeyError(name)
    if precision == F32:
        q, qinf = f32(q), f32(qinf)
    return g, qinf, q, d, parts, M


@pytest.mark.parametrize("name,precision", [("wavy_k3", F64), ("wavy_k3", F32), ("ogrid_i2", F64), ("cgrid_k2", F32)])
def test_halo_slabs_equal_the_unsplit_block(name, precision):
    g, qinf, q, d, parts, M = _case(name, precision)
    whole = Block(g, metric_order=M, precision=precision, q_inf=qinf)
    grids, nbrs, sizes = S.slab_grids(g, parts, d)
    blocks = [Block(gr, metric_order=M, precision=precision, q_inf=qinf) for gr in grids]
    backends = [S.BlockSlab(b, d) for b in blocks]
    ax = 3 - d
    cuts = np.cumsum(sizes)[:-1]
    states = [b.to_device(np.ascontiguousarray(p)) for b, p in zip(blocks, np.split(q, cuts, axis=ax))]
    stepper = S.SlabStepper(backends, S.LocalHalo(backends, nbrs), states)
    qd = whole.to_device(q)
    ref = whole.rhs(qd).cpu().numpy()
    got = np.concatenate([o.cpu().numpy() for o in stepper.rhs([torch.empty_like(s) for s in states])], axis=ax)
    cfg = O.cfg_for(g, M=M, qinf=qinf)
    met = O.metrics(cfg, g.nodes, g.Gn)
    P = Parity(cfg, met, q)
    tol = 1e-14 if precision == F64 else 1e-6
    assert residual_err(-got * P.invJ, -ref * P.invJ, P.tau) <= tol
    assert P.err(got) <= (max(1e-12, 2.0 * ulp_sensitivity(cfg, met, q)) if precision == F64 else 1e-5)
    dt = 0.5 * min(stepper.cfl_dt(0.5), whole.cfl_dt(qd, 0.5))
    for _ in range(2):
        stepper.rk3_step(dt)
        whole.rk3_step(qd, dt)
    torch.cuda.synchronize()
    stepped = np.concatenate([s.cpu().numpy() for s in states], axis=ax)
    assert state_err(stepped - q, qd.cpu().numpy() - q) <= (1e-13 if precision == F64 else 1e-5)
    if precision == F64:
        qo = O.rk3_step(cfg, met, O.rk3_step(cfg, met, q, dt), dt)
        assert state_err(stepped - q, qo - q) <= 1e-11
    assert all(b.status() == B.FP_OK for b in blocks)
    for b in blocks + [whole]:
        b.close()


def _process_slab(rank, world, port, name, precision, q_out):
    """One process, one slab on cuda:0, halos exchanged with the other process through host
    memory over gloo (DistHalo staging="host"): its residual and two RK3 steps."""
    import os

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, qinf, q, d, parts, M = _case(name, precision)
    grids, nbrs, sizes = S.slab_grids(g, world, d)
    ax = 3 - d
    k0 = sum(sizes[:rank])
    blk = Block(grids[rank], metric_order=M, precision=precision, q_inf=qinf)
    sl = S.BlockSlab(blk, d)
    mine = np.ascontiguousarray(np.take(q, np.arange(k0, k0 + sizes[rank]), axis=ax))
    state = blk.to_device(mine)
    stepper = S.SlabStepper([sl], S.DistHalo(sl, nbrs[rank], rank, staging="host"), [state])
    rhs = stepper.rhs([torch.empty_like(state)])[0].cpu().numpy()
    dt = stepper.cfl_dt(0.5) * 0.5
    for _ in range(2):
        stepper.rk3_step(dt)
    torch.cuda.synchronize()
    q_out.put((rank, rhs, state.cpu().numpy(), dt, blk.status()))
    dist.barrier()
    blk.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("name,precision", [("wavy_k3", F64), ("wavy_k3", F32)])
def test_two_processes_with_host_staged_halos_equal_the_unsplit_block(name, precision):
    """The slab decomposition as it runs across processes (one slab per process, the halo cells
    packed on the device, exchanged between the processes before every RK stage, the time step
    reduced over them), here with two processes that share this GPU and exchange through host
    memory over gloo.  No kernel of one process waits on the other's; the processes meet on the
    host between stages.  Their residual and two RK3 steps equal the unsplit block's."""
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q_out = ctx.Queue()
    procs = [ctx.Process(target=_process_slab, args=(r, 2, port, name, precision, q_out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q_out.get(timeout=600) for _ in range(2)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(r[4] == B.FP_OK for r in res)
    assert res[0][3] == res[1][3]                      # one time step for both processes
    g, qinf, q, d, parts, M = _case(name, precision)
    ax = 3 - d
    whole = Block(g, metric_order=M, precision=precision, q_inf=qinf)
    qd = whole.to_device(q)
    ref = whole.rhs(qd).cpu().numpy()
    got = np.concatenate([r[1] for r in res], axis=ax)
    cfg = O.cfg_for(g, M=M, qinf=qinf)
    P = Parity(cfg, O.metrics(cfg, g.nodes, g.Gn), q)
    assert residual_err(-got * P.invJ, -ref * P.invJ, P.tau) <= (1e-14 if precision == F64 else 1e-6)
    dt = res[0][3]
    for _ in range(2):
        whole.rk3_step(qd, dt)
    torch.cuda.synchronize()
    stepped = np.concatenate([r[2] for r in res], axis=ax)
    assert state_err(stepped - q, qd.cpu().numpy() - q) <= (1e-13 if precision == F64 else 1e-5)
    whole.close()


def test_halo_blocks_refuse_calls_that_cannot_refresh_their_halos():
    g, qinf, q, d, parts, M = _case("wavy_k3", F64)
    grids, nbrs, sizes = S.slab_grids(g, parts, d)
    blk = Block(grids[0], metric_order=M, precision=F64, q_inf=qinf)
    qd = blk.to_device(np.ascontiguousarray(q[:, :sizes[0]]))
    with pytest.raises(B.FPError):                     # halo buffers not registered yet
        blk.rhs(qd)
    with pytest.raises(B.FPError):                     # a side that is not FP_BC_HALO
        B.fp_set_halo(blk.ctx, 0, 0, qd.data_ptr())
    S.BlockSlab(blk, d)                                # registers both halos
    with pytest.raises(B.FPError):                     # one call cannot exchange between stages
        blk.rk3_step(qd, 1e-3)
    with pytest.raises(B.FPError):                     # nor can a batch graph
        Batch([blk], [qd], autotune=False)
    with pytest.raises(B.FPError):
        B.fp_rk3_stage(blk.ctx, qd.data_ptr(), 1e-3, 3)
    blk.close()
