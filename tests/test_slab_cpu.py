"""Slab decomposition of one block across processes, on CPU ranks (gloo): the exchange
logic of paper_2101_05886_gb300.slab (neighbours, packing of the G cells next to each
split side, message order, one exchange per RK stage, the time step reduced over ranks)
drives a backend that evaluates each slab with the FP64 oracle on the slab grown by its
halos.  Two RK3 steps of the split block must equal two oracle steps of the unsplit block."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N = (10, 9, 14)          # the unsplit periodic wavy block (k split in two slabs of 7 >= G)
M = 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleSlab:
    """Test backend: one k-slab [k0, k1) of the periodic wavy grid, advanced by the oracle on
    the slab grown by its two halos (the RK stages written out as the oracle's step does)."""

    device = "cpu"

    def __init__(self, k0, k1, qinf):
        import oracle as O
        from paper_2101_05886_gb300 import inputs as I
        self.O = O
        G = O.ghost(M)
        self.G = G
        Gn = O.node_ghost(M)
        ext = I.periodic_wavy_3d(N, L=10.0, amp=0.08, Gn=Gn, k_range=(k0 - G, k1 + G))
        self.cfg = O.make_cfg(3, ext.n, M=M, bc=((0, 0), (0, 0), (2, 2)), qinf=qinf)
        self.met = O.metrics(self.cfg, ext.nodes, Gn)
        own = I.periodic_wavy_3d(N, L=10.0, amp=0.08, Gn=Gn, k_range=(k0, k1))
        self.cfg_own = O.make_cfg(3, own.n, M=M, bc=((0, 0), (0, 0), (2, 2)), qinf=qinf)
        self.met_own = O.metrics(self.cfg_own, own.nodes, Gn)
        shape = (5, G, N[1], N[0])
        self.recv = [torch.zeros(shape, dtype=torch.float64), torch.zeros(shape, dtype=torch.float64)]
        self.send = [torch.zeros(shape, dtype=torch.float64), torch.zeros(shape, dtype=torch.float64)]
        self.stages = [None, None, None]

    def has_halo(self, side):
        return True

    def pack(self, q, stage, side):
        src = q if stage == 0 else torch.from_numpy(self.stages[stage])
        self.send[side].copy_(src[:, :self.G] if side == 0 else src[:, -self.G:])

    def sync(self):
        pass

    def recv_into(self, side, src):
        self.recv[side].copy_(src)

    def _L(self, qs):
        ext = np.concatenate([self.recv[0].numpy(), qs, self.recv[1].numpy()], axis=1)
        _, dq = self.O.rhs(self.cfg, self.met, ext)
        return dq[:, self.G:-self.G]

    def stage(self, q, dt, stage):
        if stage == 0:
            self.stages[0] = q.numpy().copy()
            self.stages[1] = self.stages[0] + dt * self._L(self.stages[0])
        elif stage == 1:
            q1 = self.stages[1]
            self.stages[2] = 0.75 * self.stages[0] + 0.25 * (q1 + dt * self._L(q1))
        else:
            q2 = self.stages[2]
            q.copy_(torch.from_numpy((1.0 / 3.0) * self.stages[0] + (2.0 / 3.0) * (q2 + dt * self._L(q2))))

    def rhs(self, q, out):
        out.copy_(torch.from_numpy(self._L(q.numpy())))

    def cfl_dt(self, q, cfl):
        return self.O.cfl_dt(self.cfg_own, self.met_own, q.numpy(), cfl)


def _worker(rank, world, port, q_out, staging=None):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2101_05886_gb300 import inputs as I
    from paper_2101_05886_gb300 import slab as S
    full = I.periodic_wavy_3d(N, L=10.0, amp=0.08, Gn=12)
    grids, nbrs, sizes = S.slab_grids(full, world)
    k0 = sum(sizes[:rank])
    qinf = I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0)
    q_full = I.vortex_3d(full, mach=0.8, eps=5.0, L=10.0)
    q = torch.from_numpy(np.ascontiguousarray(q_full[:, k0:k0 + sizes[rank]]))
    b = OracleSlab(k0, k0 + sizes[rank], qinf)
    stepper = S.SlabStepper([b], S.DistHalo(b, nbrs[rank], rank, staging=staging), [q])
    dt = 0.5 * stepper.cfl_dt(0.5)
    rhs = stepper.rhs([torch.empty_like(q)])[0].numpy().copy()
    for _ in range(2):
        stepper.rk3_step(dt)
    q_out.put((rank, k0, dt, rhs, q.numpy().copy(), nbrs[rank]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("staging", [None, "host"])
def test_two_rank_slab_steps_equal_the_unsplit_oracle(staging):
    """The messages go straight between the ranks' halo buffers, or (staging="host") through
    separate host buffers, as for device slabs over a host transport."""
    import oracle as O
    from paper_2101_05886_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q_out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q_out, staging)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q_out.get(timeout=300) for _ in range(2)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    # a periodic split in two: each rank is the other's low and high neighbour
    assert res[0][5] == (1, 1) and res[1][5] == (0, 0)
    full = I.periodic_wavy_3d(N, L=10.0, amp=0.08, Gn=O.node_ghost(M))
    qinf = I.uniform_qinf(0.8, 0.0, rho=1.0, p=1.0)
    q = I.vortex_3d(full, mach=0.8, eps=5.0, L=10.0)
    cfg = O.cfg_for(full, M=M, qinf=qinf)
    met = O.metrics(cfg, full.nodes, full.Gn)
    dt = 0.5 * O.cfl_dt(cfg, met, q, 0.5)
    assert res[0][2] == dt and res[1][2] == dt          # the same, global, time step on both ranks
    _, dq = O.rhs(cfg, met, q)
    rhs = np.concatenate([r[3] for r in res], axis=1)
    assert np.array_equal(rhs, dq)
    qo = O.rk3_step(cfg, met, O.rk3_step(cfg, met, q, dt), dt)
    stepped = np.concatenate([r[4] for r in res], axis=1)
    assert np.array_equal(stepped, qo)


def test_slab_partition_and_neighbours():
    from paper_2101_05886_gb300 import inputs as I
    from paper_2101_05886_gb300 import slab as S
    assert S.slab_sizes(10, 3) == [4, 3, 3]
    g = I.cylinder_ogrid((12, 10, 11), Lz=2.0, Gn=12)        # k periodic: the ring closes
    grids, nbrs, sizes = S.slab_grids(g, 3)
    assert sizes == [4, 4, 3] and nbrs == [(2, 1), (0, 2), (1, 0)]
    assert all(gr.bc[2] == (I.BC_HALO, I.BC_HALO) for gr in grids)
    w = I.cgrid_wing(n=(48, 24, 16), Gn=12)                  # k not periodic: the ends keep their rule
    grids, nbrs, sizes = S.slab_grids(w, 2)
    assert nbrs == [(None, 1), (0, None)]
    assert grids[0].bc[2] == (w.bc[2][0], I.BC_HALO) and grids[1].bc[2] == (I.BC_HALO, w.bc[2][1])
    # every slab's nodes are the unsplit grid's, ghosts included
    k0 = 0
    for gr, n in zip(grids, sizes):
        assert np.array_equal(gr.nodes, w.nodes[:, k0:k0 + n + 2 * w.Gn])
        k0 += n
