"""One large block split into slabs along one direction, each slab advanced by its own
process (one GPU each), with a halo exchange before every Runge-Kutta stage.

The residual of a point depends on the states within G = fp_ghost_width points along each
direction (Sec. 3.2: the five- or seven-point upwind stencils and the order-M face
interpolation), so a slab whose split sides are FP_BC_HALO computes exactly the unsplit
block's values once its halos hold its neighbours' G cells of the same RK stage.  The
geometry needs no exchange: each slab is built from the neighbours' nodes as ghost nodes
(inputs.split_grid with side_bc=BC_HALO), so every metric equals the unsplit grid's.  The
time step is the minimum over all slabs (one all-reduce per step).

Message order between two neighbours is fixed (each rank posts its receives, low side first,
then its sends, high side first, with tags naming the receiving side, all in one group of
point-to-point operations), so the same code runs over NCCL (device tensors) and gloo (host
tensors), including two ranks that are each other's low and high neighbour on a periodic
split.
"""
from __future__ import annotations

import numpy as np

from . import binding as B
from . import inputs as I


def slab_sizes(n: int, parts: int):
    """Extents of `parts` consecutive slabs of n points, as equal as possible."""
    if parts < 1 or parts > n:
        raise ValueError("need 1 <= parts <= n")
    return [len(a) for a in np.array_split(np.arange(n), parts)]


def slab_grids(grid: I.Grid, parts: int, direction: int | None = None):
    """The slabs of a grid along `direction` (default: the slowest index, k in 3-D, j in
    2-D), their split sides FP_BC_HALO.  Returns (grids, neighbours, sizes), neighbours[p] =
    (low neighbour or None, high neighbour or None)."""
    d = (grid.dims - 1) if direction is None else direction
    sizes = slab_sizes(grid.n[d], parts)
    grids, links = I.split_grid(grid, d, sizes, side_bc=I.BC_HALO)
    nbr = [[None, None] for _ in range(parts)]
    for a, _, side, b in links:
        nbr[a][side] = b
    return grids, [tuple(x) for x in nbr], sizes


class LocalHalo:
    """Halo exchange between slabs held by one process (several slabs on one GPU, or the
    single slab of a periodic block that is its own neighbour): direct copies."""

    def __init__(self, backends, neighbours):
        self.backends = list(backends)
        self.neighbours = list(neighbours)

    def exchange(self, states, stage):
        for b, q in zip(self.backends, states):
            for side in (0, 1):
                if b.has_halo(side):
                    b.pack(q, stage, side)
        for p, b in enumerate(self.backends):
            lo, hi = self.neighbours[p]
            if lo is not None:             # my low halo: the low neighbour's high-side cells
                b.recv_into(0, self.backends[lo].send[1])
            if hi is not None:             # my high halo: the high neighbour's low-side cells
                b.recv_into(1, self.backends[hi].send[0])


class DistHalo:
    """Halo exchange between processes through torch.distributed point-to-point messages.

    staging="host" moves the messages through page-locked host buffers (for a transport that
    takes no device buffers, such as gloo, with device slabs): the packed cells are copied to
    the host before the exchange and the received ones back to the device halos after it, on
    the current stream, so the next stage sees them."""

    def __init__(self, backend, neighbours, rank, staging=None):
        self.b = backend
        self.lo, self.hi = neighbours
        self.rank = rank
        self.staging = staging
        if staging not in (None, "host"):
            raise ValueError("staging is None or 'host'")
        if staging == "host":
            import torch
            pin = getattr(backend, "device", "cpu") != "cpu"
            self.hsend = [None if t is None else torch.empty(t.shape, dtype=t.dtype, pin_memory=pin) for t in backend.send]
            self.hrecv = [None if t is None else torch.empty(t.shape, dtype=t.dtype, pin_memory=pin) for t in backend.recv]

    def exchange(self, q, stage):
        import torch.distributed as dist
        b = self.b
        for side in (0, 1):
            if b.has_halo(side):
                b.pack(q, stage, side)
        b.sync()
        send, recv = (self.hsend, self.hrecv) if self.staging else (b.send, b.recv)
        if self.staging:
            for side in (0, 1):
                if send[side] is not None:
                    send[side].copy_(b.send[side])        # waits for the packing
        ops = []
        # receives: low halo first (tag 0), then high halo (tag 1); a halo on side s is sent
        # by the neighbour's side 1 - s
        if self.lo is not None:
            ops.append(dist.P2POp(dist.irecv, recv[0], self.lo, tag=0))
        if self.hi is not None:
            ops.append(dist.P2POp(dist.irecv, recv[1], self.hi, tag=1))
        # sends: high side first (it lands in the high neighbour's low halo, tag 0)
        if self.hi is not None:
            ops.append(dist.P2POp(dist.isend, send[1], self.hi, tag=0))
        if self.lo is not None:
            ops.append(dist.P2POp(dist.isend, send[0], self.lo, tag=1))
        # one group of point-to-point operations (NCCL runs them together, so two ranks that
        # both receive first cannot wait on each other)
        for r in dist.batch_isend_irecv(ops) if ops else []:
            r.wait()
        if self.staging:
            for side in (0, 1):
                if recv[side] is not None:
                    b.recv_into(side, recv[side])


class SlabStepper:
    """SSP-RK3 steps of one slab (or of several local slabs) with a halo exchange before
    every stage, and the time step shared by all slabs."""

    def __init__(self, backends, halo, states, group=None):
        self.backends = list(backends)
        self.halo = halo
        self.states = list(states)
        self.group = group

    def _exchange(self, stage):
        if isinstance(self.halo, DistHalo):
            self.halo.exchange(self.states[0], stage)
        else:
            self.halo.exchange(self.states, stage)

    def rk3_step(self, dt):
        for stage in range(3):
            self._exchange(stage)
            for b, q in zip(self.backends, self.states):
                b.stage(q, dt, stage)

    def rhs(self, outs):
        self._exchange(0)
        for b, q, o in zip(self.backends, self.states, outs):
            b.rhs(q, o)
        return outs

    def cfl_dt(self, cfl):
        dt = min(b.cfl_dt(q, cfl) for b, q in zip(self.backends, self.states))
        try:
            import torch
            import torch.distributed as dist
            if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
                # NCCL reduces device tensors; gloo takes the value on the host
                dev = "cpu" if dist.get_backend(self.group) == "gloo" else self.backends[0].device
                t = torch.tensor([dt], dtype=torch.float64, device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
                dt = float(t.item())
        except ImportError:
            pass
        return dt


class BlockSlab:
    """A slab on the GPU: a solver.Block whose FP_BC_HALO sides read device halo buffers that
    this object owns, packed and stepped through the C ABI."""

    def __init__(self, block, direction):
        import torch
        self.block = block
        self.d = direction
        self.device = "cuda"
        ni, nj, nk = block.n
        shape = [5, nk, nj, ni]
        shape[3 - direction] = block.G
        self.recv, self.send = [None, None], [None, None]
        bc = block.desc.bc[direction]
        for side in (0, 1):
            if bc[side] == B.FP_BC_HALO:
                self.recv[side] = torch.empty(shape, dtype=block.dtype, device="cuda")
                self.send[side] = torch.empty(shape, dtype=block.dtype, device="cuda")
                assert self.recv[side].numel() * self.recv[side].element_size() == B.fp_halo_bytes(block.ctx, direction)
                B.fp_set_halo(block.ctx, direction, side, self.recv[side].data_ptr())

    def has_halo(self, side):
        return self.recv[side] is not None

    @staticmethod
    def _stream():
        import torch
        return torch.cuda.current_stream().cuda_stream

    def pack(self, q, stage, side):
        B.fp_pack_halo(self.block.ctx, q.data_ptr(), stage, self.d, side, self.send[side].data_ptr(), self._stream())

    def recv_into(self, side, src):
        self.recv[side].copy_(src)

    def sync(self):
        pass                               # NCCL and the copies are ordered on the current stream

    def stage(self, q, dt, stage):
        B.fp_rk3_stage(self.block.ctx, q.data_ptr(), dt, stage, self._stream())

    def rhs(self, q, out):
        B.fp_rhs(self.block.ctx, q.data_ptr(), out.data_ptr(), self._stream())

    def cfl_dt(self, q, cfl):
        return self.block.cfl_dt(q, cfl)
