"""Convenience wrapper over the C ABI for torch users: one block (context) of the
free-stream-preserving residual with its state tensors.  Argument marshalling
only; all computation happens in libfpgb300.so."""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Block:
    def __init__(self, grid, metric_order=6, scheme=B.FP_WENO5_JS, fp=1, characteristic=1,
                 precision=B.FP_F64, gamma=1.4, q_inf=(1.4, 0.0, 0.0, 0.0, 2.5), global_lf=0):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.grid = grid
        self.n = tuple(int(v) for v in grid.n)
        self.dims = grid.dims
        self.metric_order = metric_order
        self.precision = precision
        self.dtype = torch.float32 if precision == B.FP_F32_MIXED else torch.float64
        self.desc = B.make_desc(grid.dims, grid.n, metric_order, scheme, fp, characteristic,
                                precision, grid.bc, gamma, q_inf, global_lf, getattr(grid, "cut", 0))
        nodes = np.ascontiguousarray(grid.nodes, dtype=np.float64)
        ni, nj, nk = self.n
        gn = int(grid.Gn)
        want = (2, nj + 2 * gn, ni + 2 * gn) if grid.dims == 2 else (3, nk + 2 * gn, nj + 2 * gn, ni + 2 * gn)
        if nodes.shape != want:   # the C call reads exactly this many values
            raise ValueError(f"node array of shape {nodes.shape}, expected {want} for n={self.n}, Gn={gn}")
        self.ctx = B.fp_init_grid(self.desc, nodes.ctypes.data, gn, _stream())
        self.G = B.fp_ghost_width(metric_order, scheme)

    @property
    def shape(self):
        ni, nj, nk = self.n
        return (5, nk, nj, ni)

    def to_device(self, q: np.ndarray) -> torch.Tensor:
        return torch.as_tensor(np.ascontiguousarray(q)).to(device="cuda", dtype=self.dtype).contiguous()

    def rhs(self, q: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        assert q.dtype == self.dtype and q.is_contiguous() and tuple(q.shape) == self.shape
        if out is None:
            out = torch.empty_like(q)
        B.fp_rhs(self.ctx, q.data_ptr(), out.data_ptr(), _stream())
        return out

    def rk3_step(self, q: torch.Tensor, dt: float) -> torch.Tensor:
        assert q.dtype == self.dtype and q.is_contiguous() and tuple(q.shape) == self.shape
        B.fp_rk3_step(self.ctx, q.data_ptr(), dt, _stream())
        return q

    def cfl_dt(self, q: torch.Tensor, cfl: float) -> float:
        return B.fp_cfl_dt(self.ctx, q.data_ptr(), cfl, _stream())

    def metrics(self) -> np.ndarray:
        ni, nj, nk = self.n
        G = self.G
        shp = (10, 1, nj + 2 * G, ni + 2 * G) if self.dims == 2 else (10, nk + 2 * G, nj + 2 * G, ni + 2 * G)
        out = np.zeros(shp)
        B.fp_get_metrics(self.ctx, out.ctypes.data)
        return out

    def face_metrics(self, d: int) -> np.ndarray:
        ni, nj, nk = self.n
        nf = [ni, nj, nk]
        nf[d] += 1
        out = np.zeros((3, nf[2], nf[1], nf[0]))
        B.fp_get_face_metrics(self.ctx, d, out.ctypes.data)
        return out

    def status(self) -> int:
        return B.fp_get_device_status(self.ctx, _stream())

    def close(self):
        if self.ctx:
            B.fp_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many blocks advanced together by one CUDA-graph replay per RK step."""

    def __init__(self, blocks, states, autotune=True, links=()):
        """links: (a, dir, side, b) tuples for the FP_BC_BLOCK sides (fp_batch_create_linked)."""
        self.blocks = list(blocks)
        self.states = list(states)
        self.batch = B.fp_batch_create_linked([b.ctx for b in self.blocks], [q.data_ptr() for q in self.states],
                                              links, int(autotune), _stream())

    def rk3_step(self, dt: float):
        B.fp_batch_rk3_step(self.batch, dt, _stream())

    def rhs(self, outs):
        B.fp_batch_rhs(self.batch, [o.data_ptr() for o in outs], _stream())
        return outs

    def launches_per_step(self):
        return B.fp_batch_launches_per_step(self.batch)

    def close(self):
        if self.batch:
            B.fp_batch_free(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipe:
    """Blocks whose states live in host memory (page-locked CPU tensors), advanced with
    the host<->device copies overlapped by compute (fp_pipe_*): the blocks are split into
    `groups` batches with a stream each.  Steps run on the pipe's own streams, so the blocks
    must not be used by other calls while a step may be in flight (synchronise first), unless
    `ordered` makes every step follow the work queued before it on the current stream."""

    def __init__(self, blocks, host_states, groups=4, autotune=True, ordered=False):
        self.blocks = list(blocks)
        self.host = list(host_states)
        for b, h in zip(self.blocks, self.host):
            assert h.device.type == "cpu" and h.is_contiguous() and tuple(h.shape) == b.shape and h.dtype == b.dtype
        self.pipe = B.fp_pipe_create([b.ctx for b in self.blocks], [h.data_ptr() for h in self.host],
                                     groups, int(autotune))
        if ordered:
            B.fp_pipe_set_ordered(self.pipe, 1)

    def rk3_step(self, dt: float):
        B.fp_pipe_rk3_step_host(self.pipe, [h.data_ptr() for h in self.host], dt, _stream())

    def launches_per_step(self):
        return B.fp_pipe_launches_per_step(self.pipe)

    def close(self):
        if self.pipe:
            B.fp_pipe_free(self.pipe)
            self.pipe = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
