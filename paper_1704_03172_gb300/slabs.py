"""Row-slab domain decomposition of one shot (one process with several slabs, or one slab
per rank under torch.distributed).

One LB step reads only nearest neighbours (the streaming of Eq. BGK-LB moves populations
one cell), so a grid split into horizontal slabs needs, per step and per cut, only the
populations that cross the cut: D2Q5 g2 up and g4 down, D2Q9 three each way.  The library
(``lb_set_slab``) pulls those from halo rows at the cuts and writes its own cut rows into
send buffers in the same launch; this module only splits the grid, routes the source and
the receivers to the slab that holds them, moves send buffers into the neighbours' halo
rows, and assembles traces, pressure and state.  It holds none of the method's arithmetic.

- ``partition`` / ``owner`` / ``route_receivers``: the host-side bookkeeping;
- ``SlabGrid``: n slabs in this process (``lb_slab_step`` steps them and copies the rows);
- ``exchange`` / ``DistSlab``: one slab per rank; the rows move with torch.distributed
  point-to-point operations (NCCL between GPUs; gloo on CPU tensors in the tests);
- ``allreduce_gradient``: the sum over ranks of per-shot gradients (several shots, one
  model: the c-gradient of a multi-shot misfit is the sum of the shots' gradients).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lbac


def partition(ny, n):
    """Row ranges [(y0, y1), ...] of n slabs tiling ny rows, as equal as possible
    (the first ny % n slabs get one row more)."""
    if n < 1 or ny < n:
        raise ValueError(f"cannot split {ny} rows into {n} slabs")
    q, r = divmod(ny, n)
    out, y = [], 0
    for k in range(n):
        h = q + (1 if k < r else 0)
        out.append((y, y + h))
        y += h
    return out


def owner(y, bounds):
    """Index of the slab whose rows hold row y."""
    for k, (y0, y1) in enumerate(bounds):
        if y0 <= y < y1:
            return k
    raise ValueError(f"row {y} outside the grid")


def route_receivers(rec, bounds):
    """Per slab: (indices into rec, local (x, y) pairs) of the receivers it holds."""
    rec = np.asarray(rec, dtype=np.int32).reshape(-1, 2)
    out = []
    for y0, y1 in bounds:
        idx = np.nonzero((rec[:, 1] >= y0) & (rec[:, 1] < y1))[0]
        loc = rec[idx].copy()
        loc[:, 1] -= y0
        out.append((idx, loc))
    return out


def assemble_traces(parts, routes, nrec, nt):
    """Global [nt][nrec] traces from per-slab [nt][n_k] traces."""
    out = np.zeros((nt, nrec), dtype=np.float32)
    for tr, (idx, _) in zip(parts, routes):
        if len(idx):
            out[:, idx] = tr[:nt]
    return out


def _halo_tensors(sim, nbytes):
    """four zeroed row buffers on the slab's device, ready before its stream uses them"""
    import torch
    n = nbytes // 4
    bufs = [torch.zeros(n, dtype=torch.float32, device=sim.device) for _ in range(4)]
    sim.stream.wait_stream(torch.cuda.current_stream(sim.device))
    return bufs


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class SlabGrid:
    """One shot split into row slabs held by this process (on one or several devices).

    Every slab is an LBSim of its own rows, marked with lb_set_slab; ``step`` calls
    lb_slab_step, which steps every slab and fills the halo rows from the neighbours.
    The results equal those of the whole grid run as one context."""

    def __init__(self, c_map, n_slabs, *, devices=None, **kw):
        import torch
        from .sim import LBSim
        c_map = np.ascontiguousarray(c_map, dtype=np.float32)
        self.ny, self.nx = c_map.shape
        self.bounds = partition(self.ny, n_slabs)
        periodic = kw.get("boundary", "zero") == "periodic"
        if kw.get("c_ref") is None:
            kw["c_ref"] = float(c_map.max())  # one eta for all slabs
        devices = devices or [torch.cuda.current_device()] * n_slabs
        self.sims, self.bufs = [], []
        for k, (y0, y1) in enumerate(self.bounds):
            self.sims.append(LBSim(c_map[y0:y1], device=devices[k], **kw))
        nbytes = lbac.lb_slab_halo_bytes(self.sims[0].ctx)
        for k, sim in enumerate(self.sims):
            send_lo, send_hi, recv_lo, recv_hi = _halo_tensors(sim, nbytes)
            has_lo = k > 0 or periodic
            has_hi = k + 1 < n_slabs or periodic
            self.bufs.append((send_lo, send_hi, recv_lo, recv_hi))
            lbac.lb_set_slab(sim.ctx, self.bounds[k][0], self.ny, _ptr(send_lo), _ptr(send_hi),
                             _ptr(recv_lo) if has_lo else None, _ptr(recv_hi) if has_hi else None)
        self.routes = None
        self.nrec = 0

    def set_source(self, x, y, wavelet):
        k = owner(y, self.bounds)
        self.sims[k].set_source(x, y - self.bounds[k][0], wavelet)

    def set_receivers(self, rec, nt_capacity):
        self.routes = route_receivers(rec, self.bounds)
        self.nrec = len(np.asarray(rec).reshape(-1, 2))
        for sim, (idx, loc) in zip(self.sims, self.routes):
            sim.set_receivers(loc, nt_capacity)

    def init_pressure(self, p0=None):
        for sim, (y0, y1) in zip(self.sims, self.bounds):
            sim.init_pressure(None if p0 is None else np.ascontiguousarray(p0[y0:y1]))

    def set_state(self, g):
        g = np.asarray(g, dtype=np.float32)
        for sim, (y0, y1) in zip(self.sims, self.bounds):
            sim.set_state(np.ascontiguousarray(g[:, y0:y1]))

    def step(self, n=1):
        lbac.lb_slab_step([s.ctx for s in self.sims], n)

    def sync(self):
        for s in self.sims:
            s.sync()

    def pressure(self):
        return np.concatenate([s.pressure().cpu().numpy() for s in self.sims], axis=0)

    def state(self):
        return np.concatenate([s.state().cpu().numpy() for s in self.sims], axis=1)

    def traces(self, nt):
        parts = [s.traces(nt).cpu().numpy() if len(idx) else None
                 for s, (idx, _) in zip(self.sims, self.routes)]
        return assemble_traces(parts, self.routes, self.nrec, nt)

    def close(self):
        for s in self.sims:
            s.close()
        self.sims = []


# ---------------------------------------------------------------------- one slab per rank --

def neighbours(rank, world, periodic):
    """(rank below, rank above), None where the grid ends."""
    lo = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    hi = rank + 1 if rank + 1 < world else (0 if periodic else None)
    return lo, hi


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic, group=None):
    """Move this rank's cut rows to its neighbours and theirs into its halo rows:
    send_hi -> the rank above's recv_lo, send_lo -> the rank below's recv_hi.  Works on
    CUDA tensors (NCCL, on the current stream) and CPU tensors (gloo).  Every rank posts
    its upward messages first, then its downward ones, so that two ranks that are each
    other's neighbour on both sides (two slabs of a periodic grid) match in order."""
    import torch.distributed as dist
    lo, hi = neighbours(rank, world, periodic)
    if world == 1:  # one slab: its own cut rows are its halo rows (periodic) or nothing
        if periodic:
            recv_lo.copy_(send_hi)
            recv_hi.copy_(send_lo)
        return
    ops = []
    if hi is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, hi, group, tag=1))
    if lo is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, lo, group, tag=1))
    if lo is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, lo, group, tag=2))
    if hi is not None:
        ops.append(dist.P2POp(dist.irecv, recv_hi, hi, group, tag=2))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()


def allreduce_gradient(grad, group=None):
    """Sum a per-rank gradient (e.g. dJ/dc of the shots this rank ran) over all ranks."""
    import torch.distributed as dist
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad


class DistSlab:
    """This rank's slab of one shot: rows partition(ny, world)[rank] of the grid, stepped
    by the library, the cut rows moved by ``exchange`` after every step."""

    def __init__(self, c_map, rank, world, **kw):
        import torch
        from .sim import LBSim
        c_map = np.ascontiguousarray(c_map, dtype=np.float32)
        self.ny, self.nx = c_map.shape
        self.rank, self.world = rank, world
        self.bounds = partition(self.ny, world)
        self.y0, self.y1 = self.bounds[rank]
        self.periodic = kw.get("boundary", "zero") == "periodic"
        if kw.get("c_ref") is None:
            kw["c_ref"] = float(c_map.max())
        self.sim = LBSim(c_map[self.y0:self.y1], **kw)
        nbytes = lbac.lb_slab_halo_bytes(self.sim.ctx)
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = _halo_tensors(self.sim, nbytes)
        lo, hi = neighbours(rank, world, self.periodic)
        lbac.lb_set_slab(self.sim.ctx, self.y0, self.ny, _ptr(self.send_lo), _ptr(self.send_hi),
                         _ptr(self.recv_lo) if lo is not None else None,
                         _ptr(self.recv_hi) if hi is not None else None)
        self.routes = None
        self.nrec = 0
        self._torch = torch

    def set_source(self, x, y, wavelet):
        if self.y0 <= y < self.y1:
            self.sim.set_source(x, y - self.y0, wavelet)

    def set_receivers(self, rec, nt_capacity):
        self.routes = route_receivers(rec, self.bounds)
        self.nrec = len(np.asarray(rec).reshape(-1, 2))
        self.sim.set_receivers(self.routes[self.rank][1], nt_capacity)

    def init_pressure(self, p0=None):
        self.sim.init_pressure(None if p0 is None else np.ascontiguousarray(p0[self.y0:self.y1]))

    def step(self, n=1):
        torch = self._torch
        for _ in range(n):
            lbac.lb_step(self.sim.ctx, 1)
            with torch.cuda.stream(self.sim.stream):  # the exchange follows the step
                exchange(self.send_lo, self.send_hi, self.recv_lo, self.recv_hi, self.rank,
                         self.world, self.periodic)

    def traces(self, nt):
        """Global [nt][nrec] traces on rank 0 (None elsewhere): every rank's rows gathered."""
        import torch.distributed as dist
        idx, _ = self.routes[self.rank]
        mine = (self.sim.traces(nt).cpu().numpy() if len(idx)
                else np.zeros((nt, 0), np.float32))
        if self.world == 1:
            return assemble_traces([mine], self.routes, self.nrec, nt)
        parts = [None] * self.world
        dist.gather_object(mine, parts if self.rank == 0 else None, dst=0)
        if self.rank != 0:
            return None
        return assemble_traces(parts, self.routes, self.nrec, nt)

    def close(self):
        self.sim.close()
