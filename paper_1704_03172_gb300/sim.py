"""PyTorch-facing wrapper of the C ABI: device memory, streams, tensors in and out.

``LBSim`` owns one ``lb_ctx``.  PyTorch supplies the CUDA stream the library
runs on and (by default) its caching allocator for every device buffer the
library allocates; all computation happens in the CUDA kernels of
``liblbac.so``.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import lbac

_STORAGE = {"f32": lbac.LB_F32, "bf16": lbac.LB_BF16, "f16": lbac.LB_F16,
            "f64": lbac.LB_F64}  # f64: test only (FP64 state, plain step kernel)
_COLL = {"bgk": lbac.LB_BGK, "mrt": lbac.LB_MRT}
_BOUND = {"zero": lbac.LB_ZERO_GHOST, "periodic": lbac.LB_PERIODIC}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


_COUPLING = {"both": lbac.LB_COUPLE_BOTH, "c2f": lbac.LB_COUPLE_C2F, "f2c": lbac.LB_COUPLE_F2C}


def patch_array(patch, coupling="both"):
    """The lb_patch array of one patch (x0, y0, nx_c, ny_c[, ratio]) or of a list of nested
    patches, each in the node coordinates of the fine grid of the one before it.  coupling:
    "both", "c2f" or "f2c", one value for all patches or one per patch."""
    plist = list(patch) if len(patch) and hasattr(patch[0], "__len__") else [patch]
    modes = [coupling] * len(plist) if isinstance(coupling, str) else list(coupling)
    if len(modes) != len(plist):
        raise ValueError(f"coupling: {len(modes)} values for {len(plist)} patches")
    if any(m not in _COUPLING for m in modes):
        raise ValueError(f"coupling must be 'both', 'c2f' or 'f2c', not {modes}")
    return (lbac.lb_patch * len(plist))(
        *[lbac.lb_patch(*[int(v) for v in q[:4]], int(q[4]) if len(q) > 4 else 2, _COUPLING[m])
          for q, m in zip(plist, modes)])


class LBSim:
    """One linear-LB acoustic simulation ("shot") on the current CUDA device."""

    def __init__(self, c_map, *, lattice=5, collision="bgk", tau=0.5, s=None, storage="f32",
                 boundary="zero", sponge_width=0, sponge_sigma_max=0.1, c_ref=None,
                 w_ref=(4 / 9, 1 / 9, 1 / 36), patch=None, coupling="both", dx=0.0, time_block=1,
                 step_kernel="auto", streaming="ab", device=None, stream=None,
                 torch_allocator=True):
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        # A dedicated stream: the legacy default stream's handle is 0, which the C ABI
        # reads as "create a private stream", so the default stream is never passed.
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        if self.stream.cuda_stream == 0:
            raise ValueError("pass a non-default torch.cuda.Stream")
        cfg = lbac.lb_config_default()
        cfg.lattice = int(lattice)
        cfg.collision = _COLL[collision] if isinstance(collision, str) else int(collision)
        cfg.storage = _STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.f64 = cfg.storage == lbac.LB_F64
        cfg.boundary = _BOUND[boundary] if isinstance(boundary, str) else int(boundary)
        if not torch.is_tensor(c_map):
            c_map = np.ascontiguousarray(c_map, dtype=np.float32)
        # [ny][nx], or [nz][ny][nx] for the 3-D lattice (D3Q7)
        nz, ny, nx = (1,) + tuple(c_map.shape) if len(c_map.shape) == 2 else tuple(c_map.shape)
        self.nx, self.ny, self.nz, self.Q = int(nx), int(ny), int(nz), int(lattice)
        cfg.nx, cfg.ny, cfg.nz = self.nx, self.ny, self.nz
        self._grid = (self.ny, self.nx) if len(c_map.shape) == 2 else (self.nz, self.ny, self.nx)
        cfg.sponge_width = int(sponge_width)
        cfg.sponge_sigma_max = float(sponge_sigma_max)
        cfg.tau = float(tau)
        if s is not None:
            for k, v in enumerate(s):
                cfg.s[k] = float(v)
        for k in range(3):
            cfg.w_ref[k] = float(w_ref[k])
        cfg.dx = float(dx)
        cfg.time_block = int(time_block)
        cfg.step_kernel = {"auto": lbac.LB_STEP_AUTO, "direct": lbac.LB_STEP_DIRECT,
                           "staged": lbac.LB_STEP_STAGED}[step_kernel]
        # "ab": pull from one population buffer into the other; "aa": in place, one buffer
        cfg.streaming = {"ab": lbac.LB_STREAM_AB, "aa": lbac.LB_STREAM_AA}[streaming]
        cfg.c_ref = float(c_ref) if c_ref is not None else 0.0
        if torch.is_tensor(c_map) and c_map.is_cuda:
            self._cmap_keep = c_map.to(torch.float32).contiguous()
            cfg.c_map = ctypes.cast(ctypes.c_void_p(self._cmap_keep.data_ptr()),
                                    ctypes.POINTER(ctypes.c_float))
            cfg.c_map_on_device = 1
            if c_ref is None:
                cfg.c_ref = float(self._cmap_keep.max())
        else:
            host = np.ascontiguousarray(c_map.cpu().numpy() if torch.is_tensor(c_map) else c_map,
                                        dtype=np.float32)
            self._cmap_keep = host
            cfg.c_map = host.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        if patch is not None:
            self._patch = patch_array(patch, coupling)
            cfg.patches = ctypes.cast(self._patch, ctypes.POINTER(lbac.lb_patch))
            cfg.n_patches = len(self._patch)
        cfg.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        if torch_allocator:
            dev, strm = self.device, self.stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=strm)
                except Exception:
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = lbac.ALLOC_FN(_alloc)
            self._free_cb = lbac.FREE_FN(_free)
            cfg.dev_alloc = self._alloc_cb
            cfg.dev_free = self._free_cb
        self.cfg = cfg
        with torch.cuda.device(self.device):
            self.ctx = lbac.lb_create(cfg)
        self.nrec = 0

    # -- inputs -----------------------------------------------------------------------
    def set_source(self, *args):
        """set_source(x, y, wavelet), or set_source(x, y, z, wavelet) on a 3-D grid."""
        *xyz, wavelet = args
        w = np.ascontiguousarray(np.asarray(wavelet, dtype=np.float64))
        wp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if len(xyz) == 3:
            lbac.lb_set_source_3d(self.ctx, *xyz, wp, len(w))
        else:
            lbac.lb_set_source(self.ctx, *xyz, wp, len(w))

    def set_receivers(self, xy, nt_capacity):
        """Receivers [n][2] = (x, y), or [n][3] = (x, y, z) on a 3-D grid."""
        d = 3 if len(self._grid) == 3 else 2
        xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, d))
        fn = lbac.lb_set_receivers_3d if d == 3 else lbac.lb_set_receivers
        fn(self.ctx, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(xy), nt_capacity)
        self.nrec = len(xy)

    def init_pressure(self, p0=None):
        if p0 is None:
            lbac.lb_init_pressure(self.ctx, None, 0)
            return
        t = torch.as_tensor(p0, dtype=torch.float32, device=self.device).contiguous()
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        lbac.lb_init_pressure(self.ctx, _ptr(t), 1)
        self.stream.synchronize()

    def set_state(self, g):
        """Populations [Q][ny][nx]; FP64 contexts take them in FP64."""
        dt = torch.float64 if self.f64 else torch.float32
        t = torch.as_tensor(g, dtype=dt, device=self.device).contiguous()
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        (lbac.lb_set_state_f64 if self.f64 else lbac.lb_set_state)(self.ctx, _ptr(t), 1)
        self.stream.synchronize()

    # -- stepping -----------------------------------------------------------------------
    def step(self, n=1):
        lbac.lb_step(self.ctx, n)

    def sync(self):
        lbac.lb_sync(self.ctx)

    @property
    def time(self):
        return lbac.lb_get_time(self.ctx)

    # -- outputs ------------------------------------------------------------------------
    def _out(self, shape, dtype=torch.float32):
        with torch.cuda.stream(self.stream):
            return torch.zeros(shape, dtype=dtype, device=self.device)

    def traces(self, nt_max=None):
        """Receiver traces [rows, nrec] (row n = pressure at time n); synchronises."""
        nt_max = self.time if nt_max is None else nt_max
        out = self._out((max(nt_max, 0), max(self.nrec, 1)))
        n = lbac.lb_record_receivers(self.ctx, _ptr(out), nt_max, 1)
        return out[:n, :self.nrec]

    def pressure(self):
        """p = c_s^2 sum_i g_i at the current time (FP64 for an FP64 context)."""
        if self.f64:
            out = self._out(self._grid, torch.float64)
            lbac.lb_get_pressure_f64(self.ctx, _ptr(out), 1)
            return out
        out = self._out(self._grid)
        lbac.lb_get_pressure(self.ctx, _ptr(out), 1)
        return out

    def state(self):
        """Populations g_i(x) [Q][ny][nx] at the current time (FP64 for an FP64 context)."""
        if self.f64:
            out = self._out((self.Q,) + self._grid, torch.float64)
            lbac.lb_get_state_f64(self.ctx, _ptr(out), 1)
            return out
        out = self._out((self.Q,) + self._grid)
        lbac.lb_get_state(self.ctx, _ptr(out), 1)
        return out

    def checkpoint_every(self, every):
        """Keep adjoint checkpoints every `every` steps from the current time."""
        lbac.lb_checkpoint_every(self.ctx, every)

    def record_rho(self, nt):
        """Record the forward density tape for the next `nt` steps (no checkpoints or replays
        needed by adjoint(); nt * ny * pitch * 4 bytes of device memory; 0 frees it)."""
        lbac.lb_record_rho(self.ctx, nt)

    def adjoint(self, dJdp, nt=None, want_g0=False):
        """Gradients of J given dJ/dp at the receivers (trace rows): returns
        (dJ/dc_map [ny, nx] float32, dJ/dS [nt] float64, dJ/dg(t0) or None)."""
        dJdp = torch.as_tensor(dJdp, dtype=torch.float32, device=self.device).contiguous()
        nt = dJdp.shape[0] if nt is None else int(nt)
        with torch.cuda.stream(self.stream):
            gc = torch.zeros((self.ny, self.nx), dtype=torch.float32, device=self.device)
            gs = torch.zeros(nt, dtype=torch.float64, device=self.device)
            gg = (torch.zeros((self.Q, self.ny, self.nx), dtype=torch.float32, device=self.device)
                  if want_g0 else None)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        lbac.lb_adjoint(self.ctx, _ptr(dJdp), nt, _ptr(gc), _ptr(gs),
                        _ptr(gg) if gg is not None else None, 1)
        return gc, gs, gg

    def invariants(self):
        """(mass, energy, max |g|, non-finite count) of the current state, FP64."""
        return lbac.lb_invariants(self.ctx)

    def info(self):
        return lbac.lb_info(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            lbac.lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class LBForward(torch.autograd.Function):
    """traces = LB(c_map, wavelet): receiver traces of one shot, differentiable with
    respect to the sound-speed map and the source samples through the library's
    discrete adjoint (lb_adjoint) rather than autograd tracing.

    forward(c_map [ny, nx], wavelet [nt], spec) -> traces [nt, nrec], where spec is a
    dict of LBSim keyword arguments plus "source_xy", "receivers", "nt" and
    "checkpoint_every" (> 0: checkpoints; < 0: the forward rho tape; 0 or absent: the tape
    when it takes at most 40 % of the free device memory, as the server decides, else
    checkpoints every 200 steps).  c_ref must be given: it is held fixed under
    differentiation.
    """

    @staticmethod
    def forward(ctx, c_map, wavelet, spec):
        spec = dict(spec)
        nt = int(spec.pop("nt"))
        sxy = spec.pop("source_xy")
        rec = spec.pop("receivers")
        every = int(spec.pop("checkpoint_every", 0))
        if spec.get("c_ref") is None:
            raise ValueError("spec['c_ref'] must be fixed for differentiation")
        sim = LBSim(c_map.detach(), **spec)
        sim.set_source(sxy[0], sxy[1], wavelet.detach().double().cpu().numpy())
        sim.set_receivers(rec, nt)
        sim.init_pressure(None)
        if every == 0:
            tape_bytes = nt * sim.ny * (-(-sim.nx // 32) * 32) * 4
            every = -1 if tape_bytes <= 0.4 * torch.cuda.mem_get_info(sim.device)[0] else 200
        if every < 0:
            sim.record_rho(nt)
        else:
            sim.checkpoint_every(every)
        sim.step(nt)
        traces = sim.traces(nt).clone()
        ctx.sim, ctx.nt = sim, nt
        ctx.wdtype, ctx.wdevice = wavelet.dtype, wavelet.device
        return traces

    @staticmethod
    def backward(ctx, grad_traces):
        gc, gs, _ = ctx.sim.adjoint(grad_traces, ctx.nt)
        ctx.sim.close()
        return gc, gs.to(dtype=ctx.wdtype, device=ctx.wdevice), None


class LBServer:
    """Continuous-batching shot server (lb_server_* of the C ABI).  tb_min_ctas: 0 (default)
    lets the eligible D2Q5 shots take 4 steps per launch when together they fill a wave of
    the GPU with chunks of at least 12 rows; > 0 when they make that many CTAs at 64 rows;
    < 0 never."""

    def __init__(self, max_active=64, hbm_budget=0, rounds_per_pass=16, adjoint_workers=2,
                 tb_min_ctas=0):
        cfg = lbac.lb_server_config(int(max_active), int(hbm_budget), int(rounds_per_pass),
                                    int(adjoint_workers), int(tb_min_ctas))
        self.srv = lbac.lb_server_create(cfg)
        self._meta = {}

    def submit(self, c_map, *, nt, source, receivers, observed=None, want_gradient=False,
               checkpoint_every=0, lattice=5, collision="bgk", tau=0.5, s=None,
               storage="f32", boundary="zero", sponge_width=0, sponge_sigma_max=0.1, c_ref=None,
               w_ref=(4 / 9, 1 / 9, 1 / 36)):
        c = np.ascontiguousarray(c_map, dtype=np.float32)
        ny, nx = c.shape
        cfg = lbac.lb_config_default()
        cfg.lattice, cfg.nx, cfg.ny = int(lattice), nx, ny
        cfg.collision = _COLL[collision] if isinstance(collision, str) else int(collision)
        cfg.storage = _STORAGE[storage] if isinstance(storage, str) else int(storage)
        cfg.boundary = _BOUND[boundary] if isinstance(boundary, str) else int(boundary)
        cfg.tau = float(tau)
        if s is not None:
            for k, v in enumerate(s):
                cfg.s[k] = float(v)
        for k in range(3):
            cfg.w_ref[k] = float(w_ref[k])
        cfg.sponge_width, cfg.sponge_sigma_max = int(sponge_width), float(sponge_sigma_max)
        cfg.c_ref = float(c_ref) if c_ref is not None else 0.0
        cfg.c_map = c.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        sx, sy, wav = source
        wav = np.ascontiguousarray(wav, dtype=np.float64)
        rec = np.ascontiguousarray(np.asarray(receivers, dtype=np.int32).reshape(-1, 2))
        req = lbac.lb_request()
        req.cfg = cfg
        req.src_x, req.src_y = int(sx), int(sy)
        req.wavelet = wav.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        req.nt_wavelet = len(wav)
        req.rec_xy = rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        req.nrec = len(rec)
        req.nt = int(nt)
        obs = None
        if want_gradient:
            obs = np.ascontiguousarray(observed, dtype=np.float32).reshape(int(nt), len(rec))
            req.observed = obs.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        req.want_gradient = int(bool(want_gradient))
        req.checkpoint_every = int(checkpoint_every)
        rid = lbac.lb_server_submit(self.srv, req)   # copies every array
        self._meta[rid] = (int(nt), len(rec), nx, ny, len(wav), bool(want_gradient))
        return rid

    def poll(self, rid):
        return lbac.lb_server_poll(self.srv, rid)

    def wait(self, rid, timeout_ms=-1):
        lbac.lb_server_wait(self.srv, rid, timeout_ms)

    def result(self, rid):
        nt, nrec, nx, ny, nw, grad = self._meta.pop(rid)
        tr = np.zeros((nt, max(nrec, 1)), np.float32)
        gc = np.zeros((ny, nx), np.float32) if grad else None
        gs = np.zeros(max(nw, 1), np.float64) if grad else None
        st, times = lbac.lb_server_result(
            self.srv, rid, ctypes.c_void_p(tr.ctypes.data),
            ctypes.c_void_p(gc.ctypes.data) if grad else None,
            ctypes.c_void_p(gs.ctypes.data) if grad else None)
        if st != lbac.LB_OK:
            raise lbac.LBError(st, lbac.lb_server_last_error(self.srv))
        return {"traces": tr[:, :nrec], "grad_c": gc, "grad_src": gs[:nw] if grad else None,
                "submit": times[0], "start": times[1], "done": times[2]}

    def stats(self):
        v = lbac.lb_server_stats(self.srv)
        return {"done": v[0], "active": v[1], "pending": v[2], "bytes": v[3], "launches": v[4]}

    def close(self):
        if getattr(self, "srv", None):
            lbac.lb_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
