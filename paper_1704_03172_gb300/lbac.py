"""ctypes binding of the C ABI in ``include/lbac.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own.  Importing this module loads ``liblbac.so`` from the
package directory and raises ``ImportError`` if it is missing: there is no
CPU fallback.  Build it with ``paper_1704_03172_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbac.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")
_lib = ctypes.CDLL(LIB_PATH)

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EUNSTABLE, LB_ETIMEOUT, LB_ESTATE = 0, -1, -2, -3, -4, -5, -6
LB_D2Q5, LB_D2Q9, LB_D3Q7 = 5, 9, 7
LB_BGK, LB_MRT = 0, 1
LB_F32, LB_BF16, LB_F16, LB_F64 = 0, 1, 2, 3
LB_STEP_AUTO, LB_STEP_DIRECT, LB_STEP_STAGED = 0, 1, 2
LB_STREAM_AB, LB_STREAM_AA = 0, 1
LB_ZERO_GHOST, LB_PERIODIC = 0, 1
STATUS_NAMES = {0: "LB_OK", -1: "LB_EINVAL", -2: "LB_ENOMEM", -3: "LB_ECUDA",
                -4: "LB_EUNSTABLE", -5: "LB_ETIMEOUT", -6: "LB_ESTATE"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lb_patch(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int), ("y0", ctypes.c_int), ("nx_c", ctypes.c_int),
                ("ny_c", ctypes.c_int), ("ratio", ctypes.c_int), ("coupling", ctypes.c_int)]


LB_COUPLE_BOTH, LB_COUPLE_C2F, LB_COUPLE_F2C = 0, 1, 2


class lb_config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("collision", ctypes.c_int), ("storage", ctypes.c_int),
        ("boundary", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("sponge_width", ctypes.c_int), ("sponge_sigma_max", ctypes.c_double),
        ("c_map", ctypes.POINTER(ctypes.c_float)), ("c_map_on_device", ctypes.c_int),
        ("c_ref", ctypes.c_double), ("dx", ctypes.c_double), ("tau", ctypes.c_double),
        ("s", ctypes.c_double * 9), ("w_ref", ctypes.c_double * 3),
        ("patches", ctypes.POINTER(lb_patch)), ("n_patches", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p), ("time_block", ctypes.c_int),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_user", ctypes.c_void_p),
        ("step_kernel", ctypes.c_int), ("nz", ctypes.c_int), ("streaming", ctypes.c_int),
    ]


class lb_server_config(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("hbm_budget", ctypes.c_size_t),
                ("rounds_per_pass", ctypes.c_int), ("adjoint_workers", ctypes.c_int),
                ("tb_min_ctas", ctypes.c_int)]


class lb_request(ctypes.Structure):
    _fields_ = [
        ("cfg", lb_config), ("src_x", ctypes.c_int), ("src_y", ctypes.c_int),
        ("wavelet", ctypes.POINTER(ctypes.c_double)), ("nt_wavelet", ctypes.c_int),
        ("rec_xy", ctypes.POINTER(ctypes.c_int)), ("nrec", ctypes.c_int), ("nt", ctypes.c_int),
        ("observed", ctypes.POINTER(ctypes.c_float)), ("want_gradient", ctypes.c_int),
        ("checkpoint_every", ctypes.c_int),
    ]


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_ctx_p = ctypes.c_void_p
_fp = ctypes.POINTER(ctypes.c_float)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_cfgp = ctypes.POINTER(lb_config)

_SIGS = {
    "lb_config_default": [_cfgp],
    "lb_create": [_cfgp, ctypes.POINTER(_ctx_p)],
    "lb_destroy": [_ctx_p],
    "lb_set_source": [_ctx_p, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int],
    "lb_set_receivers": [_ctx_p, _ip, ctypes.c_int, ctypes.c_int],
    "lb_set_source_3d": [_ctx_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int],
    "lb_set_receivers_3d": [_ctx_p, _ip, ctypes.c_int, ctypes.c_int],
    "lb_init_pressure": [_ctx_p, ctypes.c_void_p, ctypes.c_int],
    "lb_step": [_ctx_p, ctypes.c_int],
    "lb_record_receivers": [_ctx_p, ctypes.c_void_p, ctypes.c_int, _ip, ctypes.c_int],
    "lb_get_pressure": [_ctx_p, ctypes.c_void_p, ctypes.c_int],
    "lb_get_state": [_ctx_p, ctypes.c_void_p, ctypes.c_int],
    "lb_set_state": [_ctx_p, ctypes.c_void_p, ctypes.c_int],
    "lb_get_state_f64": [_ctx_p, ctypes.c_void_p, ctypes.c_int],
    "lb_set_state_f64": [_ctx_p, ctypes.c_void_p, ctypes.c_int],
    "lb_get_pressure_f64": [_ctx_p, ctypes.c_void_p, ctypes.c_int],
    "lb_get_time": [_ctx_p, ctypes.POINTER(ctypes.c_longlong)],
    "lb_sync": [_ctx_p],
    "lb_wait_selftest": [_ctx_p, ctypes.c_int],
    "lb_record_rho": [_ctx_p, ctypes.c_int],
    "lb_footprint": [_cfgp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                     ctypes.POINTER(ctypes.c_size_t)],
    "lb_info": [_ctx_p, _dp, ctypes.c_int],
    "lb_invariants": [_ctx_p, _dp],
    "lb_mode_projection": [_ctx_p, _ip, ctypes.c_int, _dp],
    "lb_invariants_noalloc": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_double, _dp, ctypes.c_void_p,
                              ctypes.c_void_p],
    "lb_stability_radius": [_cfgp, ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp],
    "lb_watch_stability": [_ctx_p, ctypes.c_int, ctypes.c_double],
    "lb_set_slab": [_ctx_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                    ctypes.c_void_p, ctypes.c_void_p],
    "lb_slab_halo_bytes": [_ctx_p, ctypes.POINTER(ctypes.c_size_t)],
    "lb_slab_step": [ctypes.POINTER(_ctx_p), ctypes.c_int, ctypes.c_int],
}
_srv_p = ctypes.c_void_p
_SIGS.update({
    "lb_server_create": [ctypes.POINTER(lb_server_config), ctypes.POINTER(_srv_p)],
    "lb_server_submit": [_srv_p, ctypes.POINTER(lb_request), ctypes.POINTER(ctypes.c_longlong)],
    "lb_server_poll": [_srv_p, ctypes.c_longlong, _ip],
    "lb_server_wait": [_srv_p, ctypes.c_longlong, ctypes.c_int],
    "lb_server_result": [_srv_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p, _dp],
    "lb_server_stats": [_srv_p, _dp, ctypes.c_int],
    "lb_server_destroy": [_srv_p],
    "lb_checkpoint_every": [_ctx_p, ctypes.c_int],
    "lb_adjoint": [_ctx_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int],
})
OPTIONAL = {}

for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
for _name, _args in OPTIONAL.items():
    if hasattr(_lib, _name):
        _f = getattr(_lib, _name)
        _f.argtypes = _args
        _f.restype = ctypes.c_int
_lib.lb_last_error.argtypes = [_ctx_p]
_lib.lb_last_error.restype = ctypes.c_char_p
_lib.lb_server_last_error.argtypes = [_srv_p]
_lib.lb_server_last_error.restype = ctypes.c_char_p

EXPORTED = sorted(list(_SIGS) + ["lb_last_error", "lb_server_last_error"] +
                  [n for n in OPTIONAL if hasattr(_lib, n)])


def lb_server_create(cfg: lb_server_config):
    srv = _srv_p()
    _check(_lib.lb_server_create(ctypes.byref(cfg), ctypes.byref(srv)))
    return srv


def lb_server_submit(srv, req: lb_request) -> int:
    rid = ctypes.c_longlong()
    _check(_lib.lb_server_submit(srv, ctypes.byref(req), ctypes.byref(rid)))
    return rid.value


def lb_server_poll(srv, rid) -> bool:
    d = ctypes.c_int()
    _check(_lib.lb_server_poll(srv, int(rid), ctypes.byref(d)))
    return bool(d.value)


def lb_server_wait(srv, rid, timeout_ms=-1):
    return _check(_lib.lb_server_wait(srv, int(rid), int(timeout_ms)))


def lb_server_result(srv, rid, traces_ptr, grad_c_ptr, grad_src_ptr):
    """Returns (status, times[3]); the caller checks status (the request's own)."""
    t = (ctypes.c_double * 3)()
    st = _lib.lb_server_result(srv, int(rid), traces_ptr, grad_c_ptr, grad_src_ptr, t)
    return st, list(t)


def lb_server_stats(srv):
    v = (ctypes.c_double * 5)()
    _check(_lib.lb_server_stats(srv, v, 5))
    return list(v)


def lb_server_destroy(srv):
    return _check(_lib.lb_server_destroy(srv))


def lb_server_last_error(srv) -> str:
    m = _lib.lb_server_last_error(srv)
    return m.decode() if m else ""


def lb_last_error(ctx=None) -> str:
    m = _lib.lb_last_error(ctx)
    return m.decode() if m else ""


def _check(status, ctx=None):
    if status != LB_OK:
        raise LBError(status, lb_last_error(ctx))
    return status


def lb_config_default() -> lb_config:
    cfg = lb_config()
    _check(_lib.lb_config_default(ctypes.byref(cfg)))
    return cfg


def lb_create(cfg: lb_config):
    ctx = _ctx_p()
    _check(_lib.lb_create(ctypes.byref(cfg), ctypes.byref(ctx)))
    return ctx


def lb_destroy(ctx):
    return _check(_lib.lb_destroy(ctx), ctx)


def lb_set_source(ctx, x, y, wavelet_ptr, nt):
    return _check(_lib.lb_set_source(ctx, int(x), int(y), wavelet_ptr, int(nt)), ctx)


def lb_set_receivers(ctx, xy_ptr, nrec, nt_capacity):
    return _check(_lib.lb_set_receivers(ctx, xy_ptr, int(nrec), int(nt_capacity)), ctx)


def lb_set_source_3d(ctx, x, y, z, wavelet_ptr, nt):
    return _check(_lib.lb_set_source_3d(ctx, int(x), int(y), int(z), wavelet_ptr, int(nt)), ctx)


def lb_set_receivers_3d(ctx, xyz_ptr, nrec, nt_capacity):
    return _check(_lib.lb_set_receivers_3d(ctx, xyz_ptr, int(nrec), int(nt_capacity)), ctx)


def lb_init_pressure(ctx, p0_ptr, on_device):
    return _check(_lib.lb_init_pressure(ctx, p0_ptr, int(on_device)), ctx)


def lb_step(ctx, n):
    return _check(_lib.lb_step(ctx, int(n)), ctx)


def lb_record_receivers(ctx, out_ptr, nt_max, on_device):
    nt = ctypes.c_int()
    _check(_lib.lb_record_receivers(ctx, out_ptr, int(nt_max), ctypes.byref(nt), int(on_device)),
           ctx)
    return nt.value


def lb_get_pressure(ctx, out_ptr, on_device):
    return _check(_lib.lb_get_pressure(ctx, out_ptr, int(on_device)), ctx)


def lb_get_state(ctx, out_ptr, on_device):
    return _check(_lib.lb_get_state(ctx, out_ptr, int(on_device)), ctx)


def lb_set_state(ctx, in_ptr, on_device):
    return _check(_lib.lb_set_state(ctx, in_ptr, int(on_device)), ctx)


def lb_get_state_f64(ctx, out_ptr, on_device):
    return _check(_lib.lb_get_state_f64(ctx, out_ptr, int(on_device)), ctx)


def lb_set_state_f64(ctx, in_ptr, on_device):
    return _check(_lib.lb_set_state_f64(ctx, in_ptr, int(on_device)), ctx)


def lb_get_pressure_f64(ctx, out_ptr, on_device):
    return _check(_lib.lb_get_pressure_f64(ctx, out_ptr, int(on_device)), ctx)


def lb_get_time(ctx) -> int:
    t = ctypes.c_longlong()
    _check(_lib.lb_get_time(ctx, ctypes.byref(t)), ctx)
    return t.value


def lb_sync(ctx):
    return _check(_lib.lb_sync(ctx), ctx)


def lb_record_rho(ctx, nt_capacity):
    return _check(_lib.lb_record_rho(ctx, int(nt_capacity)), ctx)


def lb_wait_selftest(ctx, timeout_us):
    return _check(_lib.lb_wait_selftest(ctx, int(timeout_us)), ctx)


def lb_footprint(cfg: lb_config, nt, nrec, want_adjoint) -> int:
    b = ctypes.c_size_t()
    _check(_lib.lb_footprint(ctypes.byref(cfg), int(nt), int(nrec), int(want_adjoint),
                             ctypes.byref(b)))
    return b.value


def lb_info(ctx):
    v = (ctypes.c_double * 6)()
    _check(_lib.lb_info(ctx, v, 6), ctx)
    return list(v)


def lb_invariants(ctx):
    """(mass, energy, max |g|, non-finite count); raises LBError(LB_EUNSTABLE) on non-finite."""
    v = (ctypes.c_double * 4)()
    _check(_lib.lb_invariants(ctx, v), ctx)
    return tuple(v)


def lb_invariants_noalloc(g_ptr, c_map_ptr, lattice, nx, ny, c_ref, w_ref, out_ptr, stream):
    """Allocation-free lb_invariants on caller device buffers (results stay on the device)."""
    wr = (ctypes.c_double * 3)(*w_ref) if w_ref is not None else None
    return _check(_lib.lb_invariants_noalloc(g_ptr, c_map_ptr, int(lattice), int(nx), int(ny),
                                             float(c_ref), wr, out_ptr, stream))


def lb_stability_radius(cfg: lb_config, eta, level=0, nk=64) -> float:
    """max |lambda| of the one-step map over an nk x nk grid of wave vectors (host only)."""
    r = ctypes.c_double()
    _check(_lib.lb_stability_radius(ctypes.byref(cfg), float(eta), int(level), int(nk),
                                    ctypes.byref(r)))
    return r.value


def lb_watch_stability(ctx, every, max_growth=0.0):
    return _check(_lib.lb_watch_stability(ctx, int(every), float(max_growth)), ctx)


def lb_set_slab(ctx, y_offset, ny_global, send_lo, send_hi, recv_lo, recv_hi):
    """Mark ctx as rows [y_offset, y_offset + ny) of a grid of ny_global rows; the four row
    buffers are device pointers (or None)."""
    return _check(_lib.lb_set_slab(ctx, int(y_offset), int(ny_global), send_lo, send_hi,
                                   recv_lo, recv_hi), ctx)


def lb_slab_halo_bytes(ctx) -> int:
    b = ctypes.c_size_t()
    _check(_lib.lb_slab_halo_bytes(ctx, ctypes.byref(b)), ctx)
    return b.value


def lb_slab_step(ctxs, steps):
    arr = (_ctx_p * len(ctxs))(*ctxs)
    return _check(_lib.lb_slab_step(arr, len(ctxs), int(steps)), ctxs[0])


def lb_mode_projection(ctx, modes):
    """[(mx, my), ...] integer wave numbers -> list of complex sum_x p(x) exp(-i k.x)."""
    n = len(modes)
    m = (ctypes.c_int * (2 * n))(*[int(v) for pair in modes for v in pair])
    out = (ctypes.c_double * (2 * n))()
    _check(_lib.lb_mode_projection(ctx, m, n, out), ctx)
    return [complex(out[2 * j], out[2 * j + 1]) for j in range(n)]


def lb_checkpoint_every(ctx, every):
    return _check(_lib.lb_checkpoint_every(ctx, int(every)), ctx)


def lb_adjoint(ctx, dJdp_ptr, nt, grad_c_ptr, grad_src_ptr, grad_g0_ptr, on_device):
    return _check(_lib.lb_adjoint(ctx, dJdp_ptr, int(nt), grad_c_ptr, grad_src_ptr, grad_g0_ptr,
                                  int(on_device)), ctx)


def raw():
    """The loaded CDLL (for symbol inspection)."""
    return _lib
