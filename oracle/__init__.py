"""FP64 CPU oracle for the linear lattice-Boltzmann acoustic scheme.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product library never imports, links or runs it, and it shares no code with
the CUDA path: the stepper is plain C in ``lbref.c`` (FP64, push streaming),
built here with gcc and loaded through ctypes.

What each C routine computes, and the passage of arXiv:1704.03172 it follows,
is stated at the top of ``lbref.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["lbref.c", "lbrefine.c", "lbadjoint.c", "lbref3d.c"]
_SO = os.path.join(_HERE, "liblbref.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fast-math, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "lbref.h")])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_SO)
            _declare(_lib)
        return _lib


class _Problem(ctypes.Structure):
    _fields_ = [
        ("Q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("periodic", ctypes.c_int), ("mrt", ctypes.c_int),
        ("tau", ctypes.c_double), ("s", ctypes.c_double * 9), ("w_ref", ctypes.c_double * 3),
        ("c_map", ctypes.POINTER(ctypes.c_float)), ("c_ref", ctypes.c_double),
        ("sponge_width", ctypes.c_int), ("sponge_sigma_max", ctypes.c_double),
        ("src_x", ctypes.c_int), ("src_y", ctypes.c_int),
        ("src", ctypes.POINTER(ctypes.c_double)), ("nt_src", ctypes.c_int),
        ("rec_xy", ctypes.POINTER(ctypes.c_int)), ("nrec", ctypes.c_int),
        ("nthreads", ctypes.c_int),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_pp = ctypes.POINTER(_Problem)


def _declare(L):
    L.orc_velocities.argtypes = [ctypes.c_int, _ip]
    L.orc_moment_matrix.argtypes = [ctypes.c_int, _dp]
    L.orc_moment_inverse.argtypes = [ctypes.c_int, _dp]
    L.orc_weights.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
    L.orc_equilibrium.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, _dp]
    L.orc_equilibrium.restype = None
    L.orc_collide.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp,
                              ctypes.c_double, _dp, _dp]
    L.orc_sponge_sigma.argtypes = [ctypes.c_int] * 5 + [ctypes.c_double]
    L.orc_sponge_sigma.restype = ctypes.c_double
    L.orc_init_pressure.argtypes = [_pp, _dp, _dp]
    L.orc_pressure.argtypes = [_pp, _dp, _dp]
    L.orc_run.argtypes = [_pp, _dp, ctypes.c_int, ctypes.c_int, _dp]
    L.orc_run_f32_stored.argtypes = [_pp, _dp, ctypes.c_int, ctypes.c_int, _dp]
    L.orc_run_f32_stored.restype = ctypes.c_int
    L.orc_max_threads.argtypes = []
    for name in ("orc_velocities", "orc_moment_matrix", "orc_moment_inverse", "orc_weights",
                 "orc_collide", "orc_init_pressure", "orc_pressure", "orc_run",
                 "orc_max_threads"):
        getattr(L, name).restype = ctypes.c_int
    if hasattr(L, "orc_ref_create"):
        _declare_refine(L)
    if hasattr(L, "orc_adjoint"):
        _declare_adjoint(L)


def _declare_refine(L):
    vp = ctypes.c_void_p
    L.orc_ref_create.argtypes = [_pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int]
    L.orc_ref_create.restype = vp
    L.orc_ref_destroy.argtypes = [vp]
    L.orc_ref_destroy.restype = None
    L.orc_ref_dims.argtypes = [vp, _ip, _ip]
    L.orc_ref_fine_cmap.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.orc_ref_init_pressure.argtypes = [vp, _dp]
    L.orc_ref_run.argtypes = [vp, ctypes.c_int, _dp]
    L.orc_ref_pressure.argtypes = [vp, _dp]
    L.orc_ref_fine_pressure.argtypes = [vp, _dp]
    L.orc_ref_states.argtypes = [vp, _dp, _dp]
    L.orc_ref_nest.argtypes = [vp] + [ctypes.c_int] * 4
    L.orc_ref_direction.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.orc_ref_level_dims.argtypes = [vp, ctypes.c_int, _ip, _ip]
    L.orc_ref_level_pressure.argtypes = [vp, ctypes.c_int, _dp]
    L.orc_ref_level_cmap.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
    L.orc_ref_level_state.argtypes = [vp, ctypes.c_int, ctypes.c_int, _dp]
    L.orc_ref_start.argtypes = [vp, ctypes.c_int]
    L.orc_ref_transfer.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   _dp, _dp]
    L.orc_ref_interface.argtypes = [vp, ctypes.c_int, _ip, _ip]
    L.orc_ref_apply_c2f.argtypes = [vp, ctypes.c_int, _dp, _dp, ctypes.c_double]
    L.orc_ref_apply_f2c.argtypes = [vp, ctypes.c_int]
    for n in ("orc_ref_dims", "orc_ref_fine_cmap", "orc_ref_init_pressure", "orc_ref_run",
              "orc_ref_pressure", "orc_ref_fine_pressure", "orc_ref_states", "orc_ref_nest",
              "orc_ref_direction",
              "orc_ref_level_dims", "orc_ref_level_pressure", "orc_ref_level_cmap",
              "orc_ref_level_state", "orc_ref_start", "orc_ref_transfer", "orc_ref_interface",
              "orc_ref_apply_c2f", "orc_ref_apply_f2c"):
        getattr(L, n).restype = ctypes.c_int


class Refined:
    """Refined run (Sec. 4): coarse Problem P plus a patch of coarse cells
    [x0, x0 + nxp] x [y0, y0 + nyp] refined by 2 in space and time; nest() adds patches
    refined by 2 again inside the innermost fine grid."""

    def __init__(self, P: "Problem", x0, y0, nxp, nyp, rule="viscous"):
        """rule "viscous" (R6): fine rates with tau_f - 1/2 = 2 (tau_c - 1/2) and factors
        tau_f / (2 tau_c), 2 tau_c / tau_f per relaxed moment; "paper": the printed factors
        1/2 and 2 with the coarse rates on both grids (they coincide at tau = 1/2)."""
        self.P = P
        self._S = P._struct()
        self.h = lib().orc_ref_create(ctypes.byref(self._S), int(x0), int(y0), int(nxp), int(nyp),
                                      {"viscous": 0, "paper": 1}[rule])
        if not self.h:
            raise ValueError("invalid patch")
        nxf, nyf = ctypes.c_int(), ctypes.c_int()
        self.nI = lib().orc_ref_dims(self.h, ctypes.byref(nxf), ctypes.byref(nyf))
        self.nxf, self.nyf = nxf.value, nyf.value
        self.t = 0

    def fine_cmap(self):
        cf = np.zeros((self.nyf, self.nxf), np.float32)
        lib().orc_ref_fine_cmap(self.h, _ptr(cf, ctypes.c_float))
        return cf

    def nest(self, x0, y0, nxp, nyp):
        """A patch of nodes [x0, x0 + nxp] x [y0, y0 + nyp] of the innermost fine grid (its
        node coordinates), refined by 2 again ("multiples of 2", Sec. 4).  Before
        init_pressure.  Returns the new level's index (2 for the first nested patch)."""
        level = lib().orc_ref_nest(self.h, int(x0), int(y0), int(nxp), int(nyp))
        if level < 0:
            raise ValueError("invalid nested patch")
        return level

    def direction(self, coupling, level=1):
        """Couple level `level` to the grid above it both ways ("both", population by
        population, reading R3), or only "c2f" (coarse -> fine: the coarser grid is never
        corrected) or "f2c" (fine -> coarse: nothing enters the finer grid), the paper's
        switch on the direction of propagation (Sec. 4).  Before init_pressure."""
        d = {"both": 0, "c2f": 1, "f2c": 2}[coupling]
        if lib().orc_ref_direction(self.h, int(level), d):
            raise ValueError("no such level")

    def level_dims(self, level):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        if lib().orc_ref_level_dims(self.h, int(level), ctypes.byref(nx), ctypes.byref(ny)):
            raise ValueError("no such level")
        return ny.value, nx.value

    def level_pressure(self, level):
        """pressure of refined level >= 1 on all of its own nodes"""
        p = np.zeros(self.level_dims(level))
        lib().orc_ref_level_pressure(self.h, int(level), _ptr(p, ctypes.c_double))
        return p

    def level_cmap(self, level):
        c = np.zeros(self.level_dims(level), np.float32)
        lib().orc_ref_level_cmap(self.h, int(level), _ptr(c, ctypes.c_float))
        return c

    def init_pressure(self, p0=None):
        p = None if p0 is None else np.ascontiguousarray(p0, np.float64).reshape(self.P.ny,
                                                                                  self.P.nx)
        lib().orc_ref_init_pressure(self.h, _ptr(p, ctypes.c_double) if p is not None else None)
        self.t = 0

    def run(self, nsteps):
        trace = np.zeros((nsteps, len(self.P.receivers)))
        lib().orc_ref_run(self.h, int(nsteps), _ptr(trace, ctypes.c_double))
        self.t += nsteps
        return trace

    def pressure(self):
        p = np.zeros((self.P.ny, self.P.nx))
        lib().orc_ref_pressure(self.h, _ptr(p, ctypes.c_double))
        return p

    def fine_pressure(self):
        p = np.zeros((self.nyf, self.nxf))
        lib().orc_ref_fine_pressure(self.h, _ptr(p, ctypes.c_double))
        return p

    def states(self):
        gc = np.zeros((self.P.Q, self.P.ny, self.P.nx))
        gf = np.zeros((self.P.Q, self.nyf, self.nxf))
        lib().orc_ref_states(self.h, _ptr(gc, ctypes.c_double), _ptr(gf, ctypes.c_double))
        return gc, gf

    # --- access to the individual transfer functions (the tests that pin them) ---

    def level_state(self, level):
        """state [Q][ny][nx] of level `level` (0: the coarse grid, l >= 1: patch l's fine grid)"""
        ny, nx = (self.P.ny, self.P.nx) if level == 0 else self.level_dims(level)
        g = np.zeros((self.P.Q, ny, nx))
        assert lib().orc_ref_level_state(self.h, int(level), 0, _ptr(g, ctypes.c_double)) == 0
        return g

    def set_level_state(self, level, g):
        ny, nx = (self.P.ny, self.P.nx) if level == 0 else self.level_dims(level)
        g = np.ascontiguousarray(g, np.float64).reshape(self.P.Q, ny, nx)
        assert lib().orc_ref_level_state(self.h, int(level), 1, _ptr(g, ctypes.c_double)) == 0

    def start(self, couple=True):
        """time 0 from the states set with set_level_state: snapshots and (couple) the
        coupling at time 0, as init_pressure does"""
        lib().orc_ref_start(self.h, int(bool(couple)))
        self.t = 0

    def transfer(self, level, to_fine, ax, ay, g):
        """one vector g[Q] carried into node (ax, ay) of the receiving grid of patch `level`
        (its fine grid when to_fine, else the grid above): Eq. coarse-fine dist connect"""
        g = np.ascontiguousarray(g, np.float64)
        out = np.zeros(self.P.Q)
        assert lib().orc_ref_transfer(self.h, int(level), int(bool(to_fine)), int(ax), int(ay),
                                      _ptr(g, ctypes.c_double), _ptr(out, ctypes.c_double)) == 0
        return out

    def interface(self, level=1):
        """interface nodes of patch `level`, (x, y) in the grid above, in snapshot order"""
        n = lib().orc_ref_interface(self.h, int(level), None, None)
        assert n >= 0
        ix = np.zeros(n, np.int32)
        iy = np.zeros(n, np.int32)
        lib().orc_ref_interface(self.h, int(level), _ptr(ix, ctypes.c_int), _ptr(iy, ctypes.c_int))
        return np.stack([ix, iy], 1)

    def apply_c2f(self, level, Ua, Ub, alpha):
        """one coarse -> fine transfer into patch `level` from snapshots Ua, Ub [nI][Q]"""
        Ua = np.ascontiguousarray(Ua, np.float64)
        Ub = np.ascontiguousarray(Ub, np.float64)
        assert lib().orc_ref_apply_c2f(self.h, int(level), _ptr(Ua, ctypes.c_double),
                                       _ptr(Ub, ctypes.c_double), float(alpha)) == 0

    def apply_f2c(self, level):
        """one fine -> coarse correction of the grid above patch `level`"""
        assert lib().orc_ref_apply_f2c(self.h, int(level)) == 0

    def __del__(self):
        try:
            if self.h:
                lib().orc_ref_destroy(self.h)
                self.h = None
        except Exception:
            pass


def _declare_adjoint(L):
    L.orc_adjoint.argtypes = [_pp, _dp, ctypes.c_int, _dp, _dp, _dp, _dp]
    L.orc_adjoint.restype = ctypes.c_int


def adjoint(P: "Problem", g0, nt: int, resid):
    """Discrete adjoint: (dJ/dc [ny, nx], dJ/dS [nt], dJ/dg0 [Q, ny, nx]) for
    dJ/dp^t_r = resid[t, r] over nt steps from g0 (FP64, stores every state)."""
    g0 = np.ascontiguousarray(g0, dtype=np.float64)
    R = np.ascontiguousarray(resid, dtype=np.float64).reshape(nt, len(P.receivers))
    gc = np.zeros((P.ny, P.nx))
    gs = np.zeros(nt)
    gg = np.zeros((P.Q, P.ny, P.nx))
    S = P._struct()
    rc = lib().orc_adjoint(ctypes.byref(S), _ptr(g0, ctypes.c_double), int(nt),
                           _ptr(R, ctypes.c_double), _ptr(gc, ctypes.c_double),
                           _ptr(gs, ctypes.c_double), _ptr(gg, ctypes.c_double))
    assert rc == 0, rc
    return gc, gs, gg


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Problem:
    """One LB problem as the oracle sees it (all fields FP64 except c_map).

    Q: 5 or 9; nx, ny; periodic; mrt; tau (BGK); s: MRT rates, diagonal of S
    in the moment order of App. A; w_ref: D2Q9 (w0, w1, w5) at eta = 1;
    c_map: [ny, nx] float32 sound speed; c_ref; sponge_width, sponge_sigma_max;
    source (x, y, wavelet[nt]) or None; receivers [nrec, 2] int (x, y).
    """

    def __init__(self, Q, nx, ny, c_map, c_ref=None, periodic=False, mrt=False, tau=0.5,
                 s=None, w_ref=(4 / 9, 1 / 9, 1 / 36), sponge_width=0, sponge_sigma_max=0.0,
                 source=None, receivers=None, nthreads=0):
        self.Q, self.nx, self.ny = int(Q), int(nx), int(ny)
        self.c_map = np.ascontiguousarray(c_map, dtype=np.float32).reshape(ny, nx)
        self.c_ref = float(c_ref if c_ref is not None else self.c_map.max())
        self.periodic, self.mrt, self.tau = bool(periodic), bool(mrt), float(tau)
        s = list(s) if s is not None else [1.0] * self.Q
        self.s = np.zeros(9)
        self.s[: len(s)] = s
        self.w_ref = np.asarray(w_ref, dtype=np.float64)
        self.sponge_width, self.sponge_sigma_max = int(sponge_width), float(sponge_sigma_max)
        self.source = None
        if source is not None:
            sx, sy, wav = source
            self.source = (int(sx), int(sy), np.ascontiguousarray(wav, dtype=np.float64))
        self.receivers = (np.ascontiguousarray(receivers, dtype=np.int32).reshape(-1, 2)
                          if receivers is not None else np.zeros((0, 2), np.int32))
        self.nthreads = int(nthreads)

    def _struct(self):
        P = _Problem()
        P.Q, P.nx, P.ny = self.Q, self.nx, self.ny
        P.periodic, P.mrt, P.tau = int(self.periodic), int(self.mrt), self.tau
        for k in range(9):
            P.s[k] = self.s[k]
        for k in range(3):
            P.w_ref[k] = self.w_ref[k]
        P.c_map = _ptr(self.c_map, ctypes.c_float)
        P.c_ref = self.c_ref
        P.sponge_width, P.sponge_sigma_max = self.sponge_width, self.sponge_sigma_max
        if self.source is not None:
            P.src_x, P.src_y = self.source[0], self.source[1]
            P.src = _ptr(self.source[2], ctypes.c_double)
            P.nt_src = len(self.source[2])
        P.rec_xy = _ptr(self.receivers, ctypes.c_int)
        P.nrec = len(self.receivers)
        P.nthreads = self.nthreads
        return P

    def zeros(self):
        return np.zeros((self.Q, self.ny, self.nx), dtype=np.float64)


def init_pressure(P: Problem, p0=None) -> np.ndarray:
    """g = g^eq(rho = p0 / c_s^2, j = 0) at every site."""
    g = P.zeros()
    p = None if p0 is None else np.ascontiguousarray(p0, dtype=np.float64).reshape(P.ny, P.nx)
    S = P._struct()
    rc = lib().orc_init_pressure(ctypes.byref(S), _ptr(p, ctypes.c_double) if p is not None
                                 else None, _ptr(g, ctypes.c_double))
    assert rc == 0
    return g


def pressure(P: Problem, g: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.float64)
    p = np.zeros((P.ny, P.nx))
    S = P._struct()
    assert lib().orc_pressure(ctypes.byref(S), _ptr(g, ctypes.c_double),
                              _ptr(p, ctypes.c_double)) == 0
    return p


def run(P: Problem, g: np.ndarray, nsteps: int, t0: int = 0):
    """Advance g (pre-collision state at time t0) by nsteps; returns (g, trace).

    trace[n, r] is the pressure at receiver r at time t0 + n (before that step).
    """
    g = np.ascontiguousarray(g, dtype=np.float64).copy()
    trace = np.zeros((nsteps, len(P.receivers)))
    S = P._struct()
    rc = lib().orc_run(ctypes.byref(S), _ptr(g, ctypes.c_double), int(t0), int(nsteps),
                       _ptr(trace, ctypes.c_double))
    assert rc == 0, rc
    return g, trace


def run_f32_stored(P: Problem, g: np.ndarray, nsteps: int, t0: int = 0):
    """run() with the state rounded to FP32 after every step (FP64 arithmetic): what storing
    the populations in FP32 alone does to the result."""
    g = np.ascontiguousarray(g, dtype=np.float64).copy()
    trace = np.zeros((nsteps, len(P.receivers)))
    S = P._struct()
    rc = lib().orc_run_f32_stored(ctypes.byref(S), _ptr(g, ctypes.c_double), int(t0),
                                  int(nsteps), _ptr(trace, ctypes.c_double))
    assert rc == 0, rc
    return g, trace


def velocities(Q: int) -> np.ndarray:
    c = np.zeros(2 * Q, dtype=np.int32)
    assert lib().orc_velocities(Q, _ptr(c, ctypes.c_int)) == 0
    return c.reshape(Q, 2)


def moment_matrix(Q: int) -> np.ndarray:
    M = np.zeros(Q * Q)
    assert lib().orc_moment_matrix(Q, _ptr(M, ctypes.c_double)) == 0
    return M.reshape(Q, Q)


def moment_inverse(Q: int) -> np.ndarray:
    M = np.zeros(Q * Q)
    assert lib().orc_moment_inverse(Q, _ptr(M, ctypes.c_double)) == 0
    return M.reshape(Q, Q)


def weights(Q: int, eta: float, w_ref=(4 / 9, 1 / 9, 1 / 36)):
    w = np.zeros(Q)
    wr = np.asarray(w_ref, dtype=np.float64)
    cs2 = ctypes.c_double()
    assert lib().orc_weights(Q, float(eta), _ptr(wr, ctypes.c_double), _ptr(w, ctypes.c_double),
                             ctypes.byref(cs2)) == 0
    return w, cs2.value


def equilibrium(Q, w, cs2, rho, jx, jy):
    w = np.ascontiguousarray(w, dtype=np.float64)
    geq = np.zeros(Q)
    lib().orc_equilibrium(Q, _ptr(w, ctypes.c_double), float(cs2), float(rho), float(jx),
                          float(jy), _ptr(geq, ctypes.c_double))
    return geq


def collide(Q, mrt, tau, s, w, cs2, g):
    s9 = np.zeros(9)
    s9[: len(s)] = s
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(Q)
    assert lib().orc_collide(Q, int(mrt), float(tau), _ptr(s9, ctypes.c_double),
                             _ptr(w, ctypes.c_double), float(cs2), _ptr(g, ctypes.c_double),
                             _ptr(out, ctypes.c_double)) == 0
    return out


def sponge_sigma(x, y, nx, ny, W, smax):
    return lib().orc_sponge_sigma(int(x), int(y), int(nx), int(ny), int(W), float(smax))


def max_threads() -> int:
    return lib().orc_max_threads()


# --- three dimensions (D3Q7, lbref3d.c) ------------------------------------------------

class _Problem3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int), ("tau", ctypes.c_double),
        ("c_map", ctypes.POINTER(ctypes.c_float)), ("c_ref", ctypes.c_double),
        ("sponge_width", ctypes.c_int), ("sponge_sigma_max", ctypes.c_double),
        ("src_x", ctypes.c_int), ("src_y", ctypes.c_int), ("src_z", ctypes.c_int),
        ("src", ctypes.POINTER(ctypes.c_double)), ("nt_src", ctypes.c_int),
        ("rec_xyz", ctypes.POINTER(ctypes.c_int)), ("nrec", ctypes.c_int),
        ("nthreads", ctypes.c_int),
    ]


def _declare3(L):
    pp = ctypes.POINTER(_Problem3)
    L.orc3_init_pressure.argtypes = [pp, _dp, _dp]
    L.orc3_pressure.argtypes = [pp, _dp, _dp]
    L.orc3_run.argtypes = [pp, _dp, ctypes.c_int, ctypes.c_int, _dp]
    for n in ("orc3_init_pressure", "orc3_pressure", "orc3_run"):
        getattr(L, n).restype = ctypes.c_int


class Problem3:
    """A D3Q7 BGK problem: c_map [nz, ny, nx] float32; source (x, y, z, wavelet) or None;
    receivers [nrec, 3] int (x, y, z)."""

    def __init__(self, nx, ny, nz, c_map, c_ref=None, periodic=False, tau=0.5, sponge_width=0,
                 sponge_sigma_max=0.0, source=None, receivers=None, nthreads=0):
        self.Q, self.nx, self.ny, self.nz = 7, int(nx), int(ny), int(nz)
        self.c_map = np.ascontiguousarray(c_map, dtype=np.float32).reshape(nz, ny, nx)
        self.c_ref = float(c_ref if c_ref is not None else self.c_map.max())
        self.periodic, self.tau = bool(periodic), float(tau)
        self.sponge_width, self.sponge_sigma_max = int(sponge_width), float(sponge_sigma_max)
        self.source = None
        if source is not None:
            sx, sy, sz, wav = source
            self.source = (int(sx), int(sy), int(sz), np.ascontiguousarray(wav, dtype=np.float64))
        self.receivers = (np.ascontiguousarray(receivers, dtype=np.int32).reshape(-1, 3)
                          if receivers is not None else np.zeros((0, 3), np.int32))
        self.nthreads = int(nthreads)

    def _struct(self):
        L = lib()
        if not hasattr(L, "_d3"):
            _declare3(L)
            L._d3 = True
        P = _Problem3()
        P.nx, P.ny, P.nz = self.nx, self.ny, self.nz
        P.periodic, P.tau = int(self.periodic), self.tau
        P.c_map = _ptr(self.c_map, ctypes.c_float)
        P.c_ref = self.c_ref
        P.sponge_width, P.sponge_sigma_max = self.sponge_width, self.sponge_sigma_max
        if self.source is not None:
            P.src_x, P.src_y, P.src_z = self.source[:3]
            P.src = _ptr(self.source[3], ctypes.c_double)
            P.nt_src = len(self.source[3])
        P.rec_xyz = _ptr(self.receivers, ctypes.c_int)
        P.nrec = len(self.receivers)
        P.nthreads = self.nthreads
        return P

    def zeros(self):
        return np.zeros((7, self.nz, self.ny, self.nx), dtype=np.float64)


def init_pressure3(P: Problem3, p0=None) -> np.ndarray:
    g = P.zeros()
    S = P._struct()
    p = None if p0 is None else np.ascontiguousarray(p0, np.float64).reshape(P.nz, P.ny, P.nx)
    assert lib().orc3_init_pressure(ctypes.byref(S), _ptr(p, ctypes.c_double) if p is not None
                                    else None, _ptr(g, ctypes.c_double)) == 0
    return g


def pressure3(P: Problem3, g) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.float64)
    p = np.zeros((P.nz, P.ny, P.nx))
    S = P._struct()
    assert lib().orc3_pressure(ctypes.byref(S), _ptr(g, ctypes.c_double),
                               _ptr(p, ctypes.c_double)) == 0
    return p


def run3(P: Problem3, g, nsteps: int, t0: int = 0):
    """Advance a D3Q7 state by nsteps; returns (g, trace[nsteps, nrec])."""
    g = np.ascontiguousarray(g, dtype=np.float64).copy()
    trace = np.zeros((nsteps, len(P.receivers)))
    S = P._struct()
    assert lib().orc3_run(ctypes.byref(S), _ptr(g, ctypes.c_double), int(t0), int(nsteps),
                          _ptr(trace, ctypes.c_double)) == 0
    return g, trace
