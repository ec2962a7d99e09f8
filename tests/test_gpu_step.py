"""GPU parity of the fused LB step (CUDA, FP32 storage) against the FP64 oracle.

Every case feeds the same seeded inputs to both sides through the C ABI
(``LBSim`` -> ``liblbac.so``) and to ``oracle``.  Tolerance: relative L2
<= 1e-5 on the state / pressure and on the receiver traces (FP32 arithmetic
over the stated number of steps), plus an element-wise bound.
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W
from tests.traces import check_every_trace

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def sim_cls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300.sim import LBSim
    return LBSim


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _pair(sim_cls, oracle, Q, nx, ny, c, *, collision="bgk", tau=0.5, s=None, periodic=False,
          sponge=0, smax=0.1, w_ref=(4 / 9, 1 / 9, 1 / 36), source=None, rec=None, steps=1,
          nt_cap=None, c_ref=1.0):
    sim = sim_cls(c, lattice=Q, collision=collision, tau=tau, s=s, c_ref=c_ref,
                  boundary="periodic" if periodic else "zero", sponge_width=sponge,
                  sponge_sigma_max=smax, w_ref=w_ref)
    P = oracle.Problem(Q, nx, ny, c, c_ref=c_ref, periodic=periodic, mrt=collision == "mrt",
                       tau=tau, s=s, w_ref=w_ref, sponge_width=sponge, sponge_sigma_max=smax,
                       source=source, receivers=rec)
    if source is not None:
        sim.set_source(*source)
    if rec is not None:
        sim.set_receivers(rec, nt_cap if nt_cap is not None else steps)
    return sim, P


CASES = [
    # Q, collision, tau, periodic, nx, ny, steps
    (5, "bgk", 0.5, True, 128, 128, 200),
    (5, "bgk", 1.0, False, 37, 29, 120),
    (5, "mrt", 0.5, False, 130, 7, 90),
    (5, "mrt", 0.5, True, 1, 50, 40),
    (5, "bgk", 0.7, False, 300, 1, 40),
    (5, "bgk", 0.5, False, 257, 131, 150),
    (9, "bgk", 0.5, False, 67, 45, 80),
    (9, "mrt", 0.5, True, 64, 64, 100),
    (9, "mrt", 0.5, False, 129, 33, 60),
    (9, "bgk", 0.9, True, 5, 3, 30),
]


@pytest.mark.parametrize("Q,coll,tau,periodic,nx,ny,steps", CASES)
def test_step_matches_oracle_small(sim_cls, oracle_mod, Q, coll, tau, periodic, nx, ny, steps):
    rng = np.random.default_rng(nx * 1000 + ny + Q)
    c = W.random_medium(nx, ny, rng.integers(1 << 30), 0.45, 1.0)
    s = W.mrt_rates(Q, 7) if coll == "mrt" else None
    if Q == 9 and coll == "mrt":
        s = [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3]
    w_ref = (0.4, 0.11, 0.04) if Q == 9 else (4 / 9, 1 / 9, 1 / 36)
    src = (int(rng.integers(nx)), int(rng.integers(ny)), rng.normal(size=steps // 2))
    rec = np.stack([rng.integers(0, nx, 7), rng.integers(0, ny, 7)], 1).astype(np.int32)
    sponge = 0 if periodic else min(4, max(0, min(nx, ny) // 3))
    sim, P = _pair(sim_cls, oracle_mod, Q, nx, ny, c, collision=coll, tau=tau, s=s,
                   periodic=periodic, sponge=sponge, w_ref=w_ref, source=src, rec=rec,
                   steps=steps)
    g0 = rng.normal(size=(Q, ny, nx)).astype(np.float32)
    sim.set_state(g0)
    sim.step(steps)
    gs = sim.state().cpu().numpy()
    tr = sim.traces().cpu().numpy()
    ps = sim.pressure().cpu().numpy()
    sim.close()
    go, tro = oracle_mod.run(P, g0.astype(np.float64), steps)
    assert rel(gs, go) < TOL
    assert np.abs(gs - go).max() < 10 * TOL * np.abs(go).max()
    assert rel(tr, tro) < TOL
    check_every_trace(tr, tro, TOL)
    assert rel(ps, oracle_mod.pressure(P, go)) < TOL


def test_state_roundtrip_and_zero_steps(sim_cls, oracle_mod):
    nx, ny = 45, 33
    c = W.random_medium(nx, ny, 3, 0.5, 1.0)
    sim = sim_cls(c, lattice=5, c_ref=1.0)
    g0 = np.random.default_rng(1).normal(size=(5, ny, nx)).astype(np.float32)
    sim.set_state(g0)
    sim.step(0)
    np.testing.assert_array_equal(sim.state().cpu().numpy(), g0)
    sim.close()


@pytest.mark.parametrize("tau", [1.0, 0.5])
def test_gaussian_pulse_128_periodic_500_steps(sim_cls, oracle_mod, tau):
    n, steps = 128, 500
    c = W.uniform_map(n, n, 1.0)
    p0 = W.gaussian_pulse(n, n, 64, 64, 4.0, 1e-3).astype(np.float32)
    rec = W.ring_receivers(64, 64, 32, [0, 15, 30, 45])
    sim, P = _pair(sim_cls, oracle_mod, 5, n, n, c, tau=tau, periodic=True, rec=rec, steps=steps)
    sim.init_pressure(p0)
    sim.step(steps)
    ps = sim.pressure().cpu().numpy()
    tr = sim.traces().cpu().numpy()
    sim.close()
    g = oracle_mod.init_pressure(P, p0.astype(np.float64))
    g, tro = oracle_mod.run(P, g, steps)
    assert rel(ps, oracle_mod.pressure(P, g)) < TOL
    assert rel(tr, tro) < TOL
    check_every_trace(tr, tro, TOL)


@pytest.mark.parametrize("Q,coll", [(5, "bgk"), (5, "mrt"), (9, "bgk"), (9, "mrt")])
def test_two_layer_full_length_reduced_grid(sim_cls, oracle_mod, Q, coll):
    # the two-layer workload (contrast 1:2, sponge, Ricker source, line of receivers)
    # run for its full 5000 steps on a 256^2 version of the grid
    wl = W.two_layer_workload(256, lattice=Q, collision=coll, nrec=64)
    steps = wl["steps"]
    sim, P = _pair(sim_cls, oracle_mod, Q, 256, 256, wl["c_map"], collision=coll,
                   tau=wl["tau"], s=wl.get("s"), sponge=wl["sponge_width"],
                   smax=wl["sponge_sigma_max"], w_ref=wl["w_ref"], source=wl["source"],
                   rec=wl["receivers"], steps=steps, c_ref=wl["c_ref"])
    snap = 300                 # the wavefront is inside the grid at this time
    sim.init_pressure(None)
    sim.step(snap)
    ps = sim.pressure().cpu().numpy()
    sim.step(steps - snap)
    tr = sim.traces().cpu().numpy()
    sim.close()
    g, tro1 = oracle_mod.run(P, P.zeros(), snap)
    assert rel(ps, oracle_mod.pressure(P, g)) < TOL
    _, tro2 = oracle_mod.run(P, g, steps - snap, t0=snap)
    assert rel(tr, np.concatenate([tro1, tro2])) < TOL
    check_every_trace(tr, np.concatenate([tro1, tro2]), TOL)


@pytest.mark.parametrize("Q,coll,steps", [(5, "bgk", 30), (9, "mrt", 12)])
def test_two_layer_4096_bench_configuration(sim_cls, oracle_mod, Q, coll, steps):
    # full-size grid, same lb_step launch path the benchmark times; a random
    # initial state so that every site carries signal from the first step
    wl = W.two_layer_workload(4096, lattice=Q, collision=coll)
    n = 4096
    sim, P = _pair(sim_cls, oracle_mod, Q, n, n, wl["c_map"], collision=coll, tau=wl["tau"],
                   s=wl.get("s"), sponge=wl["sponge_width"], smax=wl["sponge_sigma_max"],
                   w_ref=wl["w_ref"], source=(wl["source"][0], wl["source"][1],
                                               np.linspace(1, -1, steps)),
                   rec=wl["receivers"], steps=steps, c_ref=wl["c_ref"])
    rng = np.random.default_rng(5)
    g0 = rng.normal(size=(Q, n, n)).astype(np.float32)
    sim.set_state(g0)
    sim.step(steps)
    gs = sim.state().cpu().numpy()
    tr = sim.traces().cpu().numpy()
    sim.close()
    go, tro = oracle_mod.run(P, g0.astype(np.float64), steps)
    assert rel(gs, go) < TOL
    assert rel(tr, tro) < TOL
    check_every_trace(tr, tro, TOL)


@pytest.mark.parametrize("Q,storage,periodic,n", [(5, "f32", False, 200), (5, "bf16", False, 333),
                                                  (9, "f32", True, 96), (9, "bf16", False, 130),
                                                  (5, "f16", False, 150)])
def test_medium_index_matches_per_site_eta2_bitwise(sim_cls, Q, storage, periodic, n):
    # A layered model has few distinct speeds: with a host c_map the step reads a
    # 1-byte medium index and a table; with the same map on the device it reads
    # eta^2 per site.  Both must give bit-identical states and traces.
    import torch
    c = W.layered_fault_model(n, n + 13, 11, n_layers=9, throw=(2.0, n / 10))
    rec = W.line_receivers(24, 20, 4, n - 8)
    src = (n // 3, 20, W.ricker(120, 0.04))
    out = []
    for cm in (c, torch.tensor(c, device="cuda")):
        sim = sim_cls(cm, lattice=Q, storage=storage, c_ref=5500.0, sponge_width=8,
                      boundary="periodic" if periodic else "zero",
                      w_ref=(0.0, 0.01, 0.24) if Q == 9 else (4 / 9, 1 / 9, 1 / 36))
        sim.set_source(*src)
        sim.set_receivers(rec, 120)
        sim.init_pressure(None)
        sim.step(120)
        out.append((sim.info()[4], sim.state().cpu().numpy(), sim.traces(120).cpu().numpy()))
        sim.close()
    (n_idx, g_idx, t_idx), (n_site, g_site, t_site) = out
    assert n_idx == len(np.unique(c)) and n_site == 0
    np.testing.assert_array_equal(g_idx, g_site)
    np.testing.assert_array_equal(t_idx, t_site)
    assert np.abs(t_idx).max() > 0


def test_medium_index_not_used_beyond_256_speeds(sim_cls):
    c = W.random_medium(64, 40, 3, 0.5, 1.0)            # every site its own speed
    sim = sim_cls(c, lattice=5, c_ref=1.0)
    assert sim.info()[4] == 0
    sim.close()
    c2 = np.repeat(np.linspace(0.5, 1.0, 256, dtype=np.float32)[None, :], 3, axis=0)
    sim = sim_cls(c2, lattice=5, c_ref=1.0)             # exactly 256 speeds: indexed
    assert sim.info()[4] == 256
    sim.close()
    c3 = np.repeat(np.linspace(0.5, 1.0, 257, dtype=np.float32)[None, :], 3, axis=0)
    sim = sim_cls(c3, lattice=5, c_ref=1.0)             # 257: per-site eta^2
    assert sim.info()[4] == 0
    sim.close()


@pytest.mark.parametrize("Q,storage,coll,periodic,nx,ny,layered", [
    (5, "bf16", "bgk", False, 3000, 37, True),    # two tasks per row, ragged second task
    (5, "bf16", "mrt", True, 2056, 21, False),
    (5, "bf16", "bgk", False, 2050, 19, True),
    (5, "f16", "bgk", False, 700, 33, False),
    (5, "f16", "mrt", True, 4100, 9, True),
    (9, "bf16", "mrt", False, 2100, 17, True),
    (9, "bf16", "bgk", True, 300, 40, False),
    (9, "f16", "bgk", False, 64, 12, False),
    (5, "bf16", "bgk", True, 33, 5, False),
])
def test_staged_step_matches_direct_step_bitwise(sim_cls, Q, storage, coll, periodic, nx, ny,
                                                 layered):
    # The TMA-staged persistent kernel (forced here; automatic for 16-bit storage on wide
    # rows) runs the register-streaming step's per-site arithmetic: states and traces must agree bit for bit, including the
    # first step from an arbitrary state (read in place), the sponge, the source and
    # both medium forms.
    rng = np.random.default_rng(nx + ny)
    c = (W.layered_fault_model(nx, ny, 5, n_layers=7, throw=(1.0, 4.0)) if layered
         else W.random_medium(nx, ny, 6, 0.5, 1.0))
    g0 = (rng.normal(size=(Q, ny, nx)) * 0.1).astype(np.float32)
    rec = np.stack([rng.integers(0, nx, 12), rng.integers(0, ny, 12)], 1).astype(np.int32)
    src = (nx // 3, ny // 2, W.ricker(30, 0.05))
    s = ([1.0, 1.0, 1.0, 1.6, 1.3] if Q == 5 else [1.0, 1.0, 1.0, 1.7, 1.4, 1.6, 1.2, 1.2, 1.4])
    out = []
    for kernel in ("staged", "direct"):
        sim = sim_cls(c, lattice=Q, collision=coll, s=s if coll == "mrt" else None, tau=0.6,
                      storage=storage, c_ref=float(c.max()), sponge_width=0 if periodic else 4,
                      boundary="periodic" if periodic else "zero", step_kernel=kernel,
                      w_ref=(0.0, 0.01, 0.24) if Q == 9 else (4 / 9, 1 / 9, 1 / 36))
        sim.set_source(*src)
        sim.set_receivers(rec, 30)
        sim.set_state(g0)
        sim.step(30)
        out.append((sim.state().cpu().numpy(), sim.traces(30).cpu().numpy()))
        sim.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert np.isfinite(out[0][0]).all() and np.abs(out[0][1]).max() > 0


def test_bounded_wait_gives_up_reports_once_and_leaves_the_context_usable(sim_cls):
    # The failure path of the TMA-staged step's bounded waits, driven without any fault: a
    # one-block self-test waits on an mbarrier phase that nothing completes, gives up after
    # 2 ms and raises the fault flag.  lb_sync reports LB_ETIMEOUT once; the context keeps
    # stepping, and the state it produces equals a run without the self-test bit for bit.
    from paper_1704_03172_gb300 import lbac
    nx, ny = 2100, 16
    c = W.random_medium(nx, ny, 12, 0.5, 1.0)
    g0 = (np.random.default_rng(1).normal(size=(5, ny, nx)) * 0.1).astype(np.float32)
    out = []
    for probe in (False, True):
        sim = sim_cls(c, storage="bf16", c_ref=1.0, sponge_width=4, step_kernel="staged")
        sim.set_state(g0)
        sim.step(5)
        lbac.lb_sync(sim.ctx)
        if probe:
            lbac.lb_wait_selftest(sim.ctx, 2000)
            with pytest.raises(lbac.LBError) as e:
                lbac.lb_sync(sim.ctx)
            assert e.value.status == lbac.LB_ETIMEOUT
            lbac.lb_sync(sim.ctx)                      # reported once
        sim.step(5)
        lbac.lb_sync(sim.ctx)
        out.append(sim.state().cpu().numpy())
        sim.close()
    np.testing.assert_array_equal(out[0], out[1])
