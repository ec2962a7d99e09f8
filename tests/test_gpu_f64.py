"""GPU parity at FP64 (LB_F64, test-only storage) against the FP64 oracle.

The FP64 step runs the production per-site code (collision, weights, source,
sponge of ``lb_kernels.cuh``) with double arithmetic, so the two sides differ
only by rounding order.  Bound: relative L2 <= 1e-11 on populations and
pressure.  Each site-step is a few tens of FP64 operations (unit roundoff
1.1e-16), and the error grows at most linearly over <= 500 steps, about 1e-12.
A coefficient or a step held in FP32 anywhere on the path shows up at 1e-8 or
above.  Receiver traces are FP32 rows (one rounding of an FP64 value):
relative L2 <= 1e-6.
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL_TRACE = 1e-6


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


@pytest.mark.parametrize("tau", [1.0, 0.5])
def test_gaussian_pulse_128_periodic_500_steps_fp64(sim_cls, oracle_mod, tau):
    # 128^2 periodic, eta = 1, Gaussian pressure pulse, 500 steps, receivers on a ring
    n, steps = 128, 500
    c = W.uniform_map(n, n, 1.0)
    p0 = W.gaussian_pulse(n, n, 64, 64, 4.0, 1e-3)
    rec = W.ring_receivers(64, 64, 32, [0, 15, 30, 45])
    sim = sim_cls(c, lattice=5, tau=tau, storage="f64", c_ref=1.0, boundary="periodic")
    sim.set_receivers(rec, steps)
    sim.init_pressure(p0.astype(np.float32))
    sim.step(steps)
    ps = sim.pressure().cpu().numpy()
    gs = sim.state().cpu().numpy()
    tr = sim.traces().cpu().numpy()
    sim.close()
    assert ps.dtype == np.float64 and gs.dtype == np.float64
    P = oracle_mod.Problem(5, n, n, c, c_ref=1.0, periodic=True, tau=tau, receivers=rec)
    g = oracle_mod.init_pressure(P, p0.astype(np.float32).astype(np.float64))
    g, tro = oracle_mod.run(P, g, steps)
    assert rel(gs, g) < TOL64
    assert rel(ps, oracle_mod.pressure(P, g)) < TOL64
    assert rel(tr, tro) < TOL_TRACE


CASES = [
    # Q, collision, tau, periodic, nx, ny, steps
    (5, "bgk", 0.5, False, 257, 131, 150),
    (5, "bgk", 0.8, True, 37, 29, 120),
    (5, "mrt", 0.5, False, 130, 7, 90),
    (5, "mrt", 0.5, True, 64, 33, 100),
    (9, "bgk", 0.5, False, 67, 45, 80),
    (9, "bgk", 0.9, True, 5, 3, 30),
    (9, "mrt", 0.5, False, 129, 33, 60),
    (9, "mrt", 0.5, True, 64, 64, 100),
]


@pytest.mark.parametrize("Q,coll,tau,periodic,nx,ny,steps", CASES)
def test_step_matches_oracle_fp64(sim_cls, oracle_mod, Q, coll, tau, periodic, nx, ny, steps):
    # random heterogeneous medium, point source, sponge (zero ghost), random FP64 state
    rng = np.random.default_rng(nx * 1000 + ny + Q + 7)
    c = W.random_medium(nx, ny, int(rng.integers(1 << 30)), 0.45, 1.0)
    s = W.mrt_rates(Q, 11) if coll == "mrt" else None
    if Q == 9 and coll == "mrt":
        s = [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3]
    w_ref = (0.4, 0.11, 0.04) if Q == 9 else (4 / 9, 1 / 9, 1 / 36)
    src = (int(rng.integers(nx)), int(rng.integers(ny)), rng.normal(size=steps // 2))
    rec = np.stack([rng.integers(0, nx, 7), rng.integers(0, ny, 7)], 1).astype(np.int32)
    sponge = 0 if periodic else min(4, max(0, min(nx, ny) // 3))
    sim = sim_cls(c, lattice=Q, collision=coll, tau=tau, s=s, storage="f64", c_ref=1.0,
                  boundary="periodic" if periodic else "zero", sponge_width=sponge,
                  sponge_sigma_max=0.1, w_ref=w_ref)
    sim.set_source(*src)
    sim.set_receivers(rec, steps)
    g0 = rng.normal(size=(Q, ny, nx))
    sim.set_state(g0)
    np.testing.assert_array_equal(sim.state().cpu().numpy(), g0)  # FP64 round trip
    sim.step(steps)
    gs = sim.state().cpu().numpy()
    ps = sim.pressure().cpu().numpy()
    tr = sim.traces().cpu().numpy()
    sim.close()
    P = oracle_mod.Problem(Q, nx, ny, c, c_ref=1.0, periodic=periodic, mrt=coll == "mrt",
                           tau=tau, s=s, w_ref=w_ref, sponge_width=sponge, sponge_sigma_max=0.1,
                           source=src, receivers=rec)
    go, tro = oracle_mod.run(P, g0, steps)
    assert rel(gs, go) < TOL64
    assert np.abs(gs - go).max() < 10 * TOL64 * np.abs(go).max()
    assert rel(ps, oracle_mod.pressure(P, go)) < TOL64
    assert rel(tr, tro) < TOL_TRACE


@pytest.mark.parametrize("periodic", [False, True])
def test_d3q7_matches_oracle_fp64(sim_cls, oracle_mod, periodic):
    nx, ny, nz, steps = 41, 23, 17, 60
    rng = np.random.default_rng(5 + periodic)
    c = rng.uniform(0.5, 1.0, size=(nz, ny, nx)).astype(np.float32)
    src = (nx // 3, ny // 2, nz // 2, W.ricker(steps, 0.06))
    rec = np.stack([rng.integers(0, nx, 9), rng.integers(0, ny, 9), rng.integers(0, nz, 9)],
                   1).astype(np.int32)
    sponge = 0 if periodic else 3
    sim = sim_cls(c, lattice=7, tau=0.6, storage="f64", c_ref=1.0,
                  boundary="periodic" if periodic else "zero", sponge_width=sponge,
                  sponge_sigma_max=0.15)
    sim.set_source(*src)
    sim.set_receivers(rec, steps)
    g0 = rng.normal(size=(7, nz, ny, nx))
    sim.set_state(g0)
    sim.step(steps)
    gs = sim.state().cpu().numpy()
    tr = sim.traces(steps).cpu().numpy()
    sim.close()
    P = oracle_mod.Problem3(nx, ny, nz, c, c_ref=1.0, periodic=periodic, tau=0.6,
                            sponge_width=sponge, sponge_sigma_max=0.15, source=src, receivers=rec)
    go, tro = oracle_mod.run3(P, g0, steps)
    assert rel(gs, go) < TOL64
    assert rel(tr, tro) < TOL_TRACE


def test_fp64_rejects_what_it_does_not_serve(sim_cls):
    from paper_1704_03172_gb300 import lbac
    c = np.ones((16, 40), np.float32)
    with pytest.raises(lbac.LBError):
        sim_cls(c, lattice=5, storage="f64", c_ref=1.0, step_kernel="staged")
    with pytest.raises(lbac.LBError):
        sim_cls(c, lattice=5, storage="f64", c_ref=1.0, time_block=4)
    sim = sim_cls(c, lattice=5, storage="f64", c_ref=1.0)
    for call in (lambda: lbac.lb_checkpoint_every(sim.ctx, 10),
                 lambda: lbac.lb_record_rho(sim.ctx, 10),
                 lambda: lbac.lb_invariants(sim.ctx),
                 lambda: lbac.lb_mode_projection(sim.ctx, [(1, 0)])):
        with pytest.raises(lbac.LBError):
            call()
    sim.close()
    f32 = sim_cls(c, lattice=5, c_ref=1.0)  # the FP64 transforms need an FP64 context
    import torch
    out = torch.zeros((5, 16, 40), dtype=torch.float64, device="cuda")
    with pytest.raises(lbac.LBError):
        lbac.lb_get_state_f64(f32.ctx, out.data_ptr(), 1)
    f32.close()
