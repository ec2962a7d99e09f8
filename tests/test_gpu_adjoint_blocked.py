"""GPU adjoint with the time-blocked reverse sweep against the FP64 adjoint oracle.

lb_adjoint runs 8 (D2Q5) or 4 (D2Q9) adjoint levels per launch on 32 x 32 or 40 x 40 tiles
with a halo (48 x 48 regions), and single levels where fewer remain in a replay
sub-segment.  These cases use grids with interior tiles (16-byte region loads and tile
stores) and ragged edge tiles, receivers on tile edges and inside halos (two at the same
site), the source on a tile corner, checkpoint intervals that mix blocked and single
levels, and periodic grids smaller than one region (a site appears several times in it).
Tolerance as for the other FP32 adjoint tests: relative L2 <= 1e-4.
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-4


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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _receivers(rng, nx, ny, out):
    # tile edges and corners of the blocked sweep, halo positions, grid edges, a duplicate
    pts = [(out - 1, out), (out, out - 1), (2 * out, out + 3), (out + 5, 2 * out - 1),
           (nx - 1, ny - 1), (0, ny // 2), (nx // 2, 0), (out + 2, out + 2), (out + 2, out + 2)]
    pts = [(x % nx, y % ny) for x, y in pts]
    more = np.stack([rng.integers(0, nx, 6), rng.integers(0, ny, 6)], 1)
    return np.concatenate([np.array(pts), more]).astype(np.int32)


CASES = [
    # Q, collision, tau, s, periodic, sponge, nx, ny, checkpoint_every, nt
    (5, "bgk", 0.5, None, False, 6, 150, 110, 13, 40),
    (5, "mrt", 0.5, [1.2, 0.9, 0.9, 1.6, 1.3], False, 8, 131, 97, 40, 40),
    (5, "bgk", 0.8, None, True, 0, 100, 70, 11, 33),
    (5, "bgk", 0.6, None, True, 0, 20, 30, 16, 24),      # grid smaller than one region
    (9, "mrt", 0.5, [1.0, 1.0, 1.0, 1.7, 1.4, 1.6, 1.2, 1.2, 1.4], False, 5, 150, 110, 9, 37),
    (9, "bgk", 0.7, None, True, 0, 123, 85, 40, 40),
    (9, "bgk", 0.9, None, True, 0, 30, 22, 7, 21),       # grid smaller than one region
]


@pytest.mark.parametrize("mode", ["ckpt", "tape"])
@pytest.mark.parametrize("case", CASES)
def test_blocked_adjoint_matches_oracle(sim_cls, oracle_mod, case, mode):
    # ckpt: checkpoints every `every` steps, replays; tape: the forward run records rho
    # (lb_record_rho) and the sweep reads it, no replay
    Q, coll, tau, s, per, sponge, nx, ny, every, nt = case
    out = 48 - 2 * (8 if Q == 5 else 4)
    rng = np.random.default_rng(nx * 1000 + ny)
    c = W.random_medium(nx, ny, int(rng.integers(1 << 30)), 0.5, 1.0)
    rec = _receivers(rng, nx, ny, out)
    src = (out % nx, out % ny, rng.normal(size=nt))           # on a tile corner
    kw = dict(tau=tau, s=s, w_ref=(0.4, 0.11, 0.04), c_ref=1.0)
    sim = sim_cls(c, lattice=Q, collision=coll, boundary="periodic" if per else "zero",
                  sponge_width=sponge, sponge_sigma_max=0.15, **kw)
    sim.set_source(*src)
    sim.set_receivers(rec, nt)
    g0 = (rng.normal(size=(Q, ny, nx)) * 0.1).astype(np.float32)
    sim.set_state(g0)
    if mode == "ckpt":
        sim.checkpoint_every(every)
    else:
        sim.record_rho(nt)
    sim.step(nt)
    tr = sim.traces(nt).cpu().numpy()
    R = tr - rng.normal(size=tr.shape).astype(np.float32)
    gc, gs, gg = sim.adjoint(R, nt, want_g0=True)
    gc, gs, gg = gc.cpu().numpy(), gs.cpu().numpy(), gg.cpu().numpy()
    sim.close()
    P = oracle_mod.Problem(Q, nx, ny, c, periodic=per, mrt=coll == "mrt", sponge_width=sponge,
                           sponge_sigma_max=0.15, source=src, receivers=rec, **kw)
    oc, os_, og = oracle_mod.adjoint(P, g0.astype(np.float64), nt, R.astype(np.float64))
    assert rel(gc, oc) < TOL
    assert rel(gs, os_) < TOL
    assert rel(gg, og) < TOL
    # element-wise too: the blocked sweep must not lose a tile, a halo or a receiver
    scale = np.abs(oc).max()
    assert np.abs(gc - oc).max() < 1e-3 * scale
    assert np.abs(gg - og).max() < 1e-3 * np.abs(og).max()


def test_blocked_adjoint_bf16_storage(sim_cls, oracle_mod):
    # BF16 replays, FP32 blocked sweep.  dJ/dS and dJ/dg0 depend on the adjoint state alone
    # and keep the FP32 bound; dJ/dc weighs the BF16 densities rho^t (4e-2, as for the
    # one-level sweep).
    Q, nx, ny, nt = 5, 140, 100, 32
    rng = np.random.default_rng(7)
    c = W.random_medium(nx, ny, 3, 0.5, 1.0)
    rec = _receivers(rng, nx, ny, 32)
    src = (70, 50, rng.normal(size=nt))
    kw = dict(tau=0.5, s=[1.2, 0.9, 0.9, 1.6, 1.3], c_ref=1.0)
    P = oracle_mod.Problem(Q, nx, ny, c, mrt=True, sponge_width=6, sponge_sigma_max=0.15,
                           source=src, receivers=rec, **kw)
    _, tro = oracle_mod.run(P, P.zeros(), nt)
    R = (tro - rng.normal(size=tro.shape) * 1e-3).astype(np.float32)
    oc, os_, og = oracle_mod.adjoint(P, P.zeros(), nt, R.astype(np.float64))
    sim = sim_cls(c, lattice=Q, collision="mrt", sponge_width=6, sponge_sigma_max=0.15,
                  storage="bf16", **kw)
    sim.set_source(*src)
    sim.set_receivers(rec, nt)
    sim.init_pressure(None)
    sim.checkpoint_every(12)
    sim.step(nt)
    gc, gs, gg = sim.adjoint(R, nt, want_g0=True)
    gc, gs, gg = gc.cpu().numpy(), gs.cpu().numpy(), gg.cpu().numpy()
    sim.close()
    assert rel(gs, os_) < TOL
    assert rel(gg, og) < TOL
    assert rel(gc, oc) < 4e-2


def _tape_run(sim_cls, c, Q, nt, rec, src, storage="f32", mode="tape", time_block=1, seed=7):
    rng = np.random.default_rng(seed)
    ny, nx = c.shape
    kw = dict(tau=0.5, s=[1.2, 0.9, 0.9, 1.6, 1.3] if Q == 5 else None, c_ref=1.0,
              w_ref=(0.4, 0.11, 0.04))
    sim = sim_cls(c, lattice=Q, collision="mrt" if Q == 5 else "bgk", sponge_width=6,
                  sponge_sigma_max=0.15, storage=storage, time_block=time_block, **kw)
    sim.set_source(*src)
    sim.set_receivers(rec, nt)
    sim.init_pressure(None)
    if mode == "tape":
        sim.record_rho(nt)
    else:
        sim.checkpoint_every(12)
    sim.step(nt)
    R = (sim.traces(nt).cpu().numpy() - rng.normal(size=(nt, len(rec))) * 1e-3).astype(np.float32)
    gc, gs, gg = sim.adjoint(R, nt, want_g0=True)
    out = (gc.cpu().numpy(), gs.cpu().numpy(), gg.cpu().numpy(), R)
    sim.close()
    return out, kw


def test_tape_and_checkpoint_gradients_agree(sim_cls):
    nx, ny, nt = 150, 110, 45
    c = W.random_medium(nx, ny, 11, 0.5, 1.0)
    rec = _receivers(np.random.default_rng(2), nx, ny, 32)
    src = (75, 55, W.ricker(nt, 0.06))
    a, _ = _tape_run(sim_cls, c, 5, nt, rec, src, mode="tape")
    b, _ = _tape_run(sim_cls, c, 5, nt, rec, src, mode="ckpt")
    for x, y in zip(a[:3], b[:3]):
        assert rel(x, y) < 1e-6


@pytest.mark.parametrize("storage,tol_c", [("f16", 2e-2), ("bf16", 4e-2)])
def test_tape_adjoint_low_precision_storage(sim_cls, oracle_mod, storage, tol_c):
    # with the tape the adjoint needs only rho, so FP16 storage (whose range scales are not
    # replayed) works too; dJ/dS and dJ/dg0 depend on the adjoint state alone and keep the
    # FP32 bound, dJ/dc carries the stored densities' rounding
    Q, nx, ny, nt = 5, 140, 100, 40
    c = W.random_medium(nx, ny, 3, 0.5, 1.0)
    rec = _receivers(np.random.default_rng(5), nx, ny, 32)
    src = (70, 50, W.ricker(nt, 0.06))
    (gc, gs, gg, R), kw = _tape_run(sim_cls, c, Q, nt, rec, src, storage=storage)
    P = oracle_mod.Problem(Q, nx, ny, c, mrt=True, sponge_width=6, sponge_sigma_max=0.15,
                           source=src, receivers=rec, **kw)
    oc, os_, og = oracle_mod.adjoint(P, P.zeros(), nt, R.astype(np.float64))
    assert rel(gs, os_) < TOL
    assert rel(gg, og) < TOL
    assert rel(gc, oc) < tol_c


def test_tape_with_time_blocked_forward(sim_cls, oracle_mod):
    # an FP32 forward with 8 fused steps per launch records rho through the time-blocked
    # kernel's per-level output; steps that would leave the tape run singly
    Q, nx, ny, nt = 5, 150, 110, 43
    c = W.random_medium(nx, ny, 4, 0.5, 1.0)
    rec = _receivers(np.random.default_rng(6), nx, ny, 32)
    src = (75, 55, W.ricker(nt, 0.06))
    (gc, gs, gg, R), kw = _tape_run(sim_cls, c, Q, nt, rec, src, time_block=8)
    P = oracle_mod.Problem(Q, nx, ny, c, mrt=True, sponge_width=6, sponge_sigma_max=0.15,
                           source=src, receivers=rec, **kw)
    oc, os_, og = oracle_mod.adjoint(P, P.zeros(), nt, R.astype(np.float64))
    assert rel(gc, oc) < TOL
    assert rel(gs, os_) < TOL
    assert rel(gg, og) < TOL


def test_tape_lifecycle(sim_cls):
    from paper_1704_03172_gb300 import lbac
    nx, ny = 64, 48
    c = W.random_medium(nx, ny, 8, 0.5, 1.0)
    sim = sim_cls(c, sponge_width=4)
    sim.set_receivers(np.array([[30, 20]], np.int32), 30)
    sim.init_pressure(None)
    sim.record_rho(10)
    sim.step(20)                                   # the tape covers the first 10 steps only
    with pytest.raises(lbac.LBError) as e:         # no checkpoints, tape too short for 20
        sim.adjoint(np.ones((20, 1), np.float32), 20)
    assert e.value.status == lbac.LB_ESTATE
    gc, gs, _ = sim.adjoint(np.ones((10, 1), np.float32), 10)
    assert np.isfinite(gc.cpu().numpy()).all()
    sim.record_rho(0)                              # freed
    with pytest.raises(lbac.LBError):
        sim.adjoint(np.ones((10, 1), np.float32), 10)
    sim.close()


@pytest.mark.parametrize("Q", [5, 9])
def test_tape_from_the_staged_step(sim_cls, oracle_mod, Q):
    # BF16 on rows of >= 1024 sites runs the TMA-staged step, which writes the tape through
    # the same per-site code; dJ/dS and dJ/dg0 keep the FP32 bound, dJ/dc the BF16 one
    nx, ny, nt = 1100, 40, 30
    rng = np.random.default_rng(Q)
    c = W.random_medium(nx, ny, 9, 0.5, 1.0)
    # receivers within reach of the source in nt steps (c_s <= 0.7 cells per step)
    rec = np.stack([rng.integers(535, 566, 10), rng.integers(8, 33, 10)], 1).astype(np.int32)
    src = (550, 20, W.ricker(nt, 0.06))
    kw = dict(tau=0.5, c_ref=1.0, w_ref=(0.4, 0.11, 0.04))
    sim = sim_cls(c, lattice=Q, sponge_width=4, sponge_sigma_max=0.15, storage="bf16", **kw)
    assert sim.info()[2] == 2                       # 16-bit storage: the staged step
    sim.set_source(*src)
    sim.set_receivers(rec, nt)
    sim.init_pressure(None)
    sim.record_rho(nt)
    sim.step(nt)
    R = (sim.traces(nt).cpu().numpy() - rng.normal(size=(nt, len(rec))) * 1e-3).astype(np.float32)
    gc, gs, gg = sim.adjoint(R, nt, want_g0=True)
    gc, gs, gg = gc.cpu().numpy(), gs.cpu().numpy(), gg.cpu().numpy()
    sim.close()
    P = oracle_mod.Problem(Q, nx, ny, c, sponge_width=4, sponge_sigma_max=0.15, source=src,
                           receivers=rec, **kw)
    oc, os_, og = oracle_mod.adjoint(P, P.zeros(), nt, R.astype(np.float64))
    assert rel(gs, os_) < TOL
    assert rel(gg, og) < TOL
    assert rel(gc, oc) < 4e-2
