"""GPU parity of temporal blocking (K fused steps per launch, tile in shared memory).

Temporal blocking changes only where intermediate states live, so the results
must match the FP64 oracle to the same FP32 tolerance as single steps, for
every K, lattice, collision and boundary, with ragged tiles, step counts that
are not multiples of K, receivers in every time level and the source inside
the recomputed halo of neighbouring tiles.
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


CASES = [
    # Q, collision, s, periodic, nx, ny, steps, K
    (5, "bgk", None, False, 70, 45, 61, 4),
    (5, "bgk", None, False, 133, 97, 50, 8),
    (5, "mrt", [1.2, 0.9, 0.9, 1.6, 1.3], False, 96, 64, 47, 6),
    (5, "bgk", None, True, 64, 64, 40, 2),
    (5, "mrt", [1.0, 1.0, 1.0, 1.3, 1.9], True, 100, 36, 33, 4),
    (5, "bgk", None, False, 600, 300, 41, 8),     # 3 strips, several row chunks
    (5, "mrt", [1.2, 0.9, 0.9, 1.6, 1.3], True, 300, 70, 50, 16),
    (5, "bgk", None, True, 40, 33, 37, 8),        # periodic grid narrower than one strip
    (5, "bgk", None, False, 257, 131, 70, 16),
    (5, "bgk", None, False, 5, 300, 24, 4),
    (9, "bgk", None, False, 77, 65, 30, 4),
    (9, "mrt", [1.0, 1.0, 1.0, 1.7, 1.4, 1.6, 1.2, 1.2, 1.4], True, 64, 96, 26, 2),
]


@pytest.mark.parametrize("Q,coll,s,periodic,nx,ny,steps,K", CASES)
def test_time_blocked_steps_match_oracle(sim_cls, oracle_mod, Q, coll, s, periodic, nx, ny,
                                         steps, K):
    rng = np.random.default_rng(nx + ny + K)
    c = W.random_medium(nx, ny, 5, 0.5, 1.0)
    sponge = 0 if periodic else 7
    src = (nx // 3, ny // 2, rng.normal(size=steps))
    rec = np.stack([rng.integers(0, nx, 11), rng.integers(0, ny, 11)], 1).astype(np.int32)
    kw = dict(tau=0.5, s=s, w_ref=(0.4, 0.11, 0.04), c_ref=1.0)
    sim = sim_cls(c, lattice=Q, collision=coll, boundary="periodic" if periodic else "zero",
                  sponge_width=sponge, sponge_sigma_max=0.1, time_block=K, **kw)
    sim.set_source(*src)
    sim.set_receivers(rec, steps)
    g0 = rng.normal(size=(Q, ny, nx)).astype(np.float32)
    sim.set_state(g0)
    sim.step(steps)
    gs = sim.state().cpu().numpy()
    tr = sim.traces().cpu().numpy()
    sim.close()
    P = oracle_mod.Problem(Q, nx, ny, c, periodic=periodic, mrt=coll == "mrt",
                           sponge_width=sponge, sponge_sigma_max=0.1, source=src,
                           receivers=rec, **kw)
    go, tro = oracle_mod.run(P, g0.astype(np.float64), steps)
    assert rel(gs, go) < TOL
    assert rel(tr, tro) < TOL
    check_every_trace(tr, tro, TOL)


def test_time_blocked_two_layer_4096(sim_cls, oracle_mod):
    # the bench workload at full size with K = 4, from a random state
    wl = W.two_layer_workload(4096)
    n, steps = 4096, 22
    src = (wl["source"][0], wl["source"][1], np.linspace(1.0, -1.0, steps))
    sim = sim_cls(wl["c_map"], lattice=5, tau=0.5, c_ref=wl["c_ref"],
                  sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                  time_block=4)
    sim.set_source(*src)
    sim.set_receivers(wl["receivers"], steps)
    g0 = np.random.default_rng(6).normal(size=(5, n, n)).astype(np.float32)
    sim.set_state(g0)
    sim.step(steps)
    gs = sim.state().cpu().numpy()
    tr = sim.traces().cpu().numpy()
    sim.close()
    P = oracle_mod.Problem(5, n, n, wl["c_map"], c_ref=wl["c_ref"], tau=0.5,
                           sponge_width=wl["sponge_width"],
                           sponge_sigma_max=wl["sponge_sigma_max"], source=src,
                           receivers=wl["receivers"])
    go, tro = oracle_mod.run(P, g0.astype(np.float64), steps)
    assert rel(gs, go) < TOL
    assert rel(tr, tro) < TOL
    check_every_trace(tr, tro, TOL)


def test_time_blocking_with_adjoint_checkpoints(sim_cls, oracle_mod):
    # checkpoint times and trace rows must stay exact when steps are fused
    nx, ny, nt = 80, 52, 45
    rng = np.random.default_rng(9)
    c = W.random_medium(nx, ny, 8, 0.5, 1.0)
    src = (30, 20, rng.normal(size=nt))
    rec = np.stack([rng.integers(0, nx, 6), rng.integers(0, ny, 6)], 1).astype(np.int32)
    sim = sim_cls(c, lattice=5, tau=0.5, c_ref=1.0, sponge_width=5, time_block=4)
    sim.set_source(*src)
    sim.set_receivers(rec, nt)
    sim.init_pressure(None)
    sim.checkpoint_every(10)
    sim.step(nt)
    tr = sim.traces(nt).cpu().numpy()
    R = rng.normal(size=tr.shape).astype(np.float32)
    gc, gsrc, _ = sim.adjoint(R, nt)
    sim.close()
    P = oracle_mod.Problem(5, nx, ny, c, c_ref=1.0, tau=0.5, sponge_width=5, sponge_sigma_max=0.1,
                           source=src, receivers=rec)
    _, tro = oracle_mod.run(P, P.zeros(), nt)
    assert rel(tr, tro) < TOL
    check_every_trace(tr, tro, TOL)
    oc, os_, _ = oracle_mod.adjoint(P, P.zeros(), nt, R.astype(np.float64))
    assert rel(gc.cpu().numpy(), oc) < 1e-4
    assert rel(gsrc.cpu().numpy(), os_) < 1e-4


def test_time_block_rejected_where_unsupported(sim_cls):
    from paper_1704_03172_gb300 import lbac
    c = W.uniform_map(32, 32, 1.0)
    for kw in (dict(lattice=9, time_block=8), dict(lattice=5, time_block=3),
               dict(lattice=5, time_block=4, storage="f16"),
               dict(lattice=9, time_block=4, storage="bf16")):
        with pytest.raises(lbac.LBError):
            sim_cls(c, c_ref=1.0, **kw)


def test_time_blocked_steps_agree_with_single_steps(sim_cls):
    # the fused levels run the single step's per-site arithmetic in FP32: the two forms agree
    # to a few FP32 roundings per step on the layered model (sponge, source, receivers)
    n, steps = 520, 96
    c = W.layered_fault_model(n, n, 3, n_layers=9, throw=(2.0, 20.0))
    rec = W.line_receivers(40, 30, 20, n - 40)
    out = []
    for K in (1, 8, 16):
        sim = sim_cls(c, lattice=5, tau=0.5, c_ref=5500.0, sponge_width=20, time_block=K)
        sim.set_source(n // 2, 30, W.ricker(steps, 0.02))
        sim.set_receivers(rec, steps)
        sim.init_pressure(None)
        sim.step(steps)
        out.append((sim.state().cpu().numpy(), sim.traces(steps).cpu().numpy()))
        sim.close()
    for g, tr in out[1:]:
        assert rel(g, out[0][0]) < 1e-6
        assert rel(tr, out[0][1]) < 1e-6


@pytest.mark.parametrize("K", [8, 16])
def test_bf16_time_blocking_against_the_oracle(sim_cls, oracle_mod, K):
    # BF16 storage with K fused FP32 levels rounds to BF16 once per K steps: within the BF16
    # bound of the single-step form (rel-L2 4e-2) and closer to the oracle than it
    n, steps = 256, 400
    wl = W.two_layer_workload(n, nrec=32)
    errs = {}
    for tb in (1, K):
        sim = sim_cls(wl["c_map"], lattice=5, tau=0.5, c_ref=wl["c_ref"], storage="bf16",
                      sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                      time_block=tb)
        sim.set_source(*wl["source"])
        sim.set_receivers(wl["receivers"], steps)
        sim.init_pressure(None)
        sim.step(steps)
        errs[tb] = (sim.pressure().cpu().numpy(), sim.traces(steps).cpu().numpy())
        sim.close()
    P = oracle_mod.Problem(5, n, n, wl["c_map"], c_ref=wl["c_ref"], tau=0.5,
                           sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                           source=wl["source"], receivers=wl["receivers"])
    g, tro = oracle_mod.run(P, P.zeros(), steps)
    po = oracle_mod.pressure(P, g)
    e1 = rel(errs[1][1], tro)
    eK = rel(errs[K][1], tro)
    assert eK < 4e-2 and rel(errs[K][0], po) < 4e-2
    assert eK < e1
