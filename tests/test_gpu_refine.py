"""GPU parity of the two-level grid refinement (Sec. 4) against the FP64 refinement oracle.

Same inputs on both sides; receivers outside the patch, inside it and on the
interface; pressure fields at several times (nodes of the closed patch come
from the fine grid).  Tolerance: relative L2 <= 1e-5 (FP32 GPU vs FP64).
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
    # Q, collision, tau, s, periodic, heterogeneous
    (5, "bgk", 0.5, None, False, False),
    (5, "mrt", 0.5, [1.3, 0.8, 0.8, 2.0, 2.0], False, True),
    (5, "mrt", 0.5, [1.0, 1.0, 1.0, 1.4, 1.7], True, True),     # s != 2: viscosity-continuous
    (5, "bgk", 0.8, None, False, True),                         # tau != 1/2: fine tau = 1.1
    (9, "bgk", 0.5, None, False, False),
    (9, "bgk", 0.7, None, True, True),
    (9, "mrt", 0.5, [1.0, 1.0, 1.0, 2.0, 2.0, 2.0, 1.0, 1.0, 2.0], False, True),
]


@pytest.mark.parametrize("Q,coll,tau,s,periodic,hetero", CASES)
def test_refined_matches_oracle(sim_cls, oracle_mod, Q, coll, tau, s, periodic, hetero):
    nx, ny, steps = 96, 80, 90
    c = W.random_medium(nx, ny, 21, 0.6, 1.0) if hetero else W.uniform_map(nx, ny, 1.0)
    patch = (40, 22, 30, 36)
    wav = W.ricker(steps, 0.06)
    rec = np.array([[20, 40], [40, 40], [52, 41], [70, 58], [69, 30], [85, 40], [55, 22]],
                   np.int32)                     # outside / on I / inside / corner
    w_ref = (0.4, 0.11, 0.04)
    kw = dict(tau=tau, s=s, w_ref=w_ref, c_ref=1.0)
    sponge = 0 if periodic else 8
    sim = sim_cls(c, lattice=Q, collision=coll, boundary="periodic" if periodic else "zero",
                  sponge_width=sponge, sponge_sigma_max=0.1, patch=patch, **kw)
    sim.set_source(15, 40, wav)
    sim.set_receivers(rec, steps)
    p0 = W.gaussian_pulse(nx, ny, 30, 50, 3.0, 1e-2).astype(np.float32)
    sim.init_pressure(p0)
    P = oracle_mod.Problem(Q, nx, ny, c, periodic=periodic, mrt=coll == "mrt",
                           sponge_width=sponge, sponge_sigma_max=0.1,
                           source=(15, 40, wav), receivers=rec, **kw)
    R = oracle_mod.Refined(P, *patch)
    R.init_pressure(p0.astype(np.float64))
    assert rel(sim.pressure().cpu().numpy(), R.pressure()) < TOL      # time 0
    traces = []
    for chunk in (1, 29, 60):
        sim.step(chunk)
        traces.append(R.run(chunk))
        assert rel(sim.pressure().cpu().numpy(), R.pressure()) < TOL
    tr = sim.traces().cpu().numpy()
    sim.close()
    assert rel(tr, np.concatenate(traces)) < TOL
    check_every_trace(tr, np.concatenate(traces), TOL)


def test_refined_block_workload_reduced_full_length(sim_cls, oracle_mod):
    # the slow-block refinement workload on a 256^2 coarse grid, all 4000 coarse steps
    wl = W.refined_block_workload(256, nrec=64)
    steps = wl["steps"]
    sim = sim_cls(wl["c_map"], lattice=5, collision="mrt", s=wl["s"], c_ref=wl["c_ref"],
                  sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                  patch=wl["patch"])
    sim.set_source(*wl["source"])
    sim.set_receivers(wl["receivers"], steps)
    sim.init_pressure(None)
    snap = 150
    sim.step(snap)
    ps = sim.pressure().cpu().numpy()
    sim.step(steps - snap)
    tr = sim.traces().cpu().numpy()
    sim.close()
    P = oracle_mod.Problem(5, 256, 256, wl["c_map"], c_ref=wl["c_ref"], mrt=True, s=wl["s"],
                           sponge_width=wl["sponge_width"],
                           sponge_sigma_max=wl["sponge_sigma_max"], source=wl["source"],
                           receivers=wl["receivers"])
    R = oracle_mod.Refined(P, *wl["patch"])
    R.init_pressure(None)
    t1 = R.run(snap)
    assert rel(ps, R.pressure()) < TOL
    t2 = R.run(steps - snap)
    assert rel(tr, np.concatenate([t1, t2])) < TOL
    check_every_trace(tr, np.concatenate([t1, t2]), TOL)


def test_refined_block_workload_full_size_truncated(sim_cls, oracle_mod):
    # 2048^2 coarse grid with the 1025^2-node fine patch, the launch path the benchmark
    # times, for 40 coarse steps from a smooth initial pulse that crosses the interface
    wl = W.refined_block_workload(2048)
    n, steps = 2048, 40
    p0 = W.gaussian_pulse(n, n, wl["patch"][0], 1024, 12.0, 1e-2).astype(np.float32)
    sim = sim_cls(wl["c_map"], lattice=5, collision="mrt", s=wl["s"], c_ref=wl["c_ref"],
                  sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                  patch=wl["patch"])
    sim.set_source(*wl["source"])
    sim.set_receivers(wl["receivers"], steps)
    sim.init_pressure(p0)
    sim.step(steps)
    ps = sim.pressure().cpu().numpy()
    tr = sim.traces().cpu().numpy()
    sim.close()
    P = oracle_mod.Problem(5, n, n, wl["c_map"], c_ref=wl["c_ref"], mrt=True, s=wl["s"],
                           sponge_width=wl["sponge_width"],
                           sponge_sigma_max=wl["sponge_sigma_max"], source=wl["source"],
                           receivers=wl["receivers"])
    R = oracle_mod.Refined(P, *wl["patch"])
    R.init_pressure(p0.astype(np.float64))
    tro = R.run(steps)
    assert rel(ps, R.pressure()) < TOL
    assert rel(tr, tro) < TOL
    check_every_trace(tr, tro, TOL)


def test_source_inside_patch_is_rejected(sim_cls):
    from paper_1704_03172_gb300 import lbac
    c = W.uniform_map(64, 64, 1.0)
    sim = sim_cls(c, lattice=5, c_ref=1.0, patch=(20, 20, 10, 10))
    with pytest.raises(lbac.LBError):
        sim.set_source(25, 25, [1.0, 2.0])
    sim.close()


# ---- nested patches (ratio 4 and 8 through levels of 2; "multiples of 2", Sec. 4)

NESTED = [
    # Q, collision, tau, s, periodic, heterogeneous, nested patches after the first
    (5, "bgk", 0.5, None, False, False, [(12, 14, 30, 36)]),
    (5, "mrt", 0.5, [1.0, 1.0, 1.0, 1.4, 1.7], False, True, [(12, 14, 30, 36)]),
    (5, "bgk", 0.8, None, True, True, [(12, 14, 30, 36)]),
    (9, "bgk", 0.7, None, False, True, [(12, 14, 30, 36)]),
    (9, "mrt", 0.5, [1.0, 1.0, 1.0, 2.0, 2.0, 2.0, 1.0, 1.0, 2.0], True, False, [(12, 14, 30, 36)]),
    (5, "mrt", 0.5, [1.3, 0.8, 0.8, 2.0, 2.0], False, True, [(12, 14, 30, 36), (10, 12, 20, 24)]),
]


@pytest.mark.parametrize("Q,coll,tau,s,periodic,hetero,inner", NESTED)
def test_nested_refined_matches_oracle(sim_cls, oracle_mod, Q, coll, tau, s, periodic, hetero,
                                       inner):
    nx, ny, steps = 96, 80, 60
    c = W.random_medium(nx, ny, 23, 0.6, 1.0) if hetero else W.uniform_map(nx, ny, 1.0)
    patch = (40, 22, 30, 36)
    wav = W.ricker(steps, 0.06)
    # outside / on the first interface / level 1 only / on the nested interface / inside the
    # nested patch / its corner / bottom edge of the first patch
    rec = np.array([[20, 40], [40, 40], [43, 41], [46, 35], [52, 38], [61, 47], [69, 30],
                    [85, 40], [55, 22], [50, 33]], np.int32)
    kw = dict(tau=tau, s=s, w_ref=(0.4, 0.11, 0.04), c_ref=1.0)
    sponge = 0 if periodic else 8
    sim = sim_cls(c, lattice=Q, collision=coll, boundary="periodic" if periodic else "zero",
                  sponge_width=sponge, sponge_sigma_max=0.1, patch=[patch] + inner, **kw)
    sim.set_source(15, 40, wav)
    sim.set_receivers(rec, steps)
    p0 = W.gaussian_pulse(nx, ny, 30, 50, 3.0, 1e-2).astype(np.float32)
    p0 += W.gaussian_pulse(nx, ny, 52, 40, 2.0, 5e-3).astype(np.float32)  # inside the nest
    sim.init_pressure(p0)
    P = oracle_mod.Problem(Q, nx, ny, c, periodic=periodic, mrt=coll == "mrt",
                           sponge_width=sponge, sponge_sigma_max=0.1,
                           source=(15, 40, wav), receivers=rec, **kw)
    R = oracle_mod.Refined(P, *patch)
    for q in inner:
        R.nest(*q)
    R.init_pressure(p0.astype(np.float64))
    assert rel(sim.pressure().cpu().numpy(), R.pressure()) < TOL      # time 0
    traces = []
    for chunk in (1, 1, 18, 40):
        sim.step(chunk)
        traces.append(R.run(chunk))
        assert rel(sim.pressure().cpu().numpy(), R.pressure()) < TOL
    tr = sim.traces().cpu().numpy()
    sim.close()
    ref = np.concatenate(traces)
    assert rel(tr, ref) < TOL
    check_every_trace(tr, ref, TOL)
    for j in range(len(rec)):                    # every receiver, each from its own level
        assert np.linalg.norm(tr[:, j] - ref[:, j]) <= 1e-4 * np.linalg.norm(ref[:, j]) + 1e-9


def test_nested_patch_placement_is_checked(sim_cls):
    c = W.uniform_map(64, 48, 1.0)
    with pytest.raises(Exception):     # touches the edge of the level-1 grid
        sim_cls(c, patch=[(20, 10, 16, 20), (0, 4, 10, 10)])
    with pytest.raises(Exception):     # reaches past it
        sim_cls(c, patch=[(20, 10, 16, 20), (20, 4, 12, 10)])
    with pytest.raises(Exception):     # more than LB_MAX_PATCHES
        sim_cls(c, patch=[(20, 10, 16, 20)] + [(4, 4, 8, 8)] * 3)
    sim = sim_cls(c, patch=[(20, 10, 16, 20), (4, 4, 20, 30)])
    sim.close()


def test_nested_block_workload_reduced_full_length(sim_cls, oracle_mod):
    # the nested slow-block workload on a 256^2 coarse grid, all 4000 coarse steps
    # (16000 steps of the nested level)
    wl = W.refined_nested_workload(256, nrec=64)
    steps = wl["steps"]
    sim = sim_cls(wl["c_map"], lattice=5, collision="mrt", s=wl["s"], c_ref=wl["c_ref"],
                  sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                  patch=wl["patches"])
    sim.set_source(*wl["source"])
    sim.set_receivers(wl["receivers"], steps)
    sim.init_pressure(None)
    snap = 150
    sim.step(snap)
    ps = sim.pressure().cpu().numpy()
    sim.step(steps - snap)
    tr = sim.traces().cpu().numpy()
    sim.close()
    P = oracle_mod.Problem(5, 256, 256, wl["c_map"], c_ref=wl["c_ref"], mrt=True, s=wl["s"],
                           sponge_width=wl["sponge_width"],
                           sponge_sigma_max=wl["sponge_sigma_max"], source=wl["source"],
                           receivers=wl["receivers"])
    R = oracle_mod.Refined(P, *wl["patches"][0])
    R.nest(*wl["patches"][1])
    R.init_pressure(None)
    t1 = R.run(snap)
    assert rel(ps, R.pressure()) < TOL
    t2 = R.run(steps - snap)
    assert rel(tr, np.concatenate([t1, t2])) < TOL
    check_every_trace(tr, np.concatenate([t1, t2]), TOL)


def test_footprint_covers_refined_levels(sim_cls):
    # lb_footprint counts the patch levels: it bounds what lb_create and lb_set_receivers
    # take from the (PyTorch) allocator, without overstating it by much
    import torch
    from paper_1704_03172_gb300 import lbac
    nx, ny = 400, 300
    c = W.uniform_map(nx, ny, 1.0)
    patches = [(100, 80, 150, 120), (40, 30, 200, 150)]
    rec = np.array([[20, 20], [150, 140], [180, 150]], np.int32)
    for plist in (patches[:1], patches):
        cfg = lbac.lb_config_default()
        cfg.nx, cfg.ny = nx, ny
        arr = (lbac.lb_patch * len(plist))(*[lbac.lb_patch(*q, 2) for q in plist])
        cfg.patches = ctypes_cast(arr, lbac)
        cfg.n_patches = len(plist)
        est = lbac.lb_footprint(cfg, 50, len(rec), 0)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        sim = sim_cls(c, patch=plist)
        sim.set_receivers(rec, 50)
        torch.cuda.synchronize()
        used = torch.cuda.memory_allocated() - before
        sim.close()
        # (the allocator rounds each small buffer up to 512 bytes)
        assert used <= est + (64 << 10) and est <= 1.3 * used + (4 << 20), (len(plist), used, est)


def ctypes_cast(arr, lbac):
    import ctypes
    return ctypes.cast(arr, ctypes.POINTER(lbac.lb_patch))


ONE_WAY = [
    # Q, collision, tau, s, periodic, heterogeneous, coupling
    (5, "bgk", 0.5, None, False, True, "c2f"),
    (5, "bgk", 0.5, None, False, True, "f2c"),
    (5, "mrt", 0.5, [1.0, 1.0, 1.0, 1.4, 1.7], True, True, "f2c"),
    (9, "bgk", 0.7, None, False, True, "c2f"),
    (9, "mrt", 0.5, [1.0, 1.0, 1.0, 2.0, 2.0, 2.0, 1.0, 1.0, 2.0], True, False, "f2c"),
]


@pytest.mark.parametrize("Q,coll,tau,s,periodic,hetero,coupling", ONE_WAY)
def test_one_way_coupling_matches_oracle(sim_cls, oracle_mod, Q, coll, tau, s, periodic, hetero,
                                         coupling):
    # the paper's switch on the direction of propagation (Sec. 4): coarse -> fine only, or
    # fine -> coarse only (nothing enters the patch)
    nx, ny, steps = 96, 80, 70
    c = W.random_medium(nx, ny, 24, 0.6, 1.0) if hetero else W.uniform_map(nx, ny, 1.0)
    patch = (40, 22, 30, 36)
    wav = W.ricker(steps, 0.06)
    rec = np.array([[20, 40], [40, 40], [52, 41], [70, 58], [69, 30], [85, 40]], np.int32)
    kw = dict(tau=tau, s=s, w_ref=(0.4, 0.11, 0.04), c_ref=1.0)
    sponge = 0 if periodic else 8
    sim = sim_cls(c, lattice=Q, collision=coll, boundary="periodic" if periodic else "zero",
                  sponge_width=sponge, sponge_sigma_max=0.1, patch=patch, coupling=coupling, **kw)
    sim.set_source(15, 40, wav)
    sim.set_receivers(rec, steps)
    p0 = W.gaussian_pulse(nx, ny, 30, 50, 3.0, 1e-2).astype(np.float32)
    p0 += W.gaussian_pulse(nx, ny, 55, 40, 2.5, 5e-3).astype(np.float32)   # inside the patch
    sim.init_pressure(p0)
    P = oracle_mod.Problem(Q, nx, ny, c, periodic=periodic, mrt=coll == "mrt",
                           sponge_width=sponge, sponge_sigma_max=0.1,
                           source=(15, 40, wav), receivers=rec, **kw)
    R = oracle_mod.Refined(P, *patch)
    R.direction(coupling)
    R.init_pressure(p0.astype(np.float64))
    assert rel(sim.pressure().cpu().numpy(), R.pressure()) < TOL
    traces = []
    for chunk in (1, 29, 40):
        sim.step(chunk)
        traces.append(R.run(chunk))
        assert rel(sim.pressure().cpu().numpy(), R.pressure()) < TOL
    tr = sim.traces().cpu().numpy()
    sim.close()
    assert rel(tr, np.concatenate(traces)) < TOL
    check_every_trace(tr, np.concatenate(traces), TOL)


@pytest.mark.parametrize("modes", [("c2f", "f2c"), ("f2c", "both"), ("both", "c2f")])
def test_nested_one_way_coupling_matches_oracle(sim_cls, oracle_mod, modes):
    nx, ny, steps = 96, 80, 40
    c = W.random_medium(nx, ny, 25, 0.6, 1.0)
    patch, inner = (40, 22, 30, 36), (8, 14, 30, 30)
    wav = W.ricker(steps, 0.06)
    rec = np.array([[20, 40], [43, 41], [52, 38], [61, 47], [69, 30]], np.int32)
    kw = dict(tau=0.5, w_ref=(0.4, 0.11, 0.04), c_ref=1.0)
    sim = sim_cls(c, lattice=5, sponge_width=8, sponge_sigma_max=0.1, patch=[patch, inner],
                  coupling=list(modes), **kw)
    sim.set_source(15, 40, wav)
    sim.set_receivers(rec, steps)
    p0 = W.gaussian_pulse(nx, ny, 30, 50, 3.0, 1e-2).astype(np.float32)
    p0 += W.gaussian_pulse(nx, ny, 52, 40, 2.0, 5e-3).astype(np.float32)
    sim.init_pressure(p0)
    P = oracle_mod.Problem(5, nx, ny, c, sponge_width=8, sponge_sigma_max=0.1,
                           source=(15, 40, wav), receivers=rec, **kw)
    R = oracle_mod.Refined(P, *patch)
    R.nest(*inner)
    R.direction(modes[0], level=1)
    R.direction(modes[1], level=2)
    R.init_pressure(p0.astype(np.float64))
    traces = []
    for chunk in (1, 19, 20):
        sim.step(chunk)
        traces.append(R.run(chunk))
        assert rel(sim.pressure().cpu().numpy(), R.pressure()) < TOL
    tr = sim.traces().cpu().numpy()
    sim.close()
    assert rel(tr, np.concatenate(traces)) < TOL
    check_every_trace(tr, np.concatenate(traces), TOL)


def test_coupling_mode_is_checked(sim_cls):
    c = W.uniform_map(64, 48, 1.0)
    with pytest.raises(ValueError):
        sim_cls(c, lattice=5, c_ref=1.0, patch=(10, 10, 20, 20), coupling="sideways")
    with pytest.raises(ValueError):  # one value per patch
        sim_cls(c, lattice=5, c_ref=1.0, patch=[(10, 10, 20, 20), (4, 4, 8, 8)],
                coupling=["c2f"])
