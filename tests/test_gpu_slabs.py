"""GPU: row-slab domain decomposition of one shot (lb_set_slab, lb_slab_step).

A grid split into row slabs must give exactly the whole grid's result: each slab runs the
same per-site arithmetic (the sponge is measured in the whole grid) and pulls across a
cut from halo rows holding the neighbour's cut rows.  So states, pressures and receiver
traces of 2, 3 and 4 slabs (even and uneven splits, source and receivers on cut rows) are
compared bit for bit with a single context, and with the FP64 oracle at the FP32 bound.
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W
from tests.traces import check_every_trace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300 import slabs
    from paper_1704_03172_gb300.sim import LBSim
    return LBSim, slabs


CASES = [  # Q, collision, storage, periodic, nx, ny, n_slabs, steps
    (5, "bgk", "f32", False, 130, 96, 2, 80),
    (5, "mrt", "f32", False, 257, 131, 3, 70),
    (5, "bgk", "bf16", False, 200, 77, 4, 60),
    (5, "bgk", "f32", True, 64, 60, 2, 50),
    (9, "mrt", "f32", False, 90, 70, 3, 40),
    (9, "bgk", "bf16", True, 72, 64, 4, 30),
    (5, "bgk", "f32", True, 40, 33, 1, 25),
]


@pytest.mark.parametrize("Q,coll,storage,periodic,nx,ny,n,steps", CASES)
def test_slabs_equal_the_whole_grid_bitwise(mods, oracle_mod, Q, coll, storage, periodic, nx, ny,
                                            n, steps):
    LBSim, slabs = mods
    rng = np.random.default_rng(nx + ny + n)
    c = W.random_medium(nx, ny, nx + n, 0.5, 1.0)
    bounds = slabs.partition(ny, n)
    cut = bounds[-1][0] if n > 1 else ny // 2
    s = ([1.0, 1.0, 1.0, 1.6, 1.3] if Q == 5 else [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3])
    kw = dict(lattice=Q, collision=coll, s=s if coll == "mrt" else None, tau=0.6, c_ref=1.0,
              storage=storage, boundary="periodic" if periodic else "zero",
              sponge_width=0 if periodic else 6, sponge_sigma_max=0.1, w_ref=(0.4, 0.11, 0.04))
    src = (nx // 3, cut - 1, rng.normal(size=steps))             # just below a cut
    rec = np.array([[5, cut - 1], [6, cut], [nx - 1, 0], [nx // 2, ny - 1], [7, cut],
                    [nx // 2, ny // 3]], np.int32)                # on and beside cut rows
    g0 = (rng.normal(size=(Q, ny, nx)) * 0.1).astype(np.float32)
    whole = LBSim(c, **kw)
    whole.set_source(*src)
    whole.set_receivers(rec, steps)
    whole.set_state(g0)
    whole.step(steps)
    ref = (whole.state().cpu().numpy(), whole.pressure().cpu().numpy(),
           whole.traces(steps).cpu().numpy())
    whole.close()
    grid = slabs.SlabGrid(c, n, **kw)
    grid.set_source(*src)
    grid.set_receivers(rec, steps)
    grid.set_state(g0)
    half = steps // 2
    grid.step(half)
    grid.step(steps - half)
    got = (grid.state(), grid.pressure(), grid.traces(steps))
    grid.close()
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    assert np.abs(ref[2]).max() > 0
    if storage == "f32":
        P = oracle_mod.Problem(Q, nx, ny, c, c_ref=1.0, periodic=periodic, mrt=coll == "mrt",
                               tau=0.6, s=s, w_ref=(0.4, 0.11, 0.04),
                               sponge_width=0 if periodic else 6, sponge_sigma_max=0.1,
                               source=src, receivers=rec)
        go, tro = oracle_mod.run(P, g0.astype(np.float64), steps)
        assert np.linalg.norm(got[0] - go) / np.linalg.norm(go) < 1e-5
        check_every_trace(got[2], tro, 1e-5)


def test_slabs_from_a_pressure_field_on_the_two_layer_workload(mods):
    # the two-layer workload at 512^2 in 4 slabs, from rest with the Ricker source: the
    # wavefront crosses three cuts; equal to the whole grid bit for bit
    LBSim, slabs = mods
    wl = W.two_layer_workload(512, nrec=64)
    steps = 600
    kw = dict(lattice=5, tau=0.5, c_ref=wl["c_ref"], sponge_width=wl["sponge_width"],
              sponge_sigma_max=wl["sponge_sigma_max"])
    out = []
    for n in (1, 4):
        if n == 1:
            sim = LBSim(wl["c_map"], **kw)
        else:
            sim = slabs.SlabGrid(wl["c_map"], n, **kw)
        sim.set_source(*wl["source"])
        sim.set_receivers(wl["receivers"], steps)
        sim.init_pressure(None)
        sim.step(steps)
        p = sim.pressure()
        tr = sim.traces(steps)
        out.append((np.asarray(p.cpu().numpy() if hasattr(p, "cpu") else p),
                    np.asarray(tr.cpu().numpy() if hasattr(tr, "cpu") else tr)))
        sim.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert np.abs(out[0][1]).max() > 0


def test_slab_refusals(mods):
    LBSim, slabs = mods
    from paper_1704_03172_gb300 import lbac
    c = W.uniform_map(64, 32, 1.0)
    sim = LBSim(c, c_ref=1.0, time_block=4)
    with pytest.raises(lbac.LBError):
        lbac.lb_set_slab(sim.ctx, 0, 64, None, None, None, None)   # time blocking
    sim.close()
    sim = LBSim(c, c_ref=1.0)
    with pytest.raises(lbac.LBError):
        lbac.lb_set_slab(sim.ctx, 40, 64, None, None, None, None)  # rows beyond the grid
    lbac.lb_set_slab(sim.ctx, 0, 64, None, None, None, None)
    with pytest.raises(lbac.LBError):
        sim.invariants()
    with pytest.raises(lbac.LBError):
        sim.checkpoint_every(10)
    sim.close()
