"""GPU parity of the three-dimensional (D3Q7) step against the FP64 3-D oracle.

The 3-D grid is stored as nz * ny rows of the 2-D layout; the step kernel pulls along x by
warp shuffles and along y and z by reading other rows.  Every case starts from an arbitrary
state (read in place by the first step), runs a source, receivers and, without periodicity,
a zero ghost and a sponge.  Tolerance: FP32 relative L2 <= 1e-5 on the state and the traces;
16-bit storage against the same bounds as in 2-D (BF16 4e-2, FP16 5e-3).
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W

pytestmark = pytest.mark.gpu
BOUND = {"f32": 1e-5, "f16": 5e-3, "bf16": 4e-2}


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


def _layered3(nx, ny, nz):
    """Few distinct speeds (the 1-byte medium index applies): layers along z."""
    c = np.empty((nz, ny, nx), np.float32)
    for z in range(nz):
        c[z] = 0.5 + 0.5 * ((z * 5) // nz) / 4
    return c


@pytest.mark.parametrize("storage,periodic,nx,ny,nz,layered,tau", [
    ("f32", True, 37, 20, 11, False, 0.5),
    ("f32", False, 70, 33, 17, False, 0.7),
    ("f32", False, 130, 9, 14, True, 0.5),
    ("bf16", False, 64, 24, 20, True, 0.5),
    ("f16", True, 40, 16, 12, False, 0.6),
])
def test_d3q7_matches_oracle(sim_cls, oracle_mod, storage, periodic, nx, ny, nz, layered, tau):
    rng = np.random.default_rng(nx + ny + nz)
    c = (_layered3(nx, ny, nz) if layered
         else rng.uniform(0.45, 1.0, size=(nz, ny, nx)).astype(np.float32))
    steps = 40
    g0 = (rng.normal(size=(7, nz, ny, nx)) * 0.05).astype(np.float32)
    if storage != "f32":  # a state the 16-bit forms hold exactly: only the steps round
        g0 = (np.round(g0 * 256) / 256).astype(np.float32)
    src = (nx // 3, ny // 2, nz // 2, W.ricker(steps, 0.06))
    rec = np.stack([rng.integers(0, nx, 10), rng.integers(0, ny, 10), rng.integers(0, nz, 10)],
                   1).astype(np.int32)
    sponge = 0 if periodic else 3
    sim = sim_cls(c, lattice=7, tau=tau, storage=storage, c_ref=1.0,
                  boundary="periodic" if periodic else "zero", sponge_width=sponge,
                  sponge_sigma_max=0.15)
    sim.set_source(*src)
    sim.set_receivers(rec, steps)
    sim.set_state(g0)
    sim.step(steps)
    gs = sim.state().cpu().numpy()
    tr = sim.traces(steps).cpu().numpy()
    ps = sim.pressure().cpu().numpy()
    info = sim.info()
    sim.close()
    assert info[0] == 7 and (info[4] > 0) == layered
    P = oracle_mod.Problem3(nx, ny, nz, c, c_ref=1.0, periodic=periodic, tau=tau,
                            sponge_width=sponge, sponge_sigma_max=0.15, source=src, receivers=rec)
    go, tro = oracle_mod.run3(P, g0.astype(np.float64), steps)
    assert rel(gs, go) < BOUND[storage]
    assert rel(tr, tro) < BOUND[storage]
    assert rel(ps, oracle_mod.pressure3(P, go)) < BOUND[storage]


def test_d3q7_rejects_2d_only_features(sim_cls):
    from paper_1704_03172_gb300 import lbac
    c = np.ones((6, 8, 8), np.float32)
    with pytest.raises(lbac.LBError):
        sim_cls(c, lattice=7, collision="mrt", s=[1.0] * 7, c_ref=1.0)
    sim = sim_cls(c, lattice=7, c_ref=1.0)
    with pytest.raises(lbac.LBError):
        sim.checkpoint_every(10)
    with pytest.raises(lbac.LBError):
        sim.invariants()
    with pytest.raises(lbac.LBError):          # 2-D source call on a 3-D context
        lbac.lb_set_source(sim.ctx, 1, 1, None, 0)
    sim.close()


@pytest.mark.parametrize("storage,periodic,nx,ny,nz", [
    ("bf16", False, 2100, 6, 5),      # two row segments per row, the second ragged
    ("f32", True, 2100, 6, 5),
    ("f16", False, 2100, 6, 5),
    ("bf16", False, 256, 20, 9),      # narrow rows: one segment covers a whole row
    ("bf16", True, 200, 13, 7),       # pitch 224, periodic wraps in y and z
    ("f16", True, 96, 10, 6),
    ("f32", False, 160, 11, 5),
])
def test_d3q7_staged_step_matches_direct_bitwise(sim_cls, storage, periodic, nx, ny, nz):
    rng = np.random.default_rng(5)
    steps = 12
    c = rng.uniform(0.45, 1.0, size=(nz, ny, nx)).astype(np.float32)
    g0 = (np.round(rng.normal(size=(7, nz, ny, nx)) * 0.05 * 256) / 256).astype(np.float32)
    rec = np.stack([rng.integers(0, nx, 8), rng.integers(0, ny, 8), rng.integers(0, nz, 8)],
                   1).astype(np.int32)
    out = []
    for kernel in ("staged", "direct"):
        sim = sim_cls(c, lattice=7, tau=0.6, storage=storage, c_ref=1.0, step_kernel=kernel,
                      boundary="periodic" if periodic else "zero",
                      sponge_width=0 if periodic else 2)
        sim.set_source(nx // 2, 3, 2, W.ricker(steps, 0.05))
        sim.set_receivers(rec, steps)
        sim.set_state(g0)
        sim.step(steps)
        out.append((sim.state().cpu().numpy(), sim.traces(steps).cpu().numpy()))
        sim.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
