"""GPU tests of in-place streaming (LB_STREAM_AA: one population buffer).

The in-place steps alternate a site-local update and a neighbour exchange, but the per-site
arithmetic is the two-buffer step's, so traces, pressure, populations, invariants and mode
projections must equal the two-buffer context's bit for bit after any number of steps
(odd and even), for both lattices, both collisions, both boundaries and both storage types,
on ragged grids with receivers on the domain's edges.  Against the FP64 oracle the FP32
results keep the FP32 tolerance, and the context holds one population buffer.
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W
from tests.traces import check_every_trace

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300 import lbac
    from paper_1704_03172_gb300.sim import LBSim
    return LBSim, lbac


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


MRT5 = [1.0, 1.0, 1.0, 1.3, 1.7]
MRT9 = [1.0, 1.0, 1.0, 1.7, 1.4, 1.6, 1.2, 1.2, 1.4]
CASES = [
    # Q, collision, storage, periodic, nx, ny
    (5, "bgk", "f32", False, 300, 77),
    (5, "mrt", "f32", True, 257, 64),
    (5, "bgk", "bf16", False, 129, 130),
    (5, "bgk", "bf16", True, 64, 33),
    (9, "bgk", "f32", False, 200, 51),
    (9, "mrt", "f32", True, 96, 96),
    (9, "mrt", "bf16", False, 513, 40),
    (5, "mrt", "f32", False, 1, 70),      # one column: every site on two faces
    # rows wide enough for warps with no site on a face (the exchange step's interior form:
    # 128 FP32 / 256 16-bit sites a warp)
    (9, "bgk", "f32", True, 400, 40),
    (9, "mrt", "f32", False, 390, 20),
    (5, "mrt", "bf16", True, 700, 24),
    # BF16 rows of >= 1024 sites take the TMA-staged kernel in both forms (2048-site tasks;
    # ragged last tasks)
    (5, "bgk", "bf16", False, 1100, 40),
    (5, "mrt", "bf16", True, 2100, 20),
    (9, "bgk", "bf16", False, 4200, 12),
    (9, "mrt", "bf16", True, 1024, 16),
]


def _pair(LBSim, Q, coll, storage, periodic, nx, ny, seed):
    rng = np.random.default_rng(seed)
    c = W.random_medium(nx, ny, 5, 0.5, 1.0)
    kw = dict(lattice=Q, collision=coll, storage=storage,
              s=(MRT5 if Q == 5 else MRT9) if coll == "mrt" else None,
              tau=0.5 if coll == "bgk" else 1.0, w_ref=(0.4, 0.11, 0.04), c_ref=1.0,
              boundary="periodic" if periodic else "zero",
              sponge_width=0 if periodic else 6, sponge_sigma_max=0.1)
    src = (nx // 3, ny // 2, rng.normal(size=200))
    # receivers on the four faces, the corners, the source, and two at one site
    rec = [(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0), (nx // 2, 0), (nx // 2, ny - 1),
           (0, ny // 2), (nx - 1, ny // 2), (nx // 3, ny // 2), (nx // 3, ny // 2)]
    rec += [tuple(v) for v in np.stack([rng.integers(0, nx, 12), rng.integers(0, ny, 12)], 1)]
    rec = np.asarray(rec, np.int32)
    sims = []
    for streaming in ("ab", "aa"):
        s = LBSim(c, streaming=streaming, **kw)
        s.set_source(*src)
        s.set_receivers(rec, 200)
        sims.append(s)
    return sims, c, kw, src, rec


def _same(ab, aa):
    np.testing.assert_array_equal(aa.pressure().cpu().numpy(), ab.pressure().cpu().numpy())
    np.testing.assert_array_equal(aa.state().cpu().numpy(), ab.state().cpu().numpy())
    np.testing.assert_array_equal(aa.traces().cpu().numpy(), ab.traces().cpu().numpy())


@pytest.mark.parametrize("Q,coll,storage,periodic,nx,ny", CASES)
def test_in_place_equals_two_buffers_bitwise(mods, Q, coll, storage, periodic, nx, ny):
    LBSim, lbac = mods
    (ab, aa), _, _, _, _ = _pair(LBSim, Q, coll, storage, periodic, nx, ny, nx * 7 + ny)
    staged = storage == "bf16" and nx >= 1024   # the TMA-staged kernel (info[5]) in both
    assert aa.info()[5] == ab.info()[5] == (1.0 if staged else 0.0)
    rng = np.random.default_rng(3)
    g0 = (rng.normal(size=(Q, ny, nx)) * 1e-2).astype(np.float32)
    for s in (ab, aa):
        s.set_state(g0)
    _same(ab, aa)                     # the state as written
    for n in (1, 36, 1, 2, 17):       # odd and even totals: both forms of the buffer
        ab.step(n)
        aa.step(n)
        _same(ab, aa)
    assert aa.time == ab.time == 57
    inv_ab, inv_aa = ab.invariants(), aa.invariants()
    assert list(inv_aa) == list(inv_ab)
    if nx > 1:
        modes = [(1, 0), (0, 1), (2, 3)]
        assert lbac.lb_mode_projection(aa.ctx, modes) == lbac.lb_mode_projection(ab.ctx, modes)
    # a new state in the middle of a run, after an odd number of steps (swapped form)
    aa.step(1)
    ab.step(1)
    for s in (ab, aa):
        s.set_state(g0 * 0.5)
        s.step(3)
    _same(ab, aa)
    ab.close()
    aa.close()


@pytest.mark.parametrize("Q,coll,periodic", [(5, "bgk", False), (5, "mrt", True),
                                             (9, "mrt", False)])
def test_in_place_matches_oracle(mods, oracle_mod, Q, coll, periodic):
    LBSim, _ = mods
    nx, ny, steps = 140, 90, 61
    (ab, aa), c, kw, src, rec = _pair(LBSim, Q, coll, "f32", periodic, nx, ny, 11)
    ab.close()
    rng = np.random.default_rng(5)
    g0 = rng.normal(size=(Q, ny, nx)).astype(np.float32)
    aa.set_state(g0)
    aa.step(steps)
    gs = aa.state().cpu().numpy()
    tr = aa.traces().cpu().numpy()
    aa.close()
    P = oracle_mod.Problem(Q, nx, ny, c, periodic=periodic, mrt=coll == "mrt",
                           sponge_width=kw["sponge_width"], sponge_sigma_max=0.1, source=src,
                           receivers=rec, tau=kw["tau"], s=kw["s"], w_ref=kw["w_ref"],
                           c_ref=1.0)
    go, tro = oracle_mod.run(P, g0.astype(np.float64), steps)
    assert rel(gs, go) < TOL
    assert rel(tr, tro) < TOL
    check_every_trace(tr, tro, TOL)


def test_in_place_from_pressure_two_layer(mods):
    # the bench's two-layer medium (1-byte medium index), started from lb_init_pressure
    LBSim, _ = mods
    n = 512
    c = W.two_layer(n, n, 1.0, 2.0)
    out = []
    for streaming in ("ab", "aa"):
        s = LBSim(c, lattice=5, tau=0.5, sponge_width=40, sponge_sigma_max=0.1,
                  streaming=streaming)
        s.set_source(n // 2, n // 4, W.ricker(400, 1.0 / 30))
        s.set_receivers(W.line_receivers(64, n // 4, 0, n - 1), 400)
        s.init_pressure(None)
        assert s.info()[4] == 2     # two speeds behind the medium index
        s.step(333)
        out.append((s.traces().cpu().numpy(), s.pressure().cpu().numpy()))
        s.close()
    np.testing.assert_array_equal(out[1][0], out[0][0])
    np.testing.assert_array_equal(out[1][1], out[0][1])


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_in_place_4096_bench_configuration(mods, storage):
    # the bench's in-place lines: the 4096^2 two-layer workload with its sponge, source and
    # receiver line (BF16 on the TMA-staged kernel), both forms of the step, against the
    # two-buffer step bit for bit
    LBSim, _ = mods
    n = 4096
    c = W.two_layer(n, n, 1.0, 2.0)
    out = []
    for streaming in ("ab", "aa"):
        s = LBSim(c, lattice=5, tau=0.5, sponge_width=40, sponge_sigma_max=0.1,
                  storage=storage, streaming=streaming)
        s.set_source(n // 2, n // 4, W.ricker(64, 1.0 / 30))
        s.set_receivers(W.line_receivers(512, n // 4 + 3, 0, n - 1), 64)
        s.init_pressure(None)
        assert s.info()[5] == (1.0 if storage == "bf16" else 0.0)
        s.step(7)                     # 4 site-local and 3 exchange steps in place
        out.append((s.traces().cpu().numpy(), s.pressure().cpu().numpy(),
                    s.state().cpu().numpy()))
        s.close()
    for a, b in zip(out[1], out[0]):
        np.testing.assert_array_equal(a, b)
    assert np.abs(out[0][0]).max() > 0   # the source reached the receiver line


def test_in_place_holds_one_population_buffer(mods):
    import torch
    LBSim, lbac = mods
    n = 1024
    c = np.ones((n, n), np.float32)
    used = {}
    for streaming in ("ab", "aa"):
        torch.cuda.synchronize()
        m0 = torch.cuda.memory_allocated()
        s = LBSim(c, lattice=9, streaming=streaming)
        torch.cuda.synchronize()
        used[streaming] = torch.cuda.memory_allocated() - m0
        s.close()
    buf = 9 * n * n * 4
    assert used["ab"] - used["aa"] == buf, used
    assert used["aa"] < buf * 1.2


def test_in_place_refuses_checkpoints_tape_and_slabs(mods):
    LBSim, lbac = mods
    s = LBSim(np.ones((32, 32), np.float32), streaming="aa")
    for call in (lambda: s.checkpoint_every(8), lambda: s.record_rho(8),
                 lambda: s.adjoint(np.zeros((4, 0), np.float32), 4)):
        with pytest.raises(lbac.LBError) as e:
            call()
        assert e.value.status == lbac.LB_ESTATE
        assert "LB_STREAM_AA" in lbac.lb_last_error(s.ctx)
    with pytest.raises(lbac.LBError) as e:
        lbac.lb_set_slab(s.ctx, 0, 64, None, None, None, None)
    assert e.value.status == lbac.LB_ESTATE
    s.close()


def test_in_place_stability_watch(mods):
    # the watch reads the invariants of either form of the buffer
    LBSim, lbac = mods
    n = 64
    s = LBSim(W.uniform_map(n, n, 0.8), lattice=5, c_ref=1.0, boundary="periodic",
              streaming="aa")
    rng = np.random.default_rng(2)
    s.set_state(rng.normal(size=(5, n, n)).astype(np.float32) * 1e-3)
    lbac.lb_watch_stability(s.ctx, 7, 1.0001)
    s.step(99)        # lossless, source-free: the energy stays put at odd and even checks
    assert s.time == 99
    s.close()
