"""GPU discrete adjoint (lb_adjoint, checkpointed) against the FP64 adjoint oracle and
against finite differences of the FP64 forward oracle.

Tolerance: relative L2 <= 1e-4 for the FP32 GPU gradients (they accumulate over
all steps), 1e-5 for the FP32 dot-product identity.
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


CASES = [
    # Q, collision, tau, s, periodic, sponge, checkpoint_every
    (5, "bgk", 0.5, None, False, 6, 7),
    (5, "mrt", 0.5, [1.2, 0.9, 0.9, 1.6, 1.3], False, 5, 16),
    (5, "bgk", 0.8, None, True, 0, 40),
    (9, "mrt", 0.5, [1.0, 1.0, 1.0, 1.7, 1.4, 1.6, 1.2, 1.2, 1.4], False, 5, 9),
    (9, "bgk", 0.7, None, True, 0, 1),
]


def _setup(seed, nx=70, ny=45, nt=40):
    rng = np.random.default_rng(seed)
    c = W.random_medium(nx, ny, seed, 0.5, 1.0)
    rec = np.stack([rng.integers(0, nx, 9), rng.integers(0, ny, 9)], 1).astype(np.int32)
    src = (int(rng.integers(8, nx - 8)), int(rng.integers(8, ny - 8)), rng.normal(size=nt))
    return rng, c, src, rec


def _both(sim_cls, oracle, case, c, src, rec, nt, storage="f32"):
    Q, coll, tau, s, per, sponge, every = case
    ny, nx = c.shape
    kw = dict(tau=tau, s=s, w_ref=(0.4, 0.11, 0.04), c_ref=1.0)
    sim = sim_cls(c, lattice=Q, collision=coll, boundary="periodic" if per else "zero",
                  sponge_width=sponge, sponge_sigma_max=0.15, storage=storage, **kw)
    sim.set_source(*src)
    sim.set_receivers(rec, nt)
    P = oracle.Problem(Q, nx, ny, c, periodic=per, mrt=coll == "mrt", sponge_width=sponge,
                       sponge_sigma_max=0.15, source=src, receivers=rec, **kw)
    return sim, P


@pytest.mark.parametrize("case", CASES)
def test_adjoint_matches_oracle(sim_cls, oracle_mod, case):
    Q, every = case[0], case[-1]
    rng, c, src, rec = _setup(11)
    nt = 40
    sim, P = _both(sim_cls, oracle_mod, case, c, src, rec, nt)
    g0 = (rng.normal(size=(Q,) + c.shape) * 0.1).astype(np.float32)
    sim.set_state(g0)
    sim.checkpoint_every(every)
    sim.step(nt)
    tr = sim.traces(nt).cpu().numpy()
    d = rng.normal(size=tr.shape).astype(np.float32)
    R = tr - d
    gc, gs, gg = sim.adjoint(R, nt, want_g0=True)
    gc, gs, gg = gc.cpu().numpy(), gs.cpu().numpy(), gg.cpu().numpy()
    sim.close()
    oc, os_, og = oracle_mod.adjoint(P, g0.astype(np.float64), nt, R.astype(np.float64))
    assert rel(gc, oc) < TOL
    assert rel(gs, os_) < TOL
    assert rel(gg, og) < TOL


# BF16 storage: the adjoint state is FP32 and only the replayed forward states are
# BF16.  dJ/dS depends on the adjoint state alone, so it keeps the FP32 bound;
# dJ/dc also weighs the BF16 densities rho^t and carries their rounding error
# (bounded here like the BF16 forward fields, 4e-2 relative).
BF16_GRAD_C_TOL = 4e-2


@pytest.mark.parametrize("case", [CASES[1], CASES[3]])
def test_bf16_storage_adjoint(sim_cls, oracle_mod, case):
    Q, every = case[0], case[-1]
    rng, c, src, rec = _setup(15, nt=60)
    nt = 60
    _, P = _both(sim_cls, oracle_mod, case, c, src, rec, nt)
    _, tro = oracle_mod.run(P, P.zeros(), nt)
    R = (tro - rng.normal(size=tro.shape) * 1e-3).astype(np.float32)
    oc, os_, _ = oracle_mod.adjoint(P, P.zeros(), nt, R.astype(np.float64))
    out = {}
    for st in ("f32", "bf16"):
        sim, _ = _both(sim_cls, oracle_mod, case, c, src, rec, nt, storage=st)
        sim.init_pressure(None)
        sim.checkpoint_every(every)
        sim.step(nt)
        gc, gs, _ = sim.adjoint(R, nt)
        out[st] = (gc.cpu().numpy(), gs.cpu().numpy())
        sim.close()
    assert rel(out["f32"][0], oc) < TOL
    assert rel(out["bf16"][1], os_) < TOL
    e = rel(out["bf16"][0], oc)
    print(f"BF16-storage dJ/dc vs FP64 oracle: rel L2 {e:.2e} (D2Q{Q} {case[1]})")
    assert e < BF16_GRAD_C_TOL
    assert rel(out["bf16"][0], out["f32"][0]) < BF16_GRAD_C_TOL


def test_fp16_storage_adjoint_is_refused(sim_cls):
    from paper_1704_03172_gb300 import lbac
    c = W.uniform_map(64, 64)
    sim = sim_cls(c, lattice=5, storage="f16", c_ref=1.0)
    with pytest.raises(lbac.LBError) as e:
        sim.checkpoint_every(10)
    assert e.value.status == lbac.LB_ESTATE
    sim.close()


def test_adjoint_dot_product_on_gpu(sim_cls, oracle_mod):
    case = CASES[1]
    rng, c, src, rec = _setup(12)
    nt = 40
    zero_src = (src[0], src[1], np.zeros(nt))
    sim, _ = _both(sim_cls, oracle_mod, case, c, zero_src, rec, nt)
    g0 = rng.normal(size=(5,) + c.shape).astype(np.float32)
    sim.set_state(g0)
    sim.checkpoint_every(10)
    sim.step(nt)
    tr = sim.traces(nt).cpu().numpy().astype(np.float64)
    R = rng.normal(size=tr.shape).astype(np.float32)
    _, _, gg = sim.adjoint(R, nt, want_g0=True)
    sim.close()
    lhs = (tr * R).sum()
    rhs = (g0.astype(np.float64) * gg.cpu().numpy()).sum()
    assert abs(lhs - rhs) <= 1e-5 * np.abs(tr * R).sum()


def test_adjoint_matches_finite_differences(sim_cls, oracle_mod):
    # dJ/dc from the GPU adjoint vs Richardson-extrapolated central differences of the
    # FP64 forward oracle, J = 1/2 sum (p - d)^2
    case = CASES[0]
    rng, c, src, rec = _setup(13, nx=40, ny=32, nt=30)
    nt = 30
    sim, P = _both(sim_cls, oracle_mod, case, c, src, rec, nt)
    d = rng.normal(size=(nt, len(rec))) * 0.05
    sim.init_pressure(None)
    sim.checkpoint_every(8)
    sim.step(nt)
    tr = sim.traces(nt).cpu().numpy()
    gc, gs, _ = sim.adjoint((tr - d).astype(np.float32), nt)
    gc = gc.cpu().numpy()
    sim.close()

    def J(cm):
        Pm = oracle_mod.Problem(5, 40, 32, cm, c_ref=1.0, tau=0.5, sponge_width=6,
                                sponge_sigma_max=0.15, source=src, receivers=rec)
        _, t = oracle_mod.run(Pm, Pm.zeros(), nt)
        return 0.5 * ((t - d) ** 2).sum()

    def central(y, x, h):
        cp, cm = c.copy(), c.copy()
        cp[y, x] = np.float32(c[y, x] + h)
        cm[y, x] = np.float32(c[y, x] - h)
        return (J(cp) - J(cm)) / (float(cp[y, x]) - float(cm[y, x]))

    sites = [(src[1], src[0]), (rec[0, 1], rec[0, 0])] + \
        [(int(rng.integers(32)), int(rng.integers(40))) for _ in range(6)]
    for (y, x) in sites:
        fd = (4 * central(y, x, 1e-4) - central(y, x, 2e-4)) / 3
        assert abs(fd - gc[y, x]) <= TOL * max(abs(fd), 1e-2 * np.abs(gc).max())


def test_autograd_function_matches_adjoint(sim_cls, oracle_mod):
    import torch
    from paper_1704_03172_gb300.sim import LBForward
    rng, c, src, rec = _setup(14, nt=50)
    nt = 50
    spec = dict(lattice=5, collision="bgk", tau=0.5, c_ref=1.0, sponge_width=6,
                sponge_sigma_max=0.15, source_xy=(src[0], src[1]), receivers=rec, nt=nt,
                checkpoint_every=12)
    cm = torch.tensor(c, device="cuda", requires_grad=True)
    wav = torch.tensor(src[2], device="cuda", dtype=torch.float64, requires_grad=True)
    d = torch.tensor(rng.normal(size=(nt, len(rec))) * 0.05, device="cuda", dtype=torch.float32)
    tr = LBForward.apply(cm, wav, spec)
    loss = 0.5 * ((tr - d) ** 2).sum()
    loss.backward()
    P = oracle_mod.Problem(5, c.shape[1], c.shape[0], c, c_ref=1.0, tau=0.5, sponge_width=6,
                           sponge_sigma_max=0.15, source=src, receivers=rec)
    _, tro = oracle_mod.run(P, P.zeros(), nt)
    oc, os_, _ = oracle_mod.adjoint(P, P.zeros(), nt, tro - d.cpu().numpy())
    assert rel(cm.grad.cpu().numpy(), oc) < TOL
    assert rel(wav.grad.cpu().numpy(), os_) < TOL


def test_layered_model_adjoint_with_long_checkpoint_segments(sim_cls, oracle_mod):
    # a reduced version of the layered (faulted) workload: 192^2, 300 steps,
    # checkpoints every 200 steps (two levels inside each segment)
    n, nt = 192, 300
    c = W.layered_fault_model(n, n, 7, n_layers=8, throw=(3.0, 20.0))
    rng = np.random.default_rng(3)
    rec = W.line_receivers(32, 10, 8, n - 16)
    src = (n // 2, 10, W.ricker(nt, 0.04))
    kw = dict(tau=0.5, c_ref=5500.0)
    sim = sim_cls(c, lattice=5, sponge_width=12, sponge_sigma_max=0.1, **kw)
    sim.set_source(*src)
    sim.set_receivers(rec, nt)
    sim.init_pressure(None)
    sim.checkpoint_every(200)
    sim.step(nt)
    tr = sim.traces(nt).cpu().numpy()
    d = tr * 0.9 + rng.normal(size=tr.shape).astype(np.float32) * 1e-3
    gc, gs, _ = sim.adjoint((tr - d).astype(np.float32), nt)
    sim.close()
    P = oracle_mod.Problem(5, n, n, c, sponge_width=12, sponge_sigma_max=0.1, source=src,
                           receivers=rec, **kw)
    oc, os_, _ = oracle_mod.adjoint(P, P.zeros(), nt, (tr - d).astype(np.float64))
    assert rel(gc.cpu().numpy(), oc) < TOL
    assert rel(gs.cpu().numpy(), os_) < TOL
