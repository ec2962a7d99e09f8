"""GPU tests of the continuous-batching shot server (lb_server_*).

Each served result must be the same alone and in a mix of other requests of
different sizes, storage types and kinds (the batched launch runs the same
per-shot arithmetic), must match the FP64 oracle to FP32 tolerance, and
gradient requests must match the direct adjoint.  Admission respects the
device-memory budget.
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300 import lbac
    from paper_1704_03172_gb300.sim import LBServer, LBSim
    return LBServer, LBSim, lbac


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _shot(n, seed, nt, storage="f32", grad=False, lattice=5):
    c = W.layered_fault_model(n, n, seed, n_layers=6, throw=(2.0, n / 16))
    src = (n // 2, 6, W.ricker(nt, 0.05))
    rec = W.line_receivers(16, 6, 4, n - 8)
    spec = dict(nt=nt, source=src, receivers=rec, lattice=lattice, tau=0.5, storage=storage,
                sponge_width=6, c_ref=5500.0)
    if grad:
        spec.update(want_gradient=True, observed=np.zeros((nt, len(rec)), np.float32),
                    checkpoint_every=32)
    return c, spec


# tb_min_ctas: 0 the server's own rule (these small shots never fill a wave: one launch per
# step), 1 every eligible D2Q5 shot takes 4 steps per launch, -1 never
@pytest.mark.parametrize("tb", [0, 1, -1])
def test_result_is_identical_alone_and_in_the_mix(mods, oracle_mod, tb):
    LBServer, _, _ = mods
    cA, sA = _shot(96, 1, 300)
    srv = LBServer(max_active=1, rounds_per_pass=8, tb_min_ctas=tb)
    a = srv.submit(cA, **sA)
    srv.wait(a, 60000)
    alone = srv.result(a)["traces"]
    srv.close()
    # a mix: different sizes, storage types, a gradient request, staggered arrivals
    srv = LBServer(max_active=6, rounds_per_pass=8, tb_min_ctas=tb)
    ids = []
    for k, (n, st, g) in enumerate([(128, "f32", False), (64, "bf16", False), (160, "f32", True),
                                     (80, "f16", False), (200, "bf16", False), (96, "bf16", True)]):
        c, s = _shot(n, 10 + k, 200 + 37 * k, st, g)
        ids.append(srv.submit(c, **s))
    a2 = srv.submit(cA, **sA)
    c, s = _shot(112, 30, 250)
    ids.append(srv.submit(c, **s))
    srv.wait(a2, 120000)
    mixed = srv.result(a2)["traces"]
    for i in ids:
        srv.wait(i, 120000)
        srv.result(i)
    st = srv.stats()
    srv.close()
    np.testing.assert_array_equal(mixed, alone)
    assert st["launches"] > 0
    P = oracle_mod.Problem(5, 96, 96, cA, c_ref=5500.0, tau=0.5, sponge_width=6,
                           sponge_sigma_max=0.1, source=sA["source"], receivers=sA["receivers"])
    _, tro = oracle_mod.run(P, P.zeros(), sA["nt"])
    assert rel(alone, tro) < 1e-5


def test_time_blocked_batches_cut_the_launches(mods, oracle_mod):
    # the same four FP32 / BF16 shots with 4 steps per launch and with one launch per step:
    # far fewer launches, and the same FP32 traces to rounding (BF16 differs more: the
    # time-blocked kernel rounds to BF16 once per 4 steps, the one-step kernel every step)
    LBServer, _, _ = mods
    shots = [_shot(n, 40 + k, 256, st) for k, (n, st) in
             enumerate([(96, "f32"), (160, "f32"), (128, "bf16"), (300, "f32")])]
    out = {}
    for tb in (1, -1):
        srv = LBServer(max_active=4, rounds_per_pass=32, tb_min_ctas=tb)
        ids = [srv.submit(c, **s) for c, s in shots]
        for i in ids:
            srv.wait(i, 120000)
        out[tb] = ([srv.result(i)["traces"] for i in ids], srv.stats()["launches"])
        srv.close()
    # 4 steps per launch: a quarter of the step launches, plus the one-step tails of passes
    assert out[1][1] * 2 < out[-1][1], (out[1][1], out[-1][1])
    for (c, s), a, b in zip(shots, out[1][0], out[-1][0]):
        assert rel(a, b) < (3e-6 if s["storage"] == "f32" else 0.1)
    c, s = shots[0]
    P = oracle_mod.Problem(5, 96, 96, c, c_ref=5500.0, tau=0.5, sponge_width=6,
                           sponge_sigma_max=0.1, source=s["source"], receivers=s["receivers"])
    _, tro = oracle_mod.run(P, P.zeros(), s["nt"])
    assert rel(out[1][0][0], tro) < 1e-5


def test_gradient_request_matches_direct_adjoint(mods, oracle_mod):
    LBServer, LBSim, _ = mods
    n, nt = 72, 120
    c, s = _shot(n, 4, nt, grad=True)
    rng = np.random.default_rng(2)
    d = rng.normal(size=(nt, 16)).astype(np.float32) * 1e-3
    s["observed"] = d
    srv = LBServer(max_active=4, rounds_per_pass=16)
    rid = srv.submit(c, **s)
    c2, s2 = _shot(90, 9, 180)
    rid2 = srv.submit(c2, **s2)
    srv.wait(rid, 120000)
    res = srv.result(rid)
    srv.wait(rid2, 120000)
    srv.result(rid2)
    srv.close()
    P = oracle_mod.Problem(5, n, n, c, c_ref=5500.0, tau=0.5, sponge_width=6,
                           sponge_sigma_max=0.1, source=s["source"], receivers=s["receivers"])
    _, tro = oracle_mod.run(P, P.zeros(), nt)
    assert rel(res["traces"], tro) < 1e-5
    oc, os_, _ = oracle_mod.adjoint(P, P.zeros(), nt, (res["traces"] - d).astype(np.float64))
    assert rel(res["grad_c"], oc) < 1e-4
    assert rel(res["grad_src"], os_) < 1e-4


def test_bf16_gradient_request_matches_direct_bf16_adjoint(mods, oracle_mod):
    # a served BF16 shot runs the same kernels as a direct BF16 context, so its traces
    # and its gradient (FP32 adjoint over the replayed BF16 states) match the direct ones
    LBServer, LBSim, _ = mods
    n, nt = 80, 150
    c, s = _shot(n, 6, nt, storage="bf16", grad=True)
    rng = np.random.default_rng(5)
    d = rng.normal(size=(nt, 16)).astype(np.float32) * 1e-3
    s["observed"] = d
    srv = LBServer(max_active=4, rounds_per_pass=8)
    rid = srv.submit(c, **s)
    c2, s2 = _shot(128, 8, 120, storage="f32", grad=True)
    rid2 = srv.submit(c2, **s2)
    srv.wait(rid, 120000)
    res = srv.result(rid)
    srv.wait(rid2, 120000)
    srv.result(rid2)
    srv.close()
    sim = LBSim(c, lattice=5, tau=0.5, storage="bf16", sponge_width=6, c_ref=5500.0)
    sim.set_source(*s["source"])
    sim.set_receivers(s["receivers"], nt)
    sim.init_pressure(None)
    sim.checkpoint_every(32)
    sim.step(nt)
    tr = sim.traces(nt).cpu().numpy()
    gc, gs, _ = sim.adjoint((tr - d).astype(np.float32), nt)
    sim.close()
    np.testing.assert_array_equal(res["traces"], tr)
    np.testing.assert_allclose(res["grad_c"], gc.cpu().numpy(), rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(res["grad_src"], gs.cpu().numpy(), rtol=1e-6, atol=1e-15)


def test_admission_respects_the_memory_budget(mods):
    LBServer, _, lbac = mods
    c, s = _shot(256, 3, 100)
    cfg = lbac.lb_config_default()
    cfg.nx = cfg.ny = 256
    one = lbac.lb_footprint(cfg, 100, 16, 0)
    srv = LBServer(max_active=8, hbm_budget=int(2.5 * one) + (1 << 20), rounds_per_pass=4)
    ids = [srv.submit(c, **s) for _ in range(5)]
    peak = 0
    import time
    t0 = time.time()
    while not all(srv.poll(i) for i in ids) and time.time() - t0 < 120:
        peak = max(peak, srv.stats()["active"])
        time.sleep(0.002)
    outs = [srv.result(i)["traces"] for i in ids]
    srv.close()
    assert peak <= 2                                   # at most two fit the budget at once
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    big_c, big_s = _shot(512, 3, 100)
    srv = LBServer(max_active=8, hbm_budget=int(2.5 * one), rounds_per_pass=4)
    with pytest.raises(lbac.LBError) as e:
        srv.submit(big_c, **big_s)
    assert e.value.status == lbac.LB_ENOMEM
    srv.close()


def test_wait_times_out_and_then_completes(mods):
    LBServer, _, lbac = mods
    c, s = _shot(512, 5, 3000)
    srv = LBServer(max_active=2, rounds_per_pass=4)
    rid = srv.submit(c, **s)
    with pytest.raises(lbac.LBError) as e:
        srv.wait(rid, 0)
    assert e.value.status == lbac.LB_ETIMEOUT
    srv.wait(rid, 120000)
    r = srv.result(rid)
    srv.close()
    assert r["done"] >= r["start"] >= r["submit"]
    assert np.isfinite(r["traces"]).all()


@pytest.mark.parametrize("every,storage", [(-1, "f32"), (0, "bf16"), (-1, "f16")])
def test_tape_gradient_request_matches_direct_tape_adjoint(mods, oracle_mod, every, storage):
    # gradient requests that record the forward rho tape (checkpoint_every < 0, or 0 with a
    # small tape) run no replay; FP16 storage works there.  The served shot runs the same
    # kernels as a direct context with lb_record_rho: identical traces, the same gradient
    LBServer, LBSim, _ = mods
    n, nt = 80, 150
    c, s = _shot(n, 6, nt, storage=storage, grad=True)
    s["checkpoint_every"] = every
    rng = np.random.default_rng(5)
    d = rng.normal(size=(nt, 16)).astype(np.float32) * 1e-3
    s["observed"] = d
    srv = LBServer(max_active=4, rounds_per_pass=8)
    rid = srv.submit(c, **s)
    c2, s2 = _shot(128, 8, 120, storage="f32", grad=True)
    rid2 = srv.submit(c2, **s2)
    srv.wait(rid, 120000)
    res = srv.result(rid)
    srv.wait(rid2, 120000)
    srv.result(rid2)
    srv.close()
    sim = LBSim(c, lattice=5, tau=0.5, storage=storage, sponge_width=6, c_ref=5500.0)
    sim.set_source(*s["source"])
    sim.set_receivers(s["receivers"], nt)
    sim.init_pressure(None)
    sim.record_rho(nt)
    sim.step(nt)
    tr = sim.traces(nt).cpu().numpy()
    gc, gs, _ = sim.adjoint((tr - d).astype(np.float32), nt)
    sim.close()
    np.testing.assert_array_equal(res["traces"], tr)
    np.testing.assert_allclose(res["grad_c"], gc.cpu().numpy(), rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(res["grad_src"], gs.cpu().numpy(), rtol=1e-6, atol=1e-15)
    if storage == "f32":  # and the FP64 oracle
        P = oracle_mod.Problem(5, n, n, c, c_ref=5500.0, tau=0.5, sponge_width=6,
                               sponge_sigma_max=0.1, source=s["source"], receivers=s["receivers"])
        oc, os_, _ = oracle_mod.adjoint(P, P.zeros(), nt, (res["traces"] - d).astype(np.float64))
        assert rel(res["grad_c"], oc) < 1e-4
        assert rel(res["grad_src"], os_) < 1e-4
