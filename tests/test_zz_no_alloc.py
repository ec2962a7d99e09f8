"""GPU test of lb_invariants_noalloc, the entry point for callers that cannot allocate.

It must give the same mass / energy / max|g| / non-finite count as the
context-based lb_invariants on the same state, using only a static device
scratch array.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300 import lbac
    from paper_1704_03172_gb300.sim import LBSim
    return torch, lbac, LBSim


def _noalloc(torch, lbac, sim, c_dev, c_ref, w_ref, stream):
    g = sim.state()                                     # device [Q][ny][nx] FP32
    out = torch.full((4,), -1.0, dtype=torch.float64, device=g.device)
    torch.cuda.current_stream().synchronize()
    lbac.lb_invariants_noalloc(ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(c_dev.data_ptr()),
                               sim.Q, sim.nx, sim.ny, c_ref, w_ref,
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("Q,nx,ny", [(5, 301, 77), (9, 128, 96)])
def test_noalloc_matches_context_invariants_twice(env, Q, nx, ny):
    torch, lbac, LBSim = env
    c = W.random_medium(nx, ny, 17, 0.5, 1.0)
    w_ref = (0.4, 0.11, 0.04) if Q == 9 else None
    sim = LBSim(c, lattice=Q, tau=0.7, c_ref=1.0, sponge_width=4,
                w_ref=w_ref if w_ref else (4 / 9, 1 / 9, 1 / 36))
    sim.set_state(np.random.default_rng(Q).normal(size=(Q, ny, nx)).astype(np.float32))
    c_dev = torch.as_tensor(c, device="cuda")
    stream = torch.cuda.Stream()
    for steps in (13, 29):                              # two calls in a row
        sim.step(steps)
        ref = np.array(sim.invariants())
        got = _noalloc(torch, lbac, sim, c_dev, 1.0, w_ref, stream)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    sim.close()


def test_noalloc_rejects_rows_beyond_static_scratch(env):
    torch, lbac, _ = env
    g = torch.zeros(1, device="cuda")
    with pytest.raises(lbac.LBError) as e:
        lbac.lb_invariants_noalloc(ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                   5, 4, 16385, 1.0, None, ctypes.c_void_p(g.data_ptr()), None)
    assert e.value.status == lbac.LB_EINVAL
    assert "16384" in lbac.lb_last_error(None)
