"""Pins of the FP64 adjoint oracle: dot-product identities of the linear map and
central finite differences of the nonlinear dependence on the sound speed.

The forward side is the oracle's stepper (orc_run); the adjoint is a separate
loop (orc_adjoint) that transposes it.  Neither is autodiff.
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W

CASES = [
    # Q, mrt, tau, s, periodic, sponge
    (5, False, 0.5, None, False, 4),
    (5, True, 0.5, [1.2, 0.9, 0.9, 1.6, 1.3], False, 3),
    (5, False, 0.8, None, True, 0),
    (9, True, 0.5, [1.0, 1.0, 1.0, 1.7, 1.4, 1.6, 1.2, 1.2, 1.4], False, 3),
    (9, False, 0.7, None, True, 0),
]


def _problem(oracle, Q, mrt, tau, s, periodic, sponge, c, src, rec):
    n_y, n_x = c.shape
    return oracle.Problem(Q, n_x, n_y, c, c_ref=1.0, periodic=periodic, mrt=mrt, tau=tau, s=s,
                          w_ref=(0.4, 0.11, 0.04), sponge_width=sponge, sponge_sigma_max=0.15,
                          source=src, receivers=rec)


def _setup(seed, nx=19, ny=15, nt=24):
    rng = np.random.default_rng(seed)
    c = W.random_medium(nx, ny, seed, 0.5, 1.0)
    rec = np.stack([rng.integers(0, nx, 5), rng.integers(0, ny, 5)], 1).astype(np.int32)
    src = (int(rng.integers(3, nx - 3)), int(rng.integers(3, ny - 3)), rng.normal(size=nt))
    R = rng.normal(size=(nt, len(rec)))
    return rng, c, src, rec, R


@pytest.mark.parametrize("case", CASES)
def test_dot_product_initial_state(oracle_mod, case):
    Q = case[0]
    rng, c, src, rec, R = _setup(1)
    nt = R.shape[0]
    P = _problem(oracle_mod, *case, c, (src[0], src[1], np.zeros(nt)), rec)
    g0 = rng.normal(size=(Q,) + c.shape)
    _, tr = oracle_mod.run(P, g0, nt)                      # L g0
    _, _, gg = oracle_mod.adjoint(P, g0, nt, R)            # L^T R
    lhs, rhs = (tr * R).sum(), (g0 * gg).sum()
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.abs(tr * R).sum())


@pytest.mark.parametrize("case", CASES)
def test_dot_product_source(oracle_mod, case):
    Q = case[0]
    rng, c, src, rec, R = _setup(2)
    nt = R.shape[0]
    P = _problem(oracle_mod, *case, c, src, rec)
    _, tr = oracle_mod.run(P, np.zeros((Q,) + c.shape), nt)
    _, gs, _ = oracle_mod.adjoint(P, np.zeros((Q,) + c.shape), nt, R)
    lhs, rhs = (tr * R).sum(), (src[2] * gs).sum()
    assert abs(lhs - rhs) <= 1e-12 * np.abs(tr * R).sum()


def _misfit(oracle, P, g0, nt, d):
    _, tr = oracle.run(P, g0, nt)
    return 0.5 * ((tr - d) ** 2).sum(), tr


@pytest.mark.parametrize("case", CASES)
def test_sound_speed_gradient_matches_central_differences(oracle_mod, case):
    Q = case[0]
    rng, c, src, rec, _ = _setup(3)
    nt = 24
    g0 = rng.normal(size=(Q,) + c.shape) * 0.1
    d = rng.normal(size=(nt, len(rec)))
    P = _problem(oracle_mod, *case, c, src, rec)
    _, tr = _misfit(oracle_mod, P, g0, nt, d)
    gc, _, _ = oracle_mod.adjoint(P, g0, nt, tr - d)
    sites = [(src[1], src[0]), (rec[0, 1], rec[0, 0])] + \
        [(int(rng.integers(c.shape[0])), int(rng.integers(c.shape[1]))) for _ in range(6)]
    def central(y, x, h):
        cp, cm = c.copy(), c.copy()
        cp[y, x] = np.float32(c[y, x] + h)
        cm[y, x] = np.float32(c[y, x] - h)
        heff = (float(cp[y, x]) - float(cm[y, x])) / 2       # the step the float32 map holds
        Jp, _ = _misfit(oracle_mod, _problem(oracle_mod, *case, cp, src, rec), g0, nt, d)
        Jm, _ = _misfit(oracle_mod, _problem(oracle_mod, *case, cm, src, rec), g0, nt, d)
        return (Jp - Jm) / (2 * heff)

    for (y, x) in sites:
        # Richardson extrapolation of central differences (error O(h^4)): J is strongly
        # nonlinear in c for the lossless scheme, so plain central differences carry an
        # O(h^2) truncation error of ~1e-5 at h = 1e-4
        fd = (4 * central(y, x, 1e-4) - central(y, x, 2e-4)) / 3
        assert abs(fd - gc[y, x]) <= 1e-6 * max(abs(fd), 1e-2 * np.abs(gc).max())
