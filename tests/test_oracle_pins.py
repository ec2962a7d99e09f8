"""Pins of the FP64 oracle against what arXiv:1704.03172 and the mathematics fix.

None of these compares the oracle with itself: each check is a printed value,
a closed form, an invariant, an exact reduction to another scheme, or an
independent (Fourier-space) formulation of the same linear map.
"""
import math

import numpy as np
import pytest

import lbspec
from paper_1704_03172_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _f32(x):
    """The value the oracle sees: sound speeds are handed over as float32."""
    return float(np.float32(x))


def _uniform(oracle, Q, n, eta=1.0, **kw):
    c = W.uniform_map(n, n, eta)
    return oracle.Problem(Q, n, n, c, c_ref=1.0, periodic=True, **kw)


# --- printed constants (App. A, App. B, Eq. higher moments) ------------------------------

@pytest.mark.parametrize("Q", [5, 9])
def test_moment_matrix_is_printed_matrix(oracle_mod, Q):
    M = oracle_mod.moment_matrix(Q)
    np.testing.assert_array_equal(M, lbspec.moment_matrix(Q))


def test_d2q5_inverse_matches_printed(oracle_mod):
    np.testing.assert_allclose(oracle_mod.moment_inverse(5), lbspec.golden("appB_Minv_d2q5.txt"),
                               rtol=0, atol=1e-15)


def test_d2q9_inverse_is_inverse(oracle_mod):
    M = lbspec.moment_matrix(9)
    np.testing.assert_allclose(oracle_mod.moment_inverse(9) @ M, np.eye(9), atol=1e-14)
    # rows of M are mutually orthogonal (App. A), so M^-1 = M^T diag(1/|row|^2)
    np.testing.assert_allclose(oracle_mod.moment_inverse(9),
                               M.T / (M * M).sum(axis=1)[None, :], atol=1e-15)


def test_d2q5_ex_ey_match_printed(oracle_mod):
    c = oracle_mod.velocities(5)
    M = oracle_mod.moment_matrix(5)
    Mi = oracle_mod.moment_inverse(5)
    np.testing.assert_allclose(M @ np.diag(c[:, 0]) @ Mi, lbspec.golden("appB_Ex_d2q5.txt"),
                               atol=1e-15)
    np.testing.assert_allclose(M @ np.diag(c[:, 1]) @ Mi, lbspec.golden("appB_Ey_d2q5.txt"),
                               atol=1e-15)


@pytest.mark.parametrize("eta", [1.0, 0.8, 0.5, 0.1])
def test_d2q5_weights_and_courant(oracle_mod, eta):
    w, cs2 = oracle_mod.weights(5, eta)
    c = oracle_mod.velocities(5)
    assert abs(w.sum() - 1) < 1e-15                                   # Eq. LB lattice moments
    T = (w[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0)
    np.testing.assert_allclose(T, cs2 * np.eye(2), atol=1e-15)
    assert abs(w[0] - (1 - eta * eta)) < 1e-15                         # Eq. 0th lattice weight
    assert abs(math.sqrt(cs2) - math.sqrt((1 - w[0]) / 2)) < 1e-15      # App. D Courant number
    assert (w >= 0).all()


def test_d2q9_conventional_weights(oracle_mod):
    # Sec. 3.2: D2Q9-con weights w0 = 4/9, w1 = 1/9, w5 = 1/36 at eta = 1 (c_s^2 = 1/3)
    w, cs2 = oracle_mod.weights(9, 1.0, (4 / 9, 1 / 9, 1 / 36))
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=1e-15)
    assert abs(cs2 - 1 / 3) < 1e-15
    w, cs2 = oracle_mod.weights(9, 0.6, (0.0, 0.01, 0.24))
    c = oracle_mod.velocities(9)
    T = (w[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0)
    np.testing.assert_allclose(T, cs2 * np.eye(2), atol=1e-15)
    assert abs(w.sum() - 1) < 1e-15


@pytest.mark.parametrize("eta", [1.0, 0.7, 0.3])
def test_d2q5_equilibrium_higher_moments(oracle_mod, eta):
    # Eq. higher moments e / p_xx: e^(0) = (-4 + 10 c_s^2) rho, p_xx^(0) = 0
    w, cs2 = oracle_mod.weights(5, eta)
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho, jx, jy = rng.normal(size=3)
        geq = oracle_mod.equilibrium(5, w, cs2, rho, jx, jy)
        m = lbspec.moment_matrix(5) @ geq
        np.testing.assert_allclose(m[:3], [rho, jx, jy], atol=1e-14)
        assert abs(m[3] - (-4 + 10 * cs2) * rho) < 1e-14
        assert abs(m[4]) < 1e-14


@pytest.mark.parametrize("eta,w_ref", [(1.0, (4 / 9, 1 / 9, 1 / 36)), (0.63, (0.4, 0.11, 0.04)),
                                       (0.31, (0.0, 0.01, 0.24))])
def test_d2q9_equilibrium_non_conserved_moments(oracle_mod, eta, w_ref):
    # the closed forms the D2Q9 MRT collision relaxes against (rows 3..8 of App. A's M):
    # e^eq = -4 rho + 12 w1 rho + 24 w5 rho, eps^eq = 4 rho - 24 w1 rho - 12 w5 rho,
    # q^eq = 4 (w5 - w1) / c_s^2 j, p_xx^eq = p_xy^eq = 0
    w, cs2 = oracle_mod.weights(9, eta, w_ref)
    w1, w5 = w[1], w[5]
    rng = np.random.default_rng(7)
    for _ in range(5):
        rho, jx, jy = rng.normal(size=3)
        m = lbspec.moment_matrix(9) @ oracle_mod.equilibrium(9, w, cs2, rho, jx, jy)
        np.testing.assert_allclose(m[:3], [rho, jx, jy], atol=1e-14)
        kq = 4 * (w5 - w1) / cs2
        np.testing.assert_allclose(
            m[3:], [(-4 + 12 * w1 + 24 * w5) * rho, 0.0, (4 - 24 * w1 - 12 * w5) * rho,
                    kq * jx, kq * jy, 0.0], atol=1e-13)


@pytest.mark.parametrize("Q", [5, 9])
def test_equilibrium_map_is_printed_A(oracle_mod, Q):
    # A = I - dg^eq/dg, printed for D2Q5 in Sec. 3.2 (Eq. D2Q5/D2Q9 dist to eqm dist)
    w, cs2 = oracle_mod.weights(Q, 0.77, (0.0, 0.01, 0.24))
    c = oracle_mod.velocities(Q)
    E = np.zeros((Q, Q))
    for j in range(Q):
        e = np.zeros(Q)
        e[j] = 1
        E[:, j] = oracle_mod.equilibrium(Q, w, cs2, e.sum(), c[:, 0] @ e, c[:, 1] @ e)
    np.testing.assert_allclose(np.eye(Q) - E, lbspec.a_matrix(Q, w, cs2), atol=1e-15)


# --- collision invariants (P1, P6) --------------------------------------------------------

@pytest.mark.parametrize("Q", [5, 9])
@pytest.mark.parametrize("mrt", [False, True])
def test_collision_conserves_mass_momentum(oracle_mod, Q, mrt):
    rng = np.random.default_rng(7)
    c = oracle_mod.velocities(Q)
    for _ in range(20):
        w, cs2 = oracle_mod.weights(Q, rng.uniform(0.2, 1.0), (0.0, 0.01, 0.24))
        s = rng.uniform(0.3, 2.0, size=Q)
        g = rng.normal(size=Q)
        gs = oracle_mod.collide(Q, mrt, rng.uniform(0.5, 3.0), s, w, cs2, g)
        assert abs(gs.sum() - g.sum()) < 1e-13
        np.testing.assert_allclose(c.T @ gs, c.T @ g, atol=1e-13)


def test_mrt_sp_se_2_equals_bgk_half(oracle_mod):
    # Sec. 3.2: D2Q5 MRT with s_p = s_e = 2 is identical to BGK tau = 1/2 for any s_rho, s_v
    rng = np.random.default_rng(3)
    for w0 in (0.0, 0.36, 0.75):
        w, cs2 = oracle_mod.weights(5, math.sqrt(1 - w0))
        for _ in range(10):
            s = [rng.uniform(0.2, 1.9), rng.uniform(0.2, 1.9), 0, 2.0, 2.0]
            s[2] = s[1]
            g = rng.normal(size=5)
            a = oracle_mod.collide(5, True, 0.5, s, w, cs2, g)
            b = oracle_mod.collide(5, False, 0.5, s, w, cs2, g)
            np.testing.assert_allclose(a, b, atol=1e-14)


def test_d2q9_quarter_weights_is_d2q5(oracle_mod):
    # Sec. 3.3: D2Q9 with w = (0, 1/4, 0) is the D2Q5 lattice (diagonals carry nothing)
    n = 24
    rng = np.random.default_rng(5)
    c = W.random_medium(n, n, 11, 0.5, 1.0)
    kw = dict(c_ref=1.0, periodic=True, tau=0.8, source=(5, 7, rng.normal(size=30)))
    P5 = oracle_mod.Problem(5, n, n, c, **kw)
    P9 = oracle_mod.Problem(9, n, n, c, w_ref=(0.0, 0.25, 0.0), **kw)
    g5 = rng.normal(size=(5, n, n))
    g9 = np.zeros((9, n, n))
    g9[:5] = g5
    r5, _ = oracle_mod.run(P5, g5, 30)
    r9, _ = oracle_mod.run(P9, g9, 30)
    np.testing.assert_allclose(r9[:5], r5, atol=1e-13)
    assert np.abs(r9[5:]).max() == 0.0


# --- dispersion (P2), brute force (P4) ----------------------------------------------------

@pytest.mark.parametrize("eta", [1.0, 0.6])
@pytest.mark.parametrize("kidx", [(1, 0), (5, 0), (3, 3), (7, 2), (12, 5), (0, 9)])
def test_d2q5_half_dispersion_closed_form(oracle_mod, eta, kidx):
    n = 32
    P = _uniform(oracle_mod, 5, n, eta, tau=0.5)
    T = lbspec.measured_amplification(oracle_mod, P, kidx)
    _, cs2 = oracle_mod.weights(5, _f32(eta))
    k = 2 * np.pi * np.array(kidx) / n
    om = lbspec.d2q5_closed_form_omega(k, cs2)
    # lambda is a root of det(T - lambda I): backward test via the smallest singular value
    # (eigenvalues of this non-normal matrix near lambda = 1 are only sqrt(eps)-accurate)
    for target in (np.exp(1j * om), np.exp(-1j * om), -1.0):
        assert _smin(T - target * np.eye(5)) < 1e-13
    np.testing.assert_allclose(np.abs(np.linalg.eigvals(T)), 1.0, atol=1e-7)  # lossless


def _smin(A):
    return np.linalg.svd(A, compute_uv=False)[-1]


def test_d1q3_axis_root(oracle_mod):
    # App. E: along theta = 0, omega = 2 arcsin(c_s sin(k/2)) and a root lambda = -1
    n = 40
    for eta in (1.0, 0.5):
        P = _uniform(oracle_mod, 5, n, eta, tau=0.5)
        _, cs2 = oracle_mod.weights(5, _f32(eta))
        for m in (1, 4, 10, 19):
            T = lbspec.measured_amplification(oracle_mod, P, (m, 0))
            k = 2 * np.pi * m / n
            om = 2 * np.arcsin(math.sqrt(cs2) * math.sin(k / 2))
            assert _smin(T - np.exp(1j * om) * np.eye(5)) < 1e-13
            assert _smin(T + np.eye(5)) < 1e-13


CASES = [
    (5, False, 0.5, None, 1.0, (4 / 9, 1 / 9, 1 / 36)),
    (5, False, 1.0, None, 0.8, (4 / 9, 1 / 9, 1 / 36)),
    (5, True, 0.5, [1.3, 0.7, 0.7, 1.1, 1.6], 0.9, (4 / 9, 1 / 9, 1 / 36)),
    (9, False, 0.5, None, 1.0, (4 / 9, 1 / 9, 1 / 36)),
    (9, True, 0.5, [1.0, 1.0, 1.0, 2.0, 2.0, 2.0, 1.0, 1.0, 2.0], 1.0, (4 / 9, 1 / 9, 1 / 36)),
    (9, True, 0.5, [0.7, 1.2, 1.2, 1.5, 0.9, 1.8, 1.1, 1.1, 0.9], 0.7, (0.0, 0.01, 0.24)),
]


@pytest.mark.parametrize("Q,mrt,tau,s,eta,wref", CASES)
def test_amplification_matches_paper_matrix(oracle_mod, Q, mrt, tau, s, eta, wref):
    n = 16
    P = oracle_mod.Problem(Q, n, n, W.uniform_map(n, n, eta), c_ref=1.0, periodic=True,
                           mrt=mrt, tau=tau, s=s, w_ref=wref)
    w, cs2 = oracle_mod.weights(Q, _f32(eta), wref)
    for kidx in [(1, 0), (3, 2), (8, 8), (5, 13)]:
        k = 2 * np.pi * np.array(kidx) / n
        Tm = lbspec.measured_amplification(oracle_mod, P, kidx)
        Tp = lbspec.amplification(Q, k, w, cs2, mrt, tau, s)
        np.testing.assert_allclose(Tm, Tp, atol=1e-13)


def test_d2q9_bgk_lossless_mrt_sq1_attenuates(oracle_mod):
    # Sec. 3.2: D2Q9 BGK (tau = 1/2) is attenuation free; MRT with s_q = 1 attenuates
    n = 16
    c = W.uniform_map(n, n, 1.0)
    Pb = oracle_mod.Problem(9, n, n, c, c_ref=1.0, periodic=True, tau=0.5)
    s = [1.0, 1.0, 1.0, 2.0, 2.0, 2.0, 1.0, 1.0, 2.0]
    Pm = oracle_mod.Problem(9, n, n, c, c_ref=1.0, periodic=True, mrt=True, s=s)
    lb = np.linalg.eigvals(lbspec.measured_amplification(oracle_mod, Pb, (4, 1)))
    lm = np.linalg.eigvals(lbspec.measured_amplification(oracle_mod, Pm, (4, 1)))
    np.testing.assert_allclose(np.abs(lb), 1.0, atol=1e-12)
    assert np.abs(lm).min() < 0.999


def test_dense_transition_matrix_8x8(oracle_mod):
    # brute force: the full (Q N)^2 one-step matrix of an 8x8 periodic grid has exactly
    # the eigenvalues of T(k) over the 64 grid wave vectors
    n, Q, eta = 8, 5, 0.9
    s = [1.0, 1.0, 1.0, 1.4, 1.7]
    P = oracle_mod.Problem(Q, n, n, W.uniform_map(n, n, eta), c_ref=1.0, periodic=True,
                           mrt=True, s=s)
    N = Q * n * n
    B = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1
        B[:, j] = oracle_mod.run(P, e.reshape(Q, n, n), 1)[0].ravel()
    lam_b = np.linalg.eigvals(B)
    w, cs2 = oracle_mod.weights(Q, _f32(eta))
    lam_k = np.concatenate([
        np.linalg.eigvals(lbspec.amplification(Q, 2 * np.pi * np.array([mx, my]) / n, w, cs2,
                                               True, 0.5, s))
        for mx in range(n) for my in range(n)])
    d1 = np.abs(lam_b[:, None] - lam_k[None, :]).min(axis=1).max()
    d2 = np.abs(lam_k[:, None] - lam_b[None, :]).min(axis=1).max()
    assert max(d1, d2) < 1e-6   # eigenvalues of a defective matrix are sqrt(eps)-sensitive


def test_gaussian_pulse_run_matches_per_mode_solution(oracle_mod):
    # the 128^2 periodic Gaussian-pulse workload (tau = 1), 500 steps: every Fourier mode
    # evolves as T(k)^n (exact discrete solution)
    n, steps = 128, 500
    P = oracle_mod.Problem(5, n, n, W.uniform_map(n, n, 1.0), c_ref=1.0, periodic=True, tau=1.0)
    p0 = W.gaussian_pulse(n, n, 64, 64, 4.0, 1e-3)
    g0 = oracle_mod.init_pressure(P, p0)
    g, _ = oracle_mod.run(P, g0, steps)
    w, cs2 = oracle_mod.weights(5, 1.0)
    ge = lbspec.exact_evolution(g0, 5, w, cs2, steps, tau=1.0)
    assert np.linalg.norm(g - ge) / np.linalg.norm(ge) < 1e-10


# --- exact reduction to the O[2,2] leapfrog (App. C), heterogeneous, with source (P3) -----

def test_d2q5_half_is_leapfrog_in_heterogeneous_medium(oracle_mod):
    n, steps = 24, 60
    rng = np.random.default_rng(9)
    c = W.random_medium(n, n, 13, 0.3, 1.0)
    S = rng.normal(size=steps)
    xs, ys = 7, 15
    P = oracle_mod.Problem(5, n, n, c, c_ref=1.0, periodic=True, tau=0.5, source=(xs, ys, S))
    g = rng.normal(size=(5, n, n))
    rhos = [g.sum(0)]
    for t in range(steps):
        g, _ = oracle_mod.run(P, g, 1, t0=t)
        rhos.append(g.sum(0))
    eta2 = (c.astype(np.float64) / 1.0) ** 2
    w0 = 1 - eta2            # Eq. 0th lattice weight
    w1 = eta2 / 4
    sig = np.zeros((n, n))
    sig[ys, xs] = w0[ys, xs]
    for dx, dy in ((1, 0), (0, 1), (-1, 0), (0, -1)):
        sig[(ys + dy) % n, (xs + dx) % n] += w1[ys, xs]
    err = 0.0
    for t in range(1, steps):
        r, rm = rhos[t], rhos[t - 1]
        lap = sum(np.roll(2 * w1 * r, (dy, dx), axis=(0, 1))
                  for dx, dy in ((1, 0), (0, 1), (-1, 0), (0, -1)))
        pred = 2 * w0 * r + lap - rm + sig * S[t]
        pred[ys, xs] -= S[t - 1]
        err = max(err, np.abs(pred - rhos[t + 1]).max() / np.abs(rhos[t + 1]).max())
    assert err < 1e-12


# --- energy (P5) ----------------------------------------------------------------------------

def _energy(oracle, g, Q, eta):
    w, _ = oracle.weights(Q, _f32(eta))
    keep = w > 0
    return sum((g[i] ** 2).sum() / w[i] for i in range(Q) if keep[i])


@pytest.mark.parametrize("eta", [1.0, 0.6])
def test_energy_conserved_at_half_and_decays_above(oracle_mod, eta):
    n = 32
    rng = np.random.default_rng(2)
    P = _uniform(oracle_mod, 5, n, eta, tau=0.5)
    g = rng.normal(size=(5, n, n))
    if eta == 1.0:
        g[0] = 0.0                       # w0 = 0: the rest population carries nothing
    E0 = _energy(oracle_mod, g, 5, eta)
    g1, _ = oracle_mod.run(P, g, 100)
    assert abs(_energy(oracle_mod, g1, 5, eta) - E0) / E0 < 1e-12
    Pd = _uniform(oracle_mod, 5, n, eta, tau=0.9)
    Es = [E0]
    gd = g
    for _ in range(10):
        gd, _ = oracle_mod.run(Pd, gd, 5)
        Es.append(_energy(oracle_mod, gd, 5, eta))
    assert all(b <= a * (1 + 1e-14) for a, b in zip(Es, Es[1:]))
    assert Es[-1] < 0.9 * Es[0]


# --- boundary and sponge bookkeeping ------------------------------------------------------

def test_zero_ghost_mass_balance(oracle_mod):
    # with zero-ghost edges the total mass changes only by the source and by the populations
    # that stream out across the edge (their post-collision values at the edge sites)
    n = 20
    rng = np.random.default_rng(4)
    c = W.random_medium(n, n, 3, 0.4, 1.0)
    S = rng.normal(size=5)
    P = oracle_mod.Problem(5, n, n, c, c_ref=1.0, periodic=False, tau=0.7, source=(9, 4, S))
    Pp = oracle_mod.Problem(5, n, n, c, c_ref=1.0, periodic=True, tau=0.7, source=(9, 4, S))
    g = rng.normal(size=(5, n, n))
    for t in range(5):
        gz, _ = oracle_mod.run(P, g, 1, t0=t)
        gp, _ = oracle_mod.run(Pp, g, 1, t0=t)   # periodic: nothing is lost
        # out-going populations reappear on the opposite edge in the periodic run
        lost = gp[1][:, 0].sum() + gp[3][:, -1].sum() + gp[2][0, :].sum() + gp[4][-1, :].sum()
        assert abs((gp.sum() - gz.sum()) - lost) < 1e-12
        assert abs(gp.sum() - (g.sum() + S[t])) < 1e-11
        g = gz


def test_sponge_profile(oracle_mod):
    # sigma = s_max ((W - d)/W)^2 for d < W, 0 inside; applied as a factor (1 - sigma)
    assert oracle_mod.sponge_sigma(0, 50, 100, 100, 10, 0.1) == pytest.approx(0.1)
    assert oracle_mod.sponge_sigma(5, 50, 100, 100, 10, 0.1) == pytest.approx(0.1 * 0.25)
    assert oracle_mod.sponge_sigma(10, 50, 100, 100, 10, 0.1) == 0.0
    assert oracle_mod.sponge_sigma(99, 97, 100, 100, 10, 0.1) == pytest.approx(0.1)
    n = 12
    P = oracle_mod.Problem(5, n, n, W.uniform_map(n, n, 1.0), c_ref=1.0, periodic=True,
                           tau=0.5, sponge_width=3, sponge_sigma_max=0.2)
    P0 = oracle_mod.Problem(5, n, n, W.uniform_map(n, n, 1.0), c_ref=1.0, periodic=True,
                            tau=0.5)
    g = np.random.default_rng(1).normal(size=(5, n, n))
    a, _ = oracle_mod.run(P, g, 1)
    b, _ = oracle_mod.run(P0, g, 1)
    cv = oracle_mod.velocities(5)
    for i in range(5):
        fac = np.array([[1 - oracle_mod.sponge_sigma(x, y, n, n, 3, 0.2) for x in range(n)]
                        for y in range(n)])
        fac = np.roll(fac, (cv[i, 1], cv[i, 0]), axis=(0, 1))   # factor travels with the push
        np.testing.assert_allclose(a[i], b[i] * fac, atol=1e-14)


def test_receiver_trace_is_pressure_before_step(oracle_mod):
    n = 16
    rng = np.random.default_rng(8)
    c = W.random_medium(n, n, 2, 0.5, 1.0)
    rec = np.array([[3, 4], [10, 12], [0, 15]], dtype=np.int32)
    P = oracle_mod.Problem(5, n, n, c, c_ref=1.0, tau=0.6, receivers=rec)
    g = rng.normal(size=(5, n, n))
    _, tr = oracle_mod.run(P, g, 4)
    gg = g
    for t in range(4):
        p = oracle_mod.pressure(P, gg)
        np.testing.assert_allclose(tr[t], p[rec[:, 1], rec[:, 0]], atol=1e-15)
        eta2 = (c[rec[:, 1], rec[:, 0]].astype(np.float64)) ** 2
        np.testing.assert_allclose(tr[t], eta2 / 2 * gg.sum(0)[rec[:, 1], rec[:, 0]],
                                   atol=1e-14)   # p = c_s^2 rho, c_s^2 = eta^2 / 2 (D2Q5)
        gg, _ = oracle_mod.run(P, gg, 1, t0=t)


@pytest.mark.parametrize("Q", [5, 9])
def test_seeded_mrt_rates_of_the_two_layer_workload_are_stable(Q):
    # Reading A2: the seeded MRT rates must pass a stability precheck, max |lambda(k)| <= 1 +
    # 1e-12 over a 64^2 wave-vector grid, at every speed of the medium (eta = 1/2 and 1 in
    # the two-layer workload), with the workload's weights; built from the amplification
    # matrix T(k) = D(k) (I - C A) written independently of the oracle's stepper
    wl = W.two_layer_workload(64, lattice=Q, collision="mrt")
    s, wref, n = wl["s"], wl["w_ref"], 64
    worst = 0.0
    for eta in sorted({float(v) / wl["c_ref"] for v in np.unique(wl["c_map"])}):
        e2 = eta * eta
        if Q == 5:
            w, cs2 = np.array([1 - e2] + [e2 / 4] * 4), e2 / 2
        else:
            w1, w5 = e2 * wref[1], e2 * wref[2]
            w = np.array([1 - 4 * (w1 + w5)] + [w1] * 4 + [w5] * 4)
            cs2 = e2 * (2 * wref[1] + 4 * wref[2])
        for a in range(n):
            for b in range(n):
                T = lbspec.amplification(Q, (2 * np.pi * a / n, 2 * np.pi * b / n), w, cs2,
                                         mrt=True, s=s)
                worst = max(worst, np.abs(np.linalg.eigvals(T)).max())
    assert worst <= 1 + 1e-12


def test_oracle_window_equals_the_full_grid_run(oracle_mod):
    # The parity test at 8192^2 runs the oracle on the window that a zero initial state can
    # fill in T steps from the source (one cell per step in L1 distance for D2Q5) plus the
    # sponge band of the window's own edges.  On a small grid the window run must equal the
    # full run exactly -- traces of every receiver, the field inside the window, and exact
    # zeros outside it -- heterogeneous medium, 12-cell sponge at the real edges.
    from tests.test_gpu_fulllength import diamond_window
    n, steps, W_s = 200, 60, 12
    c = W.layered_fault_model(n, n, 7, n_layers=9, throw=(2.0, 20.0))
    src = (100, 20, W.ricker(steps, 0.03))
    rec = W.line_receivers(40, 20, 12, n - 24)
    P = oracle_mod.Problem(5, n, n, c, c_ref=5500.0, tau=0.5, sponge_width=W_s,
                           sponge_sigma_max=0.1, source=src, receivers=rec)
    g, tr = oracle_mod.run(P, P.zeros(), steps)
    x0, x1, y0, y1 = diamond_window(src[:2], steps, W_s, n)
    assert (x0, y0) != (0, 0) and x1 < n and y1 < n                  # a true sub-window
    inw = (rec[:, 0] >= x0) & (rec[:, 0] < x1)
    Pw = oracle_mod.Problem(5, x1 - x0, y1 - y0, c[y0:y1, x0:x1], c_ref=5500.0, tau=0.5,
                            sponge_width=W_s, sponge_sigma_max=0.1,
                            source=(src[0] - x0, src[1] - y0, src[2]),
                            receivers=rec[inw] - np.array([x0, y0], np.int32))
    gw, trw = oracle_mod.run(Pw, Pw.zeros(), steps)
    np.testing.assert_array_equal(trw, tr[:, inw])
    assert not tr[:, ~inw].any()
    np.testing.assert_array_equal(gw, g[:, y0:y1, x0:x1])
    out = np.ones(g.shape[1:], bool)
    out[y0:y1, x0:x1] = False
    assert not g[:, out].any()
