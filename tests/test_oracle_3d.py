"""Pins of the three-dimensional (D3Q7) oracle.

D3Q7 carries the D2Q5 rule to three dimensions: w_0 = 1 - eta^2, w_1..6 = eta^2 / 6,
c_s^2 = eta^2 / 3 (Eq. 0th lattice weight; Eq. linear eqm dist; BGK, Eq. BGK-LB).  What
fixes the oracle:
- the collision conserves rho and j at every site, so a periodic run keeps total mass and
  momentum exactly, in any medium and for any tau;
- at tau = 1/2 the density obeys exactly the 3-D second-order leapfrog with the 7-point
  variable-coefficient Laplacian (the 3-D form of the reduction of App. C), source included;
- the one-step map of a Fourier mode has the eigenvalues exp(+-i w) with
  sin^2(w/2) = c_s^2 [sin^2(kx/2) + sin^2(ky/2) + sin^2(kz/2)] (the D2Q5 closed form with a
  third term), and -1; all of modulus 1;
- at tau = 1/2 the energy sum g_i^2 / w_i of a homogeneous periodic run is conserved (the
  collision is a reflection in that metric); above tau = 1/2 it decays.
"""
import numpy as np
import pytest

V7 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])


def _medium(n, seed, lo=0.3, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=(n, n, n)).astype(np.float32)


def test_mass_and_momentum_conserved_periodic(oracle_mod):
    n = 10
    P = oracle_mod.Problem3(n, n, n, _medium(n, 1), c_ref=1.0, periodic=True, tau=0.8)
    g = np.random.default_rng(2).normal(size=(7, n, n, n))
    g2, _ = oracle_mod.run3(P, g, 25)
    assert abs(g2.sum() - g.sum()) < 1e-12 * np.abs(g).sum()
    j0 = V7.T @ g.reshape(7, -1).sum(axis=1)
    j1 = V7.T @ g2.reshape(7, -1).sum(axis=1)
    assert np.abs(j1 - j0).max() < 1e-12 * np.abs(g).sum()


def test_d3q7_half_is_leapfrog_in_heterogeneous_medium(oracle_mod):
    n, steps = 12, 40
    rng = np.random.default_rng(9)
    c = _medium(n, 13)
    S = rng.normal(size=steps)
    xs, ys, zs = 3, 7, 5
    P = oracle_mod.Problem3(n, n, n, c, c_ref=1.0, periodic=True, tau=0.5, source=(xs, ys, zs, S))
    g = rng.normal(size=(7, n, n, n))
    rhos = [g.sum(0)]
    for t in range(steps):
        g, _ = oracle_mod.run3(P, g, 1, t0=t)
        rhos.append(g.sum(0))
    eta2 = c.astype(np.float64) ** 2
    w0, w1 = 1 - eta2, eta2 / 6
    sig = np.zeros((n, n, n))
    sig[zs, ys, xs] = w0[zs, ys, xs]
    for dx, dy, dz in V7[1:]:
        sig[(zs + dz) % n, (ys + dy) % n, (xs + dx) % n] += w1[zs, ys, xs]
    err = 0.0
    for t in range(1, steps):
        r, rm = rhos[t], rhos[t - 1]
        lap = sum(np.roll(2 * w1 * r, (dz, dy, dx), axis=(0, 1, 2)) for dx, dy, dz in V7[1:])
        pred = 2 * w0 * r + lap - rm + sig * S[t]
        pred[zs, ys, xs] -= S[t - 1]
        err = max(err, np.abs(pred - rhos[t + 1]).max() / np.abs(rhos[t + 1]).max())
    assert err < 1e-12


def _amplification3(oracle_mod, P, kidx):
    """One-step map of the oracle for grid wave vector kidx, column by column."""
    n = P.nx
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    phase = 2 * np.pi * (kidx[0] * x + kidx[1] * y + kidx[2] * z) / n
    T = np.zeros((7, 7), complex)
    for q in range(7):
        gc, gs = np.zeros((7, n, n, n)), np.zeros((7, n, n, n))
        gc[q], gs[q] = np.cos(phase), np.sin(phase)
        rc, _ = oracle_mod.run3(P, gc, 1)
        rs, _ = oracle_mod.run3(P, gs, 1)
        T[:, q] = ((rc + 1j * rs) * np.exp(-1j * phase)[None]).reshape(7, -1).mean(axis=1)
    return T


@pytest.mark.parametrize("eta", [1.0, 0.6])
@pytest.mark.parametrize("kidx", [(1, 0, 0), (1, 1, 0), (1, 2, 3), (4, 4, 4)])
def test_d3q7_half_dispersion_closed_form(oracle_mod, eta, kidx):
    n = 8
    P = oracle_mod.Problem3(n, n, n, np.full((n, n, n), eta, np.float32), c_ref=1.0,
                            periodic=True, tau=0.5)
    T = _amplification3(oracle_mod, P, kidx)
    cs2 = float(np.float32(eta)) ** 2 / 3
    k = 2 * np.pi * np.array(kidx) / n
    w = 2 * np.arcsin(np.sqrt(cs2 * np.sum(np.sin(k / 2) ** 2)))
    for target in (np.exp(1j * w), np.exp(-1j * w), -1.0):
        assert np.linalg.svd(T - target * np.eye(7), compute_uv=False)[-1] < 1e-13
    np.testing.assert_allclose(np.abs(np.linalg.eigvals(T)), 1.0, atol=1e-7)


def _energy(g, eta):
    w = np.array([1 - eta ** 2] + [eta ** 2 / 6] * 6)
    return float((g ** 2 / w[:, None, None, None]).sum())


def test_energy_conserved_at_half_and_decays_above(oracle_mod):
    n, eta = 8, np.float32(0.8)
    c = np.full((n, n, n), eta, np.float32)
    g = np.random.default_rng(4).normal(size=(7, n, n, n))
    e0 = _energy(g, float(eta))
    P = oracle_mod.Problem3(n, n, n, c, c_ref=1.0, periodic=True, tau=0.5)
    g1, _ = oracle_mod.run3(P, g, 50)
    assert abs(_energy(g1, float(eta)) - e0) < 1e-12 * e0
    P = oracle_mod.Problem3(n, n, n, c, c_ref=1.0, periodic=True, tau=0.9)
    e = [e0]
    gg = g
    for _ in range(5):
        gg, _ = oracle_mod.run3(P, gg, 10)
        e.append(_energy(gg, float(eta)))
    assert all(b < a for a, b in zip(e, e[1:]))


def test_receivers_sponge_and_zero_ghost(oracle_mod):
    # receivers record p = c_s^2 rho of the state entering each step; with a zero ghost and
    # a sponge the total mass only decreases once the pulse reaches the sponge
    n, steps = 16, 30
    c = _medium(n, 6, 0.5, 1.0)
    rec = np.array([[8, 8, 8], [2, 5, 9]], np.int32)
    P = oracle_mod.Problem3(n, n, n, c, c_ref=1.0, tau=0.6, sponge_width=3,
                            sponge_sigma_max=0.2, receivers=rec)
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    p0 = np.exp(-((x - 8) ** 2 + (y - 8) ** 2 + (z - 8) ** 2) / 4.0)
    g = oracle_mod.init_pressure3(P, p0)
    np.testing.assert_allclose(oracle_mod.pressure3(P, g), p0, rtol=1e-12, atol=1e-15)
    g1, tr = oracle_mod.run3(P, g, steps)
    assert tr.shape == (steps, 2) and abs(tr[0, 0] - p0[8, 8, 8]) < 1e-12
    g2, _ = oracle_mod.run3(P, g, 1)
    np.testing.assert_allclose(tr[1], oracle_mod.pressure3(P, g2)[rec[:, 2], rec[:, 1], rec[:, 0]],
                               rtol=1e-12)
    assert g1.sum() < g.sum()
