"""Dispersion diagnostics on the GPU: the single-mode analysis of Sec. 3.

On a periodic homogeneous grid every Fourier mode k = 2 pi (mx / n, my / n)
of the populations evolves on its own under the one-step amplification matrix
T(k) = D(k)(I - C A) of Eq. MRT-LB dispersion.  A run started from a
superposition of pressure modes (equilibrium populations, zero velocity) is
therefore a batch of single-mode runs in one launch stream: the GPU steps the
grid and projects the pressure onto every mode in FP64 after each step
(``lb_mode_projection``).  Each mode's time series is a sum of powers of the
eigenvalues of T(k) that the initial state excites; the matrix pencil method
(Hua and Sarkar, IEEE Trans. ASSP 38, 1990) recovers them.  The travelling
acoustic pair gives the measured phase speed arg(lambda) / |k| and the damping
|lambda| per step -- the quantities of the paper's Fig. 3 (angle, lattice,
collision) and Fig. 4 (D2Q9 weights).

Only the fit of a few hundred complex samples per mode runs on the host.
"""
from __future__ import annotations

import math

import numpy as np


def mode_series(modes, n, steps, *, lattice=5, collision="bgk", tau=0.5, s=None, eta=1.0,
                w_ref=(4 / 9, 1 / 9, 1 / 36), storage="f32"):
    """Projections P_m(t) = sum_x p(x, t) exp(-i k_m . x), t = 0..steps, of a periodic n x n
    run with c / c_ref = eta started from p0 = sum_m cos(k_m . x).  Returns [steps + 1, M]."""
    from . import lbac
    from .sim import LBSim
    modes = [(int(a), int(b)) for a, b in modes]
    y, x = np.mgrid[0:n, 0:n]
    p0 = np.zeros((n, n), np.float64)
    for mx, my in modes:
        p0 += np.cos(2.0 * np.pi * (mx * x + my * y) / n)
    sim = LBSim(np.full((n, n), eta, np.float32), lattice=lattice, collision=collision, tau=tau,
                s=s, storage=storage, boundary="periodic", c_ref=1.0, w_ref=w_ref)
    try:
        sim.init_pressure(p0.astype(np.float32))
        out = np.zeros((steps + 1, len(modes)), complex)
        for t in range(steps + 1):
            out[t] = lbac.lb_mode_projection(sim.ctx, modes)
            if t < steps:
                sim.step(1)
    finally:
        sim.close()
    return out


def matrix_pencil(z, max_order, rel_tol=1e-6):
    """Poles lambda_j and amplitudes a_j with z[t] ~ sum_j a_j lambda_j^t (matrix pencil:
    Hankel matrix of the samples, its dominant right singular vectors, and the eigenvalues
    of the shifted pencil).  The model order is the number of singular values above
    rel_tol times the largest, at most max_order."""
    z = np.asarray(z, complex)
    N = len(z)
    L = N // 2
    Y = np.array([z[i:i + L + 1] for i in range(N - L)])
    _, sv, Vh = np.linalg.svd(Y, full_matrices=False)
    M = int(min(max_order, np.count_nonzero(sv > rel_tol * sv[0])))
    # the rows of Y are combinations of (lambda_j^0 .. lambda_j^L): the first M rows of Vh
    # span that space, and shifting by one sample multiplies each basis vector by lambda_j
    V = Vh[:M].T
    poles = np.linalg.eigvals(np.linalg.pinv(V[:-1]) @ V[1:])
    Z = poles[None, :] ** np.arange(N)[:, None]
    amps = np.linalg.lstsq(Z, z, rcond=None)[0]
    return poles, amps


def fit_modes(series, max_order, skip=2):
    """Poles and amplitudes of every mode's series (the first `skip` samples are left out:
    poles at or near 0 -- modes a collision removes at once -- are not resolvable)."""
    return [matrix_pencil(series[skip:, m], max_order) for m in range(series.shape[1])]


def acoustic_pole(poles, amps):
    """The travelling acoustic pole: the largest-amplitude pole with arg > 0."""
    cand = [(abs(a), p) for p, a in zip(poles, amps) if np.angle(p) > 1e-9]
    return max(cand, key=lambda t: t[0])[1] if cand else None


def phase_speed(modes, n, steps, *, lattice=5, eta=1.0, w_ref=(4 / 9, 1 / 9, 1 / 36), **kw):
    """Per mode: points per wavelength, measured phase speed / c_s (lattice units) and
    damping |lambda| per step of the acoustic branch."""
    series = mode_series(modes, n, steps, lattice=lattice, eta=eta, w_ref=w_ref, **kw)
    fits = fit_modes(series, lattice)
    cs2 = eta * eta * (0.5 if lattice == 5 else 2 * w_ref[1] + 4 * w_ref[2])
    rows = []
    for (mx, my), (poles, amps) in zip(modes, fits):
        k = 2.0 * math.pi * math.hypot(mx, my) / n
        lam = acoustic_pole(poles, amps)
        rows.append({"mode": (mx, my), "ppw": 2.0 * math.pi / k,
                     "theta_deg": math.degrees(math.atan2(my, mx)),
                     "phase_speed_ratio": float(np.angle(lam) / k / math.sqrt(cs2)),
                     "damping": float(abs(lam))})
    return rows
