"""Pin of the oracle against the 2-D free-space Green's function (Sec. 5.1, Eq. exact solution).

A point source with the paper's wavelet (Eq. source) in a homogeneous medium:
the time-domain solution of (1/c^2) p_tt - lap p = dS/dt delta(x - x_s) is

    p(r, t) = (c / pi) int_0^inf  S'(t - r/c - u^2) / sqrt(c (2 r + c u^2)) du

(the 2-D Green's function c H(ct - r) / (2 pi sqrt(c^2 t^2 - r^2)) convolved with
S', after the substitution t - t' = r/c + u^2 that removes the singularity).
D2Q5 with tau = 1/2 and w_0 = 0 has no dispersion along theta = 45 deg (Sec. 3.2),
so there the LB trace must converge to this solution at second order in 1/R.
"""
import math

import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W

_trapz = getattr(np, "trapezoid", None) or getattr(np, "trapz")


def _wavelet_rate(t, fc):
    a = 2 * math.pi * fc / 3
    xi = a * (t - 1.5 / fc)
    e = np.exp(-2 * xi * xi)
    return a * (8 * xi * e + 4 * xi * (1 - 4 * xi * xi) * e)    # d/dt of -(1 - 4 xi^2) e^{-2 xi^2}


def _analytic(r, c, ts, fc):
    u = np.linspace(0.0, 60.0, 120001)
    out = np.empty(len(ts))
    for k, t in enumerate(ts):
        f = _wavelet_rate(t - r / c - u * u, fc) / np.sqrt(c * (2 * r + c * u * u))
        out[k] = (c / math.pi) * _trapz(f, u)
    return out


def test_wavelet_rate_is_derivative():
    fc = 0.005
    t = np.arange(600, dtype=np.float64)
    num = np.gradient(W.ricker(600, fc), t)          # central differences of Eq. source
    ref = _wavelet_rate(t, fc)
    assert np.abs(num - ref).max() < 1e-3 * np.abs(ref).max()


def _trace_error(oracle, R, r_wavelengths=6):
    n = 24 * R
    c = 1 / math.sqrt(2)            # eta = 1, w_0 = 0: c_s^2 = 1/2
    fc = c / R                      # R points per central wavelength
    xs = ys = n // 2
    d = int(round(r_wavelengths * R / math.sqrt(2)))
    rec = np.array([[xs + d, ys + d]], dtype=np.int32)
    r = d * math.sqrt(2)
    steps = int(r / c + 3 / fc + 20)
    P = oracle.Problem(5, n, n, W.uniform_map(n, n, 1.0), c_ref=1.0, tau=0.5,
                       source=(xs, ys, W.ricker(steps, fc)), receivers=rec)
    _, tr = oracle.run(P, P.zeros(), steps)
    a = _analytic(r, c, np.arange(steps), fc)
    return np.linalg.norm(tr[:, 0] - a) / np.linalg.norm(a)


@pytest.mark.slow
def test_point_source_converges_to_greens_function(oracle_mod):
    e16 = _trace_error(oracle_mod, 16)
    e32 = _trace_error(oracle_mod, 32)
    assert e16 < 0.03
    assert e32 < 0.008
    assert e16 / e32 > 3.0          # second-order convergence
