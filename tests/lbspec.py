"""Fourier-space (dispersion) description of the linear LB scheme, for the tests.

Independent of the oracle's stepper: it builds the one-step amplification
matrix of Sec. 3.2 directly from the paper's printed pieces,

    exp(-i omega) g = D(k) (I - M^-1 S M A) g,   D(k) = diag(exp(-i k.c_j))

(Eq. MRT-LB dispersion; the collide-then-stream order, which has the same
eigenvalues as the printed stream-then-collide order), with M read from the
golden fixtures of App. A and A from its printed form A_ij = delta_ij -
w_i (1 + c_i.c_j / c_s^2) (Eq. D2Q5/D2Q9 dist to eqm dist and the A matrix).
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

C5 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1]])
C9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])


def golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def lattice(Q):
    return C5 if Q == 5 else C9


def moment_matrix(Q):
    return golden("appA_M_d2q5.txt" if Q == 5 else "appA_M_d2q9.txt")


def a_matrix(Q, w, cs2):
    c = lattice(Q)
    w = np.asarray(w, dtype=np.float64)
    return np.eye(Q) - w[:, None] * (1.0 + (c @ c.T) / cs2)


def collision_matrix(Q, mrt, tau, s):
    """C = M^-1 S M (MRT) or I / tau (BGK)."""
    if not mrt:
        return np.eye(Q) / tau
    M = moment_matrix(Q)
    return np.linalg.solve(M, np.diag(np.asarray(s[:Q], dtype=np.float64)) @ M)


def amplification(Q, k, w, cs2, mrt=False, tau=0.5, s=None):
    """T(k) = D(k) (I - C A) for a wave vector k = (kx, ky) (radians per cell)."""
    c = lattice(Q)
    D = np.diag(np.exp(-1j * (c @ np.asarray(k, dtype=np.float64))))
    C = collision_matrix(Q, mrt, tau, s if s is not None else [1.0] * Q)
    return D @ (np.eye(Q) - C @ a_matrix(Q, w, cs2))


def d2q5_closed_form_omega(k, cs2):
    """Propagating root of the D2Q5, tau = 1/2 scheme.

    sin^2(omega/2) = c_s^2 [sin^2(kx/2) + sin^2(ky/2)]: the App. E root
    omega = 2 arcsin(c_s sin(k/2)) along theta = 0, extended to 2-D (it is the
    second-order leapfrog relation of App. C at Courant number c_s).
    """
    kx, ky = k
    return 2.0 * np.arcsin(np.sqrt(cs2 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2)))


def measured_amplification(oracle, P, k_index):
    """Column-by-column one-step map of the oracle for one grid wave vector.

    P must be a homogeneous periodic oracle.Problem without source/sponge.
    Column q of T(k) is the k-th Fourier coefficient of the response to
    g_i(x) = delta_iq exp(i k.x) (assembled from the cos and sin responses).
    """
    mx, my = k_index
    Q, nx, ny = P.Q, P.nx, P.ny
    y, x = np.mgrid[0:ny, 0:nx]
    phase = 2 * np.pi * (mx * x / nx + my * y / ny)
    T = np.zeros((Q, Q), dtype=complex)
    for q in range(Q):
        gc = np.zeros((Q, ny, nx))
        gs = np.zeros((Q, ny, nx))
        gc[q] = np.cos(phase)
        gs[q] = np.sin(phase)
        rc, _ = oracle.run(P, gc, 1)
        rs, _ = oracle.run(P, gs, 1)
        z = rc + 1j * rs
        T[:, q] = (z * np.exp(-1j * phase)[None]).reshape(Q, -1).mean(axis=1)
    return T


def exact_evolution(g0, Q, w, cs2, nsteps, mrt=False, tau=0.5, s=None):
    """Per-Fourier-mode exact solution g_hat(k, n) = T(k)^n g_hat(k, 0) on a periodic grid."""
    _, ny, nx = g0.shape
    G = np.fft.fft2(g0, axes=(1, 2))
    out = np.zeros_like(G)
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    KX, KY = np.meshgrid(kx, ky)
    ks = np.stack([KX.ravel(), KY.ravel()], axis=1)
    c = lattice(Q)
    C = collision_matrix(Q, mrt, tau, s if s is not None else [1.0] * Q)
    K = np.eye(Q) - C @ a_matrix(Q, w, cs2)
    D = np.exp(-1j * (ks @ c.T))                       # [nk, Q]
    T = D[:, :, None] * K[None, :, :]                  # [nk, Q, Q]
    Tn = np.linalg.matrix_power(T, nsteps)
    gk = G.reshape(Q, -1).T                            # [nk, Q]
    res = np.einsum("kij,kj->ki", Tn, gk)
    out = res.T.reshape(Q, ny, nx)
    return np.real(np.fft.ifft2(out, axes=(1, 2)))
