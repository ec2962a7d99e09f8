"""Host logic of the dispersion diagnostics: the matrix pencil fit recovers known poles
and amplitudes (no GPU)."""
import numpy as np

from paper_1704_03172_gb300.dispersion import acoustic_pole, matrix_pencil


def test_matrix_pencil_recovers_poles_and_amplitudes():
    rng = np.random.default_rng(0)
    poles = np.array([np.exp(0.3j) * 0.999, np.exp(-0.3j) * 0.999, 0.95, -0.7 + 0.1j])
    amps = np.array([1.0 + 0.5j, 0.8 - 0.2j, 0.3, 0.05j])
    t = np.arange(200)
    z = (amps[None, :] * poles[None, :] ** t[:, None]).sum(axis=1)
    z = z + 1e-9 * (rng.normal(size=z.shape) + 1j * rng.normal(size=z.shape))
    p, a = matrix_pencil(z, max_order=5)
    assert len(p) == 4
    for pk, ak in zip(poles, amps):
        j = np.argmin(np.abs(p - pk))
        assert abs(p[j] - pk) < 1e-8 and abs(a[j] - ak) < 1e-6
    lam = acoustic_pole(p, a)
    assert abs(lam - poles[0]) < 1e-8


def test_matrix_pencil_order_is_capped():
    t = np.arange(100)
    z = sum(np.exp(1j * w * t) for w in (0.1, 0.4, 0.9, 1.3))
    p, _ = matrix_pencil(z, max_order=3)
    assert len(p) == 3
