"""Linear stability of a configuration (Sec. 3's single-mode analysis; Sec. 2.3), on the host.

lb_stability_radius computes max |lambda| of the one-step map T(k) = D(k)(I - C A) over a
grid of wave vectors with its own eigenvalue routine; here it is held to numpy's
eigenvalues of the same map built independently from the printed pieces (tests/lbspec.py:
App. A's M from tests/golden, A from its printed form).  lb_create runs the same check for
D2Q9 and MRT configurations and refuses an unstable one before any CUDA call, so all of
this runs without a GPU.
"""
import numpy as np
import pytest

from tests import lbspec


@pytest.fixture(scope="module")
def lib():
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300 import lbac
    return lbac


def weights(Q, eta, w_ref):
    e2 = eta * eta
    if Q == 5:
        return np.array([1 - e2] + [e2 / 4] * 4), e2 / 2
    w1, w5 = e2 * w_ref[1], e2 * w_ref[2]
    return np.array([1 - 4 * (w1 + w5)] + [w1] * 4 + [w5] * 4), e2 * (2 * w_ref[1] + 4 * w_ref[2])


def numpy_radius(Q, mrt, tau, s, eta, w_ref, nk):
    w, cs2 = weights(Q, eta, w_ref)
    r = 0.0
    for m in range(nk):
        for n in range(nk):
            k = 2 * np.pi * np.array([m, n]) / nk
            T = lbspec.amplification(Q, k, w, cs2, mrt=mrt, tau=tau, s=s)
            r = max(r, np.abs(np.linalg.eigvals(T)).max())
    return r


def config(lib, Q, mrt, tau, s, w_ref):
    cfg = lib.lb_config_default()
    cfg.lattice = Q
    cfg.collision = lib.LB_MRT if mrt else lib.LB_BGK
    cfg.tau = tau
    for k, v in enumerate(s or []):
        cfg.s[k] = v
    for k in range(3):
        cfg.w_ref[k] = w_ref[k]
    return cfg


# stable and unstable choices: the lossless settings, seeded MRT rates, and D2Q9 rate /
# weight draws whose one-step map has an eigenvalue outside the unit circle
CASES = [
    (5, False, 0.5, None, (4 / 9, 1 / 9, 1 / 36), 0.8),
    (5, False, 1.0, None, (4 / 9, 1 / 9, 1 / 36), 1.0),
    (5, True, 0.5, [1.2, 0.9, 0.9, 1.3, 0.7], (4 / 9, 1 / 9, 1 / 36), 0.6),
    (9, False, 0.5, None, (4 / 9, 1 / 9, 1 / 36), 1.0),
    (9, False, 0.5, None, (0.0, 0.01, 0.24), 0.9),
    (9, True, 0.5, [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3], (0.4, 0.11, 0.04), 0.8),
    (9, True, 0.5, [1.89, 0.44, 0.44, 0.1, 0.37, 1.77, 1.59, 1.59, 0.48], (0.42, 0.139, 0.006), 1.0),
    (9, True, 0.5, [1.36, 1.31, 1.31, 0.8, 1.99, 1.96, 1.39, 1.39, 1.39], (0.53, 0.097, 0.0205), 1.0),
]


@pytest.mark.parametrize("Q,mrt,tau,s,w_ref,eta", CASES)
def test_radius_matches_numpy_eigenvalues(lib, Q, mrt, tau, s, w_ref, eta):
    nk = 16
    got = lib.lb_stability_radius(config(lib, Q, mrt, tau, s, w_ref), eta, 0, nk)
    ref = numpy_radius(Q, mrt, tau, s, eta, w_ref, nk)
    assert abs(got - ref) <= 1e-12 * max(1.0, ref), (got, ref)


def test_lossless_and_dissipative_settings_are_stable(lib):
    # tau = 1/2 conserves the energy norm (radius 1); tau > 1/2 damps but the conserved
    # k = 0 modes keep eigenvalue 1
    for Q, w_ref in ((5, (4 / 9, 1 / 9, 1 / 36)), (9, (4 / 9, 1 / 9, 1 / 36)), (9, (0, 0.01, 0.24))):
        for tau in (0.5, 0.7, 1.5):
            for eta in (0.3, 1.0):
                r = lib.lb_stability_radius(config(lib, Q, False, tau, None, w_ref), eta, 0, 64)
                assert abs(r - 1.0) < 1e-12, (Q, w_ref, tau, eta, r)


def test_unstable_d2q9_rates_are_found(lib):
    cfg = config(lib, 9, True, 0.5, [1.89, 0.44, 0.44, 0.1, 0.37, 1.77, 1.59, 1.59, 0.48],
                 (0.42, 0.139, 0.006))
    assert lib.lb_stability_radius(cfg, 1.0, 0, 64) > 1.1


def test_refinement_levels_use_the_viscous_rates(lib):
    # level l relaxes with tau_l - 1/2 = 2^l (tau - 1/2): its radius is that configuration's
    s = [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3]
    w = (0.4, 0.11, 0.04)
    for level in (1, 2):
        s_l = [1.0 / (0.5 + 2 ** level * (1.0 / v - 0.5)) for v in s]
        a = lib.lb_stability_radius(config(lib, 9, True, 0.5, s, w), 0.7, level, 16)
        b = numpy_radius(9, True, 0.5, s_l, 0.7, w, 16)
        assert abs(a - b) <= 1e-12


def _cfg_with_map(lib, Q, mrt, s, w_ref, c):
    cfg = config(lib, Q, mrt, 0.5, s, w_ref)
    cfg.ny, cfg.nx = c.shape
    cfg.c_map = c.ctypes.data_as(lib.ctypes.POINTER(lib.ctypes.c_float))
    cfg.c_ref = 1.0
    return cfg


def test_create_refuses_an_unstable_scheme_without_gpu(lib):
    # an unstable D2Q9 MRT choice is refused by lb_create before it touches the GPU, and the
    # message names the radius and the eta where it was found
    c = np.full((16, 24), 1.0, np.float32)
    cfg = _cfg_with_map(lib, 9, True, [1.89, 0.44, 0.44, 0.1, 0.37, 1.77, 1.59, 1.59, 0.48],
                        (0.42, 0.139, 0.006), c)
    with pytest.raises(lib.LBError) as e:
        lib.lb_create(cfg)
    assert e.value.status == lib.LB_EINVAL
    msg = lib.lb_last_error(None)
    assert "unstable" in msg and "eta = 1" in msg


def test_create_checks_the_speeds_of_the_medium(lib):
    # a layered map with two speeds: the refusal names one of the map's own eta values
    s = [1.89, 0.44, 0.44, 0.1, 0.37, 1.77, 1.59, 1.59, 0.48]
    w = (0.42, 0.139, 0.006)
    c = np.full((20, 16), 0.5, np.float32)
    c[15:] = 0.75
    with pytest.raises(lib.LBError):
        lib.lb_create(_cfg_with_map(lib, 9, True, s, w, c))
    msg = lib.lb_last_error(None)
    assert "unstable" in msg and ("eta = 0.5 " in msg or "eta = 0.75 " in msg), msg
    # stable rates on the same map pass the check (and then fail only for want of a GPU)
    c2 = np.full((20, 16), 0.5, np.float32)
    cfg = _cfg_with_map(lib, 9, True, [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3],
                        (0.4, 0.11, 0.04), c2)
    try:
        lib.lb_destroy(lib.lb_create(cfg))
    except lib.LBError:
        assert "unstable" not in lib.lb_last_error(None)


@pytest.mark.parametrize("nspeeds", [3, 12])
def test_large_maps_are_scanned_like_small_ones(lib, nspeeds):
    # a map of millions of sites is scanned on several host threads, band by band; the
    # speeds it reports to the stability check (the distinct ones up to 8, else the range)
    # and so the refusal are those of a small map holding the same speeds in the same order
    s = [1.89, 0.44, 0.44, 0.1, 0.37, 1.77, 1.59, 1.59, 0.48]
    w = (0.42, 0.139, 0.006)
    speeds = np.linspace(0.45, 0.8, nspeeds).astype(np.float32)
    msgs = []
    for ny, nx in ((2048, 2048), (nspeeds, 8)):
        c = np.empty((ny, nx), np.float32)
        for k, band in enumerate(np.array_split(np.arange(ny), nspeeds)):
            c[band] = speeds[k]               # each speed in its own band of rows
        with pytest.raises(lib.LBError) as e:
            lib.lb_create(_cfg_with_map(lib, 9, True, s, w, c))
        assert e.value.status == lib.LB_EINVAL
        msgs.append(lib.lb_last_error(None))
    assert "unstable" in msgs[0] and msgs[0] == msgs[1], msgs


def test_bad_arguments(lib):
    cfg = config(lib, 5, False, 0.5, None, (4 / 9, 1 / 9, 1 / 36))
    for eta, level, nk in ((0.0, 0, 16), (1.2, 0, 16), (0.5, -1, 16), (0.5, 0, 1)):
        with pytest.raises(lib.LBError):
            lib.lb_stability_radius(cfg, eta, level, nk)
