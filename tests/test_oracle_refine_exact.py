"""Exact pins of the refinement oracle's transfer functions (Sec. 4).

What the paper fixes about the coupling of two grids (Eq. grid refinement eqm dist, Eq.
coarse-fine dist connect): the equilibrium part of a transferred population vector is
shared, computed from the vector's own moments with the receiving grid's weights, and
only the non-equilibrium part is scaled, by 1/n from coarse to fine and by n from fine
to coarse (n = 2, tau = 1/2).  Reading R6 carries this to tau != 1/2 moment by moment;
reading R4 interpolates linearly in time (the midpoint at odd fine times) and along the
interface in space.

Each test here fixes one of these pieces exactly, with expected values built in the test
from the printed pieces alone (the App. A moment matrix from tests/golden, the weight
rule of Eq. 0th lattice weight, the linear equilibrium), not from the oracle:

- a transferred vector keeps rho and j exactly;
- at tau = 1/2 the non-equilibrium factors are exactly 1/2 and 2;
- for tau != 1/2 they are tau_f / (2 tau_c) and its inverse, per relaxed moment (R6);
- coarse -> fine -> coarse at a node the grids share returns the vector;
- the coarse -> fine transfer writes, at the fine interface nodes and for exactly the
  populations that enter the fine grid, the transfer of the coarse snapshots
  interpolated linearly in space and time (corners included);
- the fine -> coarse correction writes exactly the populations whose upstream node lies
  strictly inside the patch;
- a whole refined run (two levels and nested) carries an exact discrete solution of the
  LB scheme -- fields linear in space and time -- across the interface to rounding.

The last pin rests on a property of the scheme itself: for rho = rho0 + a.x + b t and
j = j0 + B x - c_s^2 a t with trace(B) = -b (a solution of the linear acoustic equations
whose second derivatives vanish), the state g = g^eq(rho, j) + h with the constant
h = -tau D g^eq, D g^eq_i = g^eq_i(x + c_i, t + 1) - g^eq_i(x, t), solves Eq. BGK-LB
exactly (MRT: h = -M^-1 S^-1 M D g^eq).  On a grid refined by 2, D g^eq halves, so the
fine grid's exact state is the coarse one with its non-equilibrium part scaled by
tau_f / (2 tau_c): precisely the transfer of Eq. coarse-fine dist connect under R6.
A swapped 1/n and n, an interpolation at the wrong fine time level, a wrong corner rule
or a missing population all break it.
"""
import numpy as np
import pytest

from paper_1704_03172_gb300 import workloads as W
from tests import lbspec

# the medium is FP32 (as both the oracle and the CUDA path receive it): eta = float32(0.8)
ETA = float(np.float32(0.8))


def weights(Q, eta, w_ref=(0.4, 0.11, 0.04)):
    """Eq. 0th lattice weight (D2Q5) and reading A9 (D2Q9): w_i and c_s^2 at eta."""
    e2 = eta * eta
    if Q == 5:
        return np.array([1 - e2] + [e2 / 4] * 4), e2 / 2
    w1, w5 = e2 * w_ref[1], e2 * w_ref[2]
    return np.array([1 - 4 * (w1 + w5)] + [w1] * 4 + [w5] * 4), e2 * (2 * w_ref[1] + 4 * w_ref[2])


def geq_printed(Q, w, cs2, g):
    """g^eq = (I - A) g with the printed A_ij = delta_ij - w_i (1 + c_i.c_j / c_s^2)."""
    return (np.eye(Q) - lbspec.a_matrix(Q, w, cs2)) @ g


def fine_tau(tau):
    return 0.5 + 2.0 * (tau - 0.5)


def problem(oracle, Q, n, eta=ETA, mrt=False, tau=0.5, s=None, medium="uniform", seed=1):
    c = (W.uniform_map(n, n, eta) if medium == "uniform"
         else W.random_medium(n, n, seed, 0.5, 1.0))
    return oracle.Problem(Q, n, n, c, c_ref=1.0, mrt=mrt, tau=tau, s=s, w_ref=(0.4, 0.11, 0.04))


CASES = [  # Q, mrt, tau, s
    (5, False, 0.5, None),
    (5, False, 0.8, None),
    (5, True, 0.5, [1.2, 0.9, 0.9, 2.0, 2.0]),
    (5, True, 0.5, [1.2, 0.9, 0.9, 1.3, 0.7]),
    (9, False, 0.5, None),
    (9, False, 0.65, None),
    (9, True, 0.5, [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3]),
]


def _rates(Q, mrt, tau, s):
    """relaxation time of every moment (BGK: tau for all)"""
    return np.array([1.0 / v for v in s[:Q]]) if mrt else np.full(Q, tau)


# ------------------------------------------------------------------ single vectors --

@pytest.mark.parametrize("Q,mrt,tau,s", CASES)
def test_transfer_keeps_rho_and_j(oracle_mod, Q, mrt, tau, s):
    P = problem(oracle_mod, Q, 24, mrt=mrt, tau=tau, s=s, medium="random")
    R = oracle_mod.Refined(P, 5, 6, 9, 8)
    c = lbspec.lattice(Q)
    rng = np.random.default_rng(Q + 7)
    for to_fine, (ax, ay) in ((1, (0, 3)), (1, (7, 0)), (1, (18, 16)), (0, (5, 9)), (0, (14, 6))):
        g = rng.normal(size=Q)
        out = R.transfer(1, to_fine, ax, ay, g)
        scale = np.abs(g).sum()
        assert abs(out.sum() - g.sum()) <= 1e-15 * scale
        np.testing.assert_allclose(c.T @ out, c.T @ g, rtol=0, atol=1e-15 * scale)
        assert np.abs(out - g).max() > 1e-3 * scale       # the non-equilibrium part changed


@pytest.mark.parametrize("Q,mrt,s", [(5, False, None), (5, True, [1.2, 0.9, 0.9, 2.0, 2.0]),
                                     (9, False, None), (9, True, [0.7, 1.0, 1.0] + [2.0] * 6)])
def test_factors_are_one_half_and_two_at_tau_half(oracle_mod, Q, mrt, s):
    # tau = 1/2 (MRT: every relaxed rate 2): g^f = g^eq + (g - g^eq) / 2 and
    # g^c = g^eq + 2 (g - g^eq), g^eq from the printed A with the receiving node's weights
    n = 24
    P = problem(oracle_mod, Q, n, mrt=mrt, tau=0.5, s=s, medium="random", seed=3)
    R = oracle_mod.Refined(P, 4, 5, 10, 9)
    cf = R.fine_cmap().astype(np.float64)
    rng = np.random.default_rng(11)
    for ax, ay in ((0, 0), (3, 0), (20, 7), (11, 18)):
        g = rng.normal(size=Q)
        w, cs2 = weights(Q, cf[ay, ax])
        eq = geq_printed(Q, w, cs2, g)
        np.testing.assert_allclose(R.transfer(1, 1, ax, ay, g), eq + 0.5 * (g - eq),
                                   rtol=0, atol=1e-14 * np.abs(g).max())
    cc = P.c_map.astype(np.float64)
    for X, Y in ((4, 5), (9, 14), (14, 10)):
        g = rng.normal(size=Q)
        w, cs2 = weights(Q, cc[Y, X])
        eq = geq_printed(Q, w, cs2, g)
        np.testing.assert_allclose(R.transfer(1, 0, X, Y, g), eq + 2.0 * (g - eq),
                                   rtol=0, atol=1e-14 * np.abs(g).max())


@pytest.mark.parametrize("Q,mrt,tau,s", [c for c in CASES if c[2] != 0.5 or c[1]])
def test_factors_follow_the_viscous_rule_moment_by_moment(oracle_mod, Q, mrt, tau, s):
    # reading R6: tau_f - 1/2 = 2 (tau_c - 1/2) and the non-equilibrium moments scale by
    # tau_f / (2 tau_c) coarse -> fine and 2 tau_c / tau_f fine -> coarse
    P = problem(oracle_mod, Q, 20, mrt=mrt, tau=tau, s=s)
    R = oracle_mod.Refined(P, 4, 4, 8, 8)
    M = lbspec.moment_matrix(Q)
    tc = _rates(Q, mrt, tau, s)
    tf = fine_tau(tc)
    w, cs2 = weights(Q, ETA)
    rng = np.random.default_rng(5)
    for to_fine, node, fac in ((1, (0, 5), tf / (2 * tc)), (0, (4, 9), 2 * tc / tf)):
        g = rng.normal(size=Q)
        eq = geq_printed(Q, w, cs2, g)
        m_in = M @ (g - eq)
        m_out = M @ (R.transfer(1, to_fine, *node, g) - eq)
        np.testing.assert_allclose(m_out[3:], fac[3:] * m_in[3:], rtol=0,
                                   atol=1e-14 * np.abs(g).max())
        np.testing.assert_allclose(m_out[:3], 0.0, rtol=0, atol=1e-14 * np.abs(g).max())


@pytest.mark.parametrize("Q,mrt,tau,s", CASES)
def test_coarse_to_fine_to_coarse_returns_the_vector(oracle_mod, Q, mrt, tau, s):
    # at a node the two grids share, both sides have the same weights, so the two
    # rescalings (factors f and 1/f) around the same g^eq cancel
    P = problem(oracle_mod, Q, 24, mrt=mrt, tau=tau, s=s, medium="random", seed=4)
    R = oracle_mod.Refined(P, 5, 6, 9, 8)
    rng = np.random.default_rng(17)
    for a, b in ((0, 0), (4, 0), (0, 8), (18, 10), (10, 16)):
        G = rng.normal(size=Q)
        back = R.transfer(1, 0, 5 + a // 2, 6 + b // 2, R.transfer(1, 1, a, b, G))
        np.testing.assert_allclose(back, G, rtol=0, atol=1e-14 * np.abs(G).max())


# ------------------------------------------------------------- an exact solution ---

class Linear:
    """Fields linear in space and time (coarse units) and the exact LB state carrying
    them: rho = r0 + a.x + b t, j = j0 + B x - c_s^2 a t, trace(B) = -b."""

    def __init__(self, Q, eta, mrt, tau, s):
        self.Q, self.mrt = Q, mrt
        self.c = lbspec.lattice(Q)
        self.w, self.cs2 = weights(Q, eta)
        self.M = lbspec.moment_matrix(Q)
        self.tau = _rates(Q, mrt, tau, s)
        self.r0, self.a, self.b = 0.3, np.array([0.011, -0.007]), 0.013
        self.j0 = np.array([0.05, -0.02])
        self.B = np.array([[-0.004, 0.002], [0.003, -0.009]])      # trace = -b

    def geq(self, x, y, t):
        rho = self.r0 + self.a[0] * x + self.a[1] * y + self.b * t
        jx = self.j0[0] + self.B[0, 0] * x + self.B[0, 1] * y - self.cs2 * self.a[0] * t
        jy = self.j0[1] + self.B[1, 0] * x + self.B[1, 1] * y - self.cs2 * self.a[1] * t
        cj = self.c[:, 0, None, None] * jx + self.c[:, 1, None, None] * jy
        return self.w[:, None, None] * (rho + cj / self.cs2)

    def state(self, xs, ys, t, h):
        """exact pre-collision state at nodes xs x ys (coarse units, spacing h) at time t
        (coarse steps) on a grid whose cell and step are h coarse ones"""
        X, Y = np.meshgrid(np.asarray(xs, np.float64), np.asarray(ys, np.float64))
        eq = self.geq(X, Y, t)
        # D g^eq_i = g^eq_i(x + h c_i, t + h) - g^eq_i(x, t), constant for linear fields
        D = np.array([self.geq(X[:1, :1] + h * self.c[i, 0], Y[:1, :1] + h * self.c[i, 1],
                               t + h)[i, 0, 0] - eq[i, 0, 0] for i in range(self.Q)])
        tau_h = 0.5 + (self.tau - 0.5) / h                 # reading R6 on a grid of spacing h
        if self.mrt:
            m = self.M @ D
            m[:3] = 0.0                                    # rho and j are conserved
            hneq = -np.linalg.solve(self.M, tau_h * m)
        else:
            hneq = -tau_h * D
        return eq + hneq[:, None, None]


def _fine_nodes(x0, y0, nxp, nyp, h):
    """coarse-unit coordinates of the fine nodes of a patch whose corner sits at (x0, y0)
    (coarse units) on a grid of spacing h"""
    return x0 + h * np.arange(2 * nxp + 1), y0 + h * np.arange(2 * nyp + 1)


@pytest.mark.parametrize("Q,mrt,tau,s", CASES)
def test_coarse_to_fine_interpolates_in_space_and_time(oracle_mod, Q, mrt, tau, s):
    # coarse snapshots of the exact solution at times T and T + 1 on I; the transfer with
    # alpha = 1/2 must write the exact fine state at T + 1/2 (the odd fine time), alpha = 1
    # the one at T + 1, into exactly the populations that enter the fine grid, at every
    # fine node of I (between two coarse nodes and at the corners); nothing else changes
    n, x0, y0, nxp, nyp, T = 30, 8, 7, 10, 12, 3.0
    P = problem(oracle_mod, Q, n, mrt=mrt, tau=tau, s=s)
    R = oracle_mod.Refined(P, x0, y0, nxp, nyp)
    L = Linear(Q, ETA, mrt, tau, s)
    I = R.interface(1)
    xs, ys = np.arange(n), np.arange(n)
    Ua = L.state(xs, ys, T, 1.0)[:, I[:, 1], I[:, 0]].T.copy()
    Ub = L.state(xs, ys, T + 1, 1.0)[:, I[:, 1], I[:, 0]].T.copy()
    nyf, nxf = R.level_dims(1)
    fx, fy = _fine_nodes(x0, y0, nxp, nyp, 0.5)
    c = lbspec.lattice(Q)
    for alpha, t in ((0.5, T + 0.5), (1.0, T + 1.0), (0.0, T)):
        sentinel = np.full((Q, nyf, nxf), 7.0)
        R.set_level_state(1, sentinel)
        R.apply_c2f(1, Ua, Ub, alpha)
        got = R.level_state(1)
        exact = L.state(fx, fy, t, 0.5)
        written = 0
        for i in range(Q):
            for b in range(nyf):
                for a in range(nxf):
                    on_I = a in (0, nxf - 1) or b in (0, nyf - 1)
                    ua, ub = a - c[i, 0], b - c[i, 1]
                    enters = not (0 <= ua < nxf and 0 <= ub < nyf)
                    if on_I and enters:
                        assert abs(got[i, b, a] - exact[i, b, a]) <= 1e-14, (alpha, i, a, b)
                        written += 1
                    else:
                        assert got[i, b, a] == 7.0, (alpha, i, a, b)
        assert written > 0
    # the midpoint matters: alpha = 1/2 differs from both ends by much more than rounding
    R.set_level_state(1, np.zeros((Q, nyf, nxf)))
    R.apply_c2f(1, Ua, Ub, 0.5)
    mid = R.level_state(1)[:, 0, 1:-1]
    assert np.abs(mid - L.state(fx, fy, T + 1.0, 0.5)[:, 0, 1:-1]).max() > 1e-4


@pytest.mark.parametrize("Q,mrt,tau,s", CASES)
def test_fine_to_coarse_corrects_exactly_the_populations_from_inside(oracle_mod, Q, mrt, tau,
                                                                      s):
    n, x0, y0, nxp, nyp, t = 30, 8, 7, 10, 12, 2.5
    P = problem(oracle_mod, Q, n, mrt=mrt, tau=tau, s=s)
    R = oracle_mod.Refined(P, x0, y0, nxp, nyp)
    L = Linear(Q, ETA, mrt, tau, s)
    fx, fy = _fine_nodes(x0, y0, nxp, nyp, 0.5)
    R.set_level_state(1, L.state(fx, fy, t, 0.5))
    R.set_level_state(0, np.full((Q, n, n), -5.0))
    R.apply_f2c(1)
    got = R.level_state(0)
    exact = L.state(np.arange(n), np.arange(n), t, 1.0)
    c = lbspec.lattice(Q)
    I = {tuple(v) for v in R.interface(1)}
    assert len(I) == 2 * (nxp + nyp)
    written = 0
    for i in range(Q):
        for Y in range(n):
            for X in range(n):
                up = (X - c[i, 0], Y - c[i, 1])
                inside = x0 < up[0] < x0 + nxp and y0 < up[1] < y0 + nyp
                if (X, Y) in I and inside:
                    assert abs(got[i, Y, X] - exact[i, Y, X]) <= 1e-14, (i, X, Y)
                    written += 1
                else:
                    assert got[i, Y, X] == -5.0, (i, X, Y)
    assert written > 0


RUNS = [  # Q, mrt, tau, s, nested, coupling
    (5, False, 0.5, None, False, "both"),
    (5, False, 0.8, None, False, "both"),
    (5, True, 0.5, [1.2, 0.9, 0.9, 1.3, 0.7], False, "both"),
    (9, False, 0.5, None, False, "both"),
    (9, True, 0.5, [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3], False, "both"),
    (5, False, 0.7, None, True, "both"),
    (9, True, 0.5, [1.0, 1.0, 1.0, 1.6, 1.3, 1.5, 1.2, 1.2, 1.3], True, "both"),
    (5, False, 0.5, None, False, "c2f"),
]


def _exact_run(oracle_mod, Q, mrt, tau, s, nested, coupling, steps=6):
    n, x0, y0, nxp, nyp = 48, 16, 15, 14, 16
    P = problem(oracle_mod, Q, n, mrt=mrt, tau=tau, s=s)
    R = oracle_mod.Refined(P, x0, y0, nxp, nyp)
    L = Linear(Q, ETA, mrt, tau, s)
    levels = [(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), 1.0)]
    fx, fy = _fine_nodes(x0, y0, nxp, nyp, 0.5)
    levels.append((fx, fy, 0.5))
    if nested:                 # a patch of level 1's nodes [6, 6 + 16] x [8, 8 + 14], ratio 4
        R.nest(6, 8, 16, 14)
        levels.append((fx[6] + 0.25 * np.arange(33), fy[8] + 0.25 * np.arange(29), 0.25))
    R.direction(coupling, 1)
    for lev, (xs, ys, h) in enumerate(levels):
        R.set_level_state(lev, L.state(xs, ys, 0.0, h))
    R.start(couple=True)
    R.run(steps)
    errs = []
    for lev, (xs, ys, h) in enumerate(levels):
        got = R.level_state(lev)
        exact = L.state(xs, ys, float(steps), h)
        if lev == 0:                          # the zero-ghost edges disturb an outer band
            k = steps + 2
            got, exact = got[:, k:-k, k:-k], exact[:, k:-k, k:-k]
        errs.append(np.abs(got - exact).max() / np.abs(exact).max())
    return errs


@pytest.mark.parametrize("Q,mrt,tau,s,nested,coupling", RUNS)
def test_refined_run_keeps_the_exact_linear_solution(oracle_mod, Q, mrt, tau, s, nested,
                                                     coupling):
    errs = _exact_run(oracle_mod, Q, mrt, tau, s, nested, coupling)
    assert max(errs) < 1e-13, errs


def test_the_exact_solution_detects_a_missing_coupling(oracle_mod):
    # fine -> coarse only: nothing enters the fine grid across I (zero ghost), so the fine
    # grid leaves the exact solution at once -- the pin is not satisfied by any run
    errs = _exact_run(oracle_mod, 5, False, 0.5, None, False, "f2c")
    assert errs[1] > 1e-2
