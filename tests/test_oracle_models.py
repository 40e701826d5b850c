"""Pins for the oracle's §5 models: the C^4 smooth-step firing rate, the Adams-Bashforth 5
integrator and the synaptic-depression two-field model (Eq. (nfsyndep)).  Each checks the
oracle against mathematics it does not compute itself: contact orders and symmetry of the
smooth step, the textbook AB5 weights and its convergence order, closed-form solutions of
the uncoupled models, the RK4 branch against the RK4 oracle, and the coupled system
against SciPy's DOP853."""
import numpy as np
import pytest

import nodesets
import oracle

A, B_ = 0.06, 0.54


def test_smooth_step_values_and_symmetry():
    u = np.linspace(-0.2, 0.8, 1001)
    f = oracle.rate(u, kind=1, a=A, b=B_)
    assert np.all(f[u < A] == 0.0) and np.all(f[u >= B_] == 1.0)
    assert abs(oracle.rate(np.array([0.5 * (A + B_)]), kind=1, a=A, b=B_)[0] - 0.5) < 1e-15
    # f(a + b - u) = 1 - f(u), and monotone non-decreasing
    np.testing.assert_allclose(oracle.rate(A + B_ - u, kind=1, a=A, b=B_), 1.0 - f, rtol=0, atol=1e-12)
    assert np.all(np.diff(f) >= -1e-15)


@pytest.mark.parametrize("end", ["a", "b"])
def test_smooth_step_fifth_order_contact(end):
    """C^4 at both ends: f - f(end) vanishes to fifth order, so halving the distance to the
    end divides it by 2^5 (to leading order)."""
    for h in (1e-2, 3e-3):
        if end == "a":
            r = oracle.rate(np.array([A + h]), kind=1, a=A, b=B_)[0] / oracle.rate(np.array([A + h / 2]), kind=1, a=A, b=B_)[0]
        else:
            r = (1 - oracle.rate(np.array([B_ - h]), kind=1, a=A, b=B_)[0]) / (
                1 - oracle.rate(np.array([B_ - h / 2]), kind=1, a=A, b=B_)[0])
        assert abs(r - 32.0) < 32.0 * 0.05 * (h / 1e-2)


def test_smooth_step_integral():
    """By the symmetry, the transition's mean over [a, b] is 1/2 (Simpson is exact enough)."""
    u = np.linspace(A, B_, 20001)
    f = oracle.rate(u, kind=1, a=A, b=B_)
    h = u[1] - u[0]
    integral = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
    assert abs(integral / (B_ - A) - 0.5) < 1e-12


def test_ab5_weights_textbook():
    c = oracle.ab5_weights()
    np.testing.assert_allclose(c * 720.0, [1901, -2774, 2616, -1274, 251], rtol=0, atol=1e-10)
    assert abs(c.sum() - 1.0) < 1e-14


def _decay_case():
    ns = nodesets.torus_lattice(200, seed=1)
    mu = np.full(ns.n, ns.area / ns.n)
    u0 = nodesets.spiral_bumps_u0(ns)[None, :]
    return ns, mu, u0


@pytest.mark.parametrize("integrator,order", [("rk4", 4), ("ab5", 5)])
def test_linear_decay_convergence_order(integrator, order):
    """A1 = A2 = 0: du/dt = -u, u(T) = u0 e^{-T}; the error falls at the method's order."""
    ns, mu, u0 = _decay_case()
    T = 2.0
    errs = []
    for nst in (20, 40):
        u = oracle.field_advance(ns.nodes, mu, u0, (0.0, 0.1, 0.0, 0.2), 20.0, 0.2, T / nst, nst,
                                 integrator=integrator)
        errs.append(np.abs(u - u0 * np.exp(-T)).max())
    p = np.log2(errs[0] / errs[1])
    assert abs(p - order) < 0.35, (errs, p)


def test_rk4_branch_is_the_rk4_oracle():
    ns = nodesets.torus_lattice(300, seed=2)
    mu = np.full(ns.n, ns.area / ns.n)
    u0 = np.stack([nodesets.spiral_bumps_u0(ns), 0.5 * nodesets.spiral_bumps_u0(ns)])
    kern = (1.0, 0.1, 0.5, 0.2)
    beta, theta = np.array([20.0, 12.0]), np.array([0.2, 0.25])
    a = oracle.field_advance(ns.nodes, mu, u0, kern, beta, theta, 0.02, 7, integrator="rk4")
    b = oracle.rk4(ns.nodes, mu, u0, kern, beta, theta, 0.0, 0.02, 7)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14 * np.abs(b).max())


@pytest.mark.parametrize("integrator", ["rk4", "ab5"])
def test_depression_uncoupled_closed_forms(integrator):
    """A1 = A2 = 0.  (i) beta_d = 0: s(t) = 1 + (s0 - 1) e^{-t/tau}.  (ii) u0 large enough that
    u stays above b (smooth step saturated, f = 1): s(t) = s_inf + (s0 - s_inf) e^{-(1+beta_d) t/tau},
    s_inf = 1/(1 + beta_d); u(t) = u0 e^{-t} throughout."""
    ns, mu, _ = _decay_case()
    n = ns.n
    rng = np.random.default_rng(3)
    T, nst, tau = 1.5, 150, 4.0
    s0 = rng.uniform(0.2, 0.9, (1, n))
    u0 = np.full((1, n), 3.0)
    u, s = oracle.field_advance(ns.nodes, mu, u0, (0.0, 0.1, 0.0, 0.2), 20.0, 0.2, T / nst, nst, s0=s0, kind=1,
                                rate_kind=1, tau=tau, beta_d=0.0, integrator=integrator)
    np.testing.assert_allclose(s, 1 + (s0 - 1) * np.exp(-T / tau), rtol=0, atol=1e-9)
    bd = 0.7
    u, s = oracle.field_advance(ns.nodes, mu, u0, (0.0, 0.1, 0.0, 0.2), 20.0, 0.2, T / nst, nst, s0=s0, kind=1,
                                rate_kind=1, tau=tau, beta_d=bd, integrator=integrator)
    sinf = 1.0 / (1.0 + bd)
    np.testing.assert_allclose(s, sinf + (s0 - sinf) * np.exp(-(1 + bd) * T / tau), rtol=0, atol=1e-9)
    np.testing.assert_allclose(u, u0 * np.exp(-T), rtol=1e-9)


@pytest.mark.parametrize("rate_kind", [0, 1])
def test_depression_coupled_against_dop853(rate_kind):
    """The coupled model on a small torus node set against SciPy's DOP853 (rtol 1e-12) of
    the same ODE system; RK4 and AB5 with dt = 2.5e-3 agree to better than 1e-8."""
    from scipy.integrate import solve_ivp

    ns = nodesets.torus_lattice(120, seed=4)
    n = ns.n
    X = ns.nodes
    mu = np.full(n, ns.area / n)
    kern = (5.0, 0.3, 7.0, 0.6)
    beta, theta, tau, bd = 20.0, 0.2, 3.0, 0.6
    u0 = 0.6 * nodesets.spiral_bumps_u0(ns)[None, :]
    s0 = np.full((1, n), 0.9)
    r2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    Wm = kern[0] * np.exp(-r2 / kern[1] ** 2) - kern[2] * np.exp(-r2 / kern[3] ** 2)

    def f(u):
        if rate_kind == 0:
            return 1.0 / (1.0 + np.exp(-beta * (u - theta)))
        t = np.clip((u - A) / (B_ - A), 0.0, 1.0)
        return t ** 5 * (126 - 420 * t + 540 * t ** 2 - 315 * t ** 3 + 70 * t ** 4)

    def rhs(_, y):
        u, s = y[:n], y[n:]
        fu = f(u)
        return np.concatenate([-u + Wm @ (mu * s * fu), (1 - s - bd * s * fu) / tau])

    T = 1.0
    ref = solve_ivp(rhs, (0, T), np.concatenate([u0[0], s0[0]]), method="DOP853", rtol=1e-12, atol=1e-13).y[:, -1]
    for integ in ("rk4", "ab5"):
        u, s = oracle.field_advance(X, mu, u0, kern, beta, theta, T / 400, 400, s0=s0, kind=1, rate_kind=rate_kind,
                                    tau=tau, beta_d=bd, integrator=integ)
        err = np.abs(np.concatenate([u[0], s[0]]) - ref).max() / np.abs(ref).max()
        assert err < 1e-8, (integ, err)
