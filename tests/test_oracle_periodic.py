"""Pins for the oracle's doubly periodic distance (§4, Eq. (dist)) and the manufactured
solution of the convergence study on the square (§4.3; with scale r, §4.4's torus study).

The periodic nonlocal sum is checked against the Euclidean sum over the 3 x 3 tiling of the
node set and against translation invariance; the manufactured forcing against a closed form
of its convolution term (separable Gaussians, split where the minimum image changes,
integrated with erf) plus a fourth-order finite difference of u* in t; and the whole chain
by the convergence of the semi-discrete solution to u*."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle

L = 2.0 * math.pi


def _grid(m, L=L, shift=0.0):
    t = (np.arange(m) + shift) * (L / m)
    X, Y = np.meshgrid(t, t, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.zeros(m * m)], 1)


def test_periodic_sum_is_the_tiled_euclidean_sum():
    """A kernel far narrower than the cell: only the nearest image contributes (the others
    are below 1e-25), so the periodic sum equals the Euclidean sum over the 3 x 3 tiling."""
    rng = np.random.default_rng(0)
    n = 300
    x = np.concatenate([rng.uniform(0, L, (n, 2)), np.zeros((n, 1))], 1)
    q = rng.uniform(0.5, 1.5, n)
    u = rng.normal(size=(2, n))
    kern = (2.0, 0.25, 1.2, 0.4)
    tiles = np.concatenate([x + np.array([i * L, j * L, 0.0]) for i in (-1, 0, 1) for j in (-1, 0, 1)])
    got = oracle.nonlocal_sum(x, q, u, kern, [8.0, 3.0], [0.1, -0.2], period=L)
    big = oracle.nonlocal_sum(tiles, np.tile(q, 9), np.tile(u, (1, 9)), kern, [8.0, 3.0], [0.1, -0.2],
                              rows=np.arange(4 * n, 5 * n))
    np.testing.assert_allclose(got, big, rtol=1e-13, atol=1e-13 * np.abs(big).max())
    # and it differs from the Euclidean sum on the cell (nodes near the edges see wrapped neighbours)
    flat = oracle.nonlocal_sum(x, q, u, kern, [8.0, 3.0], [0.1, -0.2])
    assert np.abs(flat - got).max() > 1e-3


def test_periodic_translation_invariance():
    """A kernel as wide as a third of the cell: translating every node by a vector and
    reducing mod L leaves the sum unchanged (the periodic distance is translation invariant);
    a wrong set of shifts breaks this for nodes moved across the edges."""
    rng = np.random.default_rng(1)
    n = 250
    x = np.concatenate([rng.uniform(0, L, (n, 2)), np.zeros((n, 1))], 1)
    q = rng.uniform(0.5, 1.5, n)
    u = rng.normal(size=n)
    kern = (1.0, 1.2, 0.7, 2.0)
    base = oracle.nonlocal_sum(x, q, u, kern, 5.0, 0.0, period=L)
    for v in ((2.1, 0.0), (0.7, 4.4), (5.9, 3.3)):
        y = x.copy()
        y[:, :2] = np.mod(y[:, :2] + np.array(v), L)
        np.testing.assert_allclose(oracle.nonlocal_sum(y, q, u, kern, 5.0, 0.0, period=L), base,
                                   rtol=1e-12, atol=1e-12 * np.abs(base).max())


def test_zero_period_is_euclidean():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (100, 3))
    q, u = rng.uniform(size=100), rng.normal(size=100)
    kern = (1.0, 0.3, 0.5, 0.6)
    np.testing.assert_array_equal(oracle.nonlocal_sum(x, q, u, kern, 3.0, 0.1, period=0.0),
                                  oracle.nonlocal_sum(x, q, u, kern, 3.0, 0.1))


# ------------------------------------------------------------------ manufactured solution

SIG, C0, RAD = 1.1, 0.1, 0.2
BETA, THETA = 20.0, 0.3


def _minimg(d, L=L):
    return d - L * np.round(d / L)


def _piece(p, r, a, d0, d1):
    """int_{d0}^{d1} exp(-p d^2 - r (d - a)^2) dd, completing the square."""
    s = p + r
    m = r * a / s
    return math.exp(-p * r * a * a / s) * 0.5 * math.sqrt(math.pi / s) * (
        erf(math.sqrt(s) * (d1 - m)) - erf(math.sqrt(s) * (d0 - m)))


def _J(xk, x0k, p, L=L):
    """int_{-L/2}^{L/2} exp(-p d^2) exp(-minimg(xk - d - x0k)^2 / (2 SIG^2)) dd: the minimum
    image a - d (a = minimg(xk - x0k)) jumps by L at one point of the interval."""
    r = 1.0 / (2 * SIG * SIG)
    a = float(_minimg(xk - x0k, L))
    h = 0.5 * L
    if a >= 0:
        ds = a - h
        return _piece(p, r, a - L, -h, ds) + _piece(p, r, a, ds, h)
    ds = a + h
    return _piece(p, r, a, -h, ds) + _piece(p, r, a + L, ds, h)


def _conv_closed(x, t, kern, L=L):
    """C(t, x) = int_cell w(dist(x, y)) (G(y, x0(t); SIG) + C0) dy for the Mexican hat."""
    A1, s1, A2, s2 = kern
    x0 = (RAD * math.cos(t), RAD * math.sin(t))
    out = np.empty(len(x))
    for i, (px, py, _) in enumerate(x):
        tot = 0.0
        for A, s in ((A1, s1), (-A2, s2)):
            if A == 0.0:
                continue
            p = 1.0 / (s * s)
            tot += C0 * A * (math.sqrt(math.pi) * s * erf(0.5 * L / s)) ** 2
            tot += A / (2 * math.pi * SIG * SIG) * _J(px, x0[0], p, L) * _J(py, x0[1], p, L)
        out[i] = tot
    return out


def _points(t):
    """Nodes in general position and on both sides of the lines where G's nearest image of
    x0(t) changes (x - x0 = +-L/2), where the convolution's integrand has its kink (not on
    them: there u* has a kink in t as x0(t) moves across)."""
    x0 = np.array([RAD * math.cos(t), RAD * math.sin(t)])
    pts = [(0.3, 0.4), (2.0, 5.5), (6.0, 0.1), (x0[0] + L / 2 + 0.002, 1.0), (x0[0] + L / 2 + 0.01, x0[1] + L / 2 - 0.02),
           (4.0, x0[1] + L / 2 - 0.005), (x0[0] + L / 2 - 0.03, 3.0)]
    p = np.array(pts)
    return np.concatenate([np.mod(p, L), np.zeros((len(p), 1))], 1)


def _dudt(x, t, kern):
    h = 1e-3
    us = [oracle.mms_flat_solution(x, t + k * h, kern, L, BETA, THETA, C0, RAD, SIG) for k in (-2, -1, 1, 2)]
    return (us[0] - 8 * us[1] + 8 * us[2] - us[3]) / (12 * h)


def test_flat_solution_inverts_the_rate():
    t = 0.37
    x = _points(t)
    u = oracle.mms_flat_solution(x, t, (1, 1, 0, 1), L, BETA, THETA, C0, RAD, SIG)
    x0 = np.array([RAD * math.cos(t), RAD * math.sin(t)])
    d = _minimg(x[:, :2] - x0)
    z = np.exp(-(d ** 2).sum(1) / (2 * SIG ** 2)) / (2 * math.pi * SIG ** 2) + C0
    np.testing.assert_allclose(oracle.rate(u, BETA, THETA), z, rtol=1e-13)


@pytest.mark.parametrize("kern", [
    (1.0 / (2 * math.pi / 40 ** 2), math.sqrt(2) / 40, 0.0, math.sqrt(2) / 40),   # the paper's Gauss(1/40)
    (3.0, 0.5, 1.5, 1.0),                                                         # a wide Mexican hat
])
@pytest.mark.parametrize("scale", [1.0, 0.4])
def test_flat_forcing_against_closed_form(kern, scale):
    t = 0.06
    x = _points(t)
    gam = oracle.mms_flat_forcing_values(x, t, kern, L, BETA, THETA, C0, RAD, SIG, scale)
    u = oracle.mms_flat_solution(x, t, kern, L, BETA, THETA, C0, RAD, SIG)
    want = _dudt(x, t, kern) + u - scale * _conv_closed(x, t, kern)
    np.testing.assert_allclose(gam, want, rtol=0, atol=1e-10 * max(1.0, np.abs(want).max()))


def test_flat_mms_convergence():
    """The semi-discrete solution on an m x m periodic grid (equal weights (L/m)^2, the
    periodic trapezoid rule) from u*(0) converges to u*(T) as m grows; the integrand's kink
    lines limit the rate to second order."""
    kern = (3.0, 0.5, 1.5, 1.0)
    forcing = oracle.mms_flat_forcing(C0, RAD, SIG, 1.0)
    T, nst = 0.1, 5
    errs = []
    for m in (12, 24):
        x = _grid(m)
        q = np.full(m * m, (L / m) ** 2)
        u0 = oracle.mms_flat_solution(x, 0.0, kern, L, BETA, THETA, C0, RAD, SIG)[None, :]
        u = oracle.rk4(x, q, u0, kern, BETA, THETA, 0.0, T / nst, nst, forcing=forcing, period=L)
        ex = oracle.mms_flat_solution(x, T, kern, L, BETA, THETA, C0, RAD, SIG)
        errs.append(np.abs(u[0] - ex).max())
    assert errs[1] < errs[0] / 3.5, errs


def test_spatial_error_of_periodic_gaussians_averages_to_zero():
    """§4.2, Eq. (flat_spatial_error): E(x0) = (Q f_x0 - Q_n f_x0) / Q f_x0 for the
    doubly periodic Gaussians f_x0 = exp(-|x - x0|^2 / (2 sigma^2)), sigma = 1/10, on the
    unit square (point-repulsion nodes, n = 2000, r^3, k = 21, deg 3).  Q f_x0 does not
    depend on x0, so the mean of E over x0 is 1 - sum q = 0: here the mean over a 64 x 64
    grid of centres (appended to the node set with weight 0, f = 1) against the closed form
    Q f = (s sqrt(pi) erf(1 / (2 s)))^2 with s = sqrt(2) sigma (nearest image)."""
    import nodesets
    ns = nodesets.square_repulsion(2000)
    x2 = ns.coords()
    q = oracle.quad_weights(x2, ns.tris, oracle.knn(x2, ns.tris, 21), 3)
    m = 64
    t = (np.arange(m) + 0.5) / m
    c = np.stack(np.meshgrid(t, t, indexing="ij"), -1).reshape(-1, 2)
    x = np.concatenate([ns.nodes, np.concatenate([c, np.zeros((m * m, 1))], 1)])
    s = math.sqrt(2.0) * 0.1
    Qn = oracle.nonlocal_sum(x, np.concatenate([q, np.zeros(m * m)]), np.full((1, x.shape[0]), 50.0),
                             (1.0, s, 0.0, s), 1.0, 0.0, rows=np.arange(ns.n, ns.n + m * m), period=1.0)[0]
    Qf = (s * math.sqrt(math.pi) * erf(0.5 / s)) ** 2
    E = (Qf - Qn) / Qf
    rms = math.sqrt((E ** 2).mean())
    assert 1e-8 < rms < 1e-3          # small, and not identically zero
    assert abs(E.mean()) < 1e-4 * rms  # averages to zero (midpoint rule on the kink of the nearest image: < 1e-8)
