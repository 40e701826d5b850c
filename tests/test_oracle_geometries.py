"""Further curved-weight pins (the paper's deformed spheres D_gamma of §5 and the ring Dupin
cyclide of its convergence appendix): the oracle's surface RBF-QF weights integrate the
constant (area) and a polynomial test function with an error that falls at least at the
order of the appended polynomials in n^{-1/2}.  References come from high-accuracy
parameter-space quadrature of the exact surfaces (nodesets), independent of the oracle."""
import math

import pytest

import nodesets
import oracle


def _weights(ns, k=32, deg=3):
    st = oracle.knn(ns.nodes, ns.tris, k)
    return oracle.quad_weights(ns.nodes, ns.tris, st, deg, normals=ns.normals)


def _order(e0, e1, n0, n1):
    return math.log(e0 / e1) / math.log(math.sqrt(n1 / n0))


@pytest.mark.parametrize("gamma", [0.4, 0.8])
def test_deformed_sphere_area_convergence(gamma):
    errs, ns_ = [], []
    for n in (2000, 8000):
        ns = nodesets.deformed_sphere(n, gamma, jitter=0.0)
        errs.append(abs(_weights(ns).sum() - ns.area) / ns.area)
        ns_.append(ns.n)
    assert _order(errs[0], errs[1], *ns_) > 2.5, errs
    assert errs[1] < 5e-6


def test_deformed_sphere_flat_limit_is_the_sphere():
    """gamma = 0 is the unit sphere: the area reference is 4 pi."""
    assert abs(nodesets.deformed_sphere_area(0.0) - 4 * math.pi) < 1e-10


def test_cyclide_area_and_polynomial_convergence():
    f = lambda x, y, z: x ** 3 * y ** 2 * z ** 4 + 5.0
    ref = nodesets.cyclide_integral(f)
    e_area, e_poly, ns_ = [], [], []
    for n in (2000, 8000):
        ns = nodesets.cyclide_lattice(n)
        q = _weights(ns)
        X = ns.nodes
        e_area.append(abs(q.sum() - ns.area) / ns.area)
        e_poly.append(abs(q @ f(X[:, 0], X[:, 1], X[:, 2]) - ref) / abs(ref))
        ns_.append(ns.n)
    assert _order(e_area[0], e_area[1], *ns_) > 2.5, e_area
    assert _order(e_poly[0], e_poly[1], *ns_) > 2.5, e_poly
    assert e_area[1] < 1e-5 and e_poly[1] < 1e-5


def test_cyclide_reference_area_converged():
    """The periodic trapezoid reference is converged (600 vs 900 points per direction)."""
    assert abs(nodesets.cyclide_area(m=600) - nodesets.cyclide_area(m=900)) < 1e-9


def _ellipsoid_grid(a, b, c, m=400):
    """Nodes and weights on x = (a sin t cos p, b sin t sin p, c cos t): Gauss-Legendre in
    t, the periodic trapezoid in p, times the surface element |x_t x x_p|."""
    import numpy as np
    xg, wg = np.polynomial.legendre.leggauss(m)
    t = 0.5 * math.pi * (xg + 1.0)
    p = np.arange(2 * m) * math.pi / m
    T, P = np.meshgrid(t, p, indexing="ij")
    X = np.stack([a * np.sin(T) * np.cos(P), b * np.sin(T) * np.sin(P), c * np.cos(T)], -1)
    Xt = np.stack([a * np.cos(T) * np.cos(P), b * np.cos(T) * np.sin(P), -c * np.sin(T)], -1)
    Xp = np.stack([-a * np.sin(T) * np.sin(P), b * np.sin(T) * np.cos(P), 0.0 * T], -1)
    W = (0.5 * math.pi * wg)[:, None] * (math.pi / m) * np.linalg.norm(np.cross(Xt, Xp), axis=-1)
    return X, W


def test_ellipsoid_area_closed_form_and_convergence():
    """The tri-axial ellipsoid (1, 0.8, 0.6) of the many-trajectory workload: its area is
    4 pi a b c R_G(a^-2, b^-2, c^-2) with Carlson's symmetric integral R_G (scipy); the
    parameter-space rule above agrees with it, then integrates e^x cos 2y + z^2.  The
    oracle's weights approach both at least at the appended degree's order."""
    import numpy as np
    sp = pytest.importorskip("scipy.special")
    a, b, c = 1.0, 0.8, 0.6
    area = 4.0 * math.pi * a * b * c * float(sp.elliprg(a ** -2, b ** -2, c ** -2))
    X, W = _ellipsoid_grid(a, b, c)
    assert abs(W.sum() - area) < 1e-12 * area
    f = lambda P: np.exp(P[..., 0]) * np.cos(2.0 * P[..., 1]) + P[..., 2] ** 2
    ref = float((W * f(X)).sum())
    ea, ef, ns_ = [], [], []
    for n in (1000, 16000):
        ns = nodesets.ellipsoid_fibonacci(n, axes=(a, b, c))
        q = _weights(ns)
        ea.append(abs(q.sum() - area) / area)
        ef.append(abs((q * f(ns.nodes)).sum() - ref) / abs(ref))
        ns_.append(ns.n)
    assert _order(ea[0], ea[1], *ns_) > 3.0, ea
    assert _order(ef[0], ef[1], *ns_) > 3.0, ef
    assert ea[1] < 1e-6 and ef[1] < 1e-6
