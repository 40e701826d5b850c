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
