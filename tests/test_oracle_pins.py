"""Pins for the FP64 oracle: each test checks it against something other than its
own code -- brute force, an independent numerical integration, a closed form, a
library routine, or a property the paper states.  CPU only."""
import math

import numpy as np
import pytest

import nodesets
import oracle


# ----------------------------------------------------------------------------------
# independent triangle quadrature: Duffy collapse + numpy Gauss-Legendre
# ----------------------------------------------------------------------------------

def _cross2(a, b):
    return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]


def duffy(f, apex, A, B, n=24):
    """Signed integral of f over triangle (apex, A, B): x = apex + u[(A-apex) + v(B-A)]."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    u = 0.5 * (xg + 1.0)
    wu = 0.5 * wg
    U, V = np.meshgrid(u, u, indexing="ij")
    W = np.outer(wu, wu)
    P = apex + U[..., None] * ((A - apex) + V[..., None] * (B - A))
    jac = U * _cross2(A - apex, B - A)
    return float((W * jac * f(P)).sum())


def tri_area(T):
    return 0.5 * abs(_cross2(T[1] - T[0], T[2] - T[0]))


def inside(p, T):
    s = [_cross2(T[(i + 1) % 3] - T[i], p - T[i]) for i in range(3)]
    return all(v > 0 for v in s) or all(v < 0 for v in s)


def r3_numeric(p, T):
    f = lambda P: np.linalg.norm(P - p, axis=-1) ** 3
    if inside(p, T):      # split at p: smooth in each Duffy chart
        tot = sum(abs(duffy(f, p, T[i], T[(i + 1) % 3], 400)) for i in range(3))
        return tot
    # p outside (or on a vertex): f is smooth on T away from a vertex singularity
    j = int(np.argmin(np.linalg.norm(T - p, axis=1)))
    return abs(duffy(f, T[j], T[(j + 1) % 3], T[(j + 2) % 3], 400))


@pytest.fixture(scope="module")
def rng():
    return np.random.default_rng(1234)


# ----------------------------------------------------------------------------------
# §3.1 stencils
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_knn_matches_full_sort(dim, rng):
    # quantised coordinates force many exact distance ties: the (d^2, index) order decides
    n = 300
    X = np.round(rng.uniform(0, 1, size=(n, dim)) * 8) / 8
    tris = rng.integers(0, n, size=(60, 3)).astype(np.int32)
    k = 17
    got = oracle.knn(X, tris, k)
    for e in range(tris.shape[0]):
        c = X[tris[e]].sum(0) / 3.0
        c = ((X[tris[e, 0]] + X[tris[e, 1]]) + X[tris[e, 2]]) / 3.0
        d2 = ((X - c) ** 2).sum(1)
        want = np.lexsort((np.arange(n), d2))[:k]
        np.testing.assert_array_equal(got[e], want)


@pytest.mark.parametrize("dim", [2, 3])
def test_knn_at_matches_full_sort_and_centroid_form(dim, rng):
    # the §3.1 selection around given centres: quantised nodes and centres (exact ties), some
    # centres outside the nodes' bounding box; at the centroids it equals knn
    n = 300
    X = np.round(rng.uniform(0, 1, size=(n, dim)) * 8) / 8
    Cq = np.round(rng.uniform(-0.5, 1.5, size=(40, dim)) * 16) / 16
    k = 13
    got = oracle.knn_at(X, Cq, k)
    for e in range(Cq.shape[0]):
        d2 = ((X - Cq[e]) ** 2).sum(1)
        np.testing.assert_array_equal(got[e], np.lexsort((np.arange(n), d2))[:k])
    tris = rng.integers(0, n, size=(30, 3)).astype(np.int32)
    cent = ((X[tris[:, 0]] + X[tris[:, 1]]) + X[tris[:, 2]]) / 3.0
    np.testing.assert_array_equal(oracle.knn_at(X, cent, k), oracle.knn(X, tris, k))


def test_knn_subset_and_permutation_invariance(rng):
    n = 400
    X = rng.uniform(size=(n, 3))
    tris = rng.integers(0, n, size=(50, 3)).astype(np.int32)
    full = oracle.knn(X, tris, 12)
    sub = oracle.knn(X, tris, 12, elems=np.array([7, 3, 49]))
    np.testing.assert_array_equal(sub, full[[7, 3, 49]])
    perm = rng.permutation(n)
    inv = np.argsort(perm)
    got = oracle.knn(X[perm], inv[tris].astype(np.int32), 12)
    # same sets (ties are absent for continuous coordinates)
    for e in range(50):
        assert set(perm[got[e]].tolist()) == set(full[e].tolist())


# ----------------------------------------------------------------------------------
# §3.2 analytic integrals over a triangle
# ----------------------------------------------------------------------------------

def test_tri_r3_against_numeric(rng):
    for trial in range(40):
        T = rng.uniform(-1, 1, size=(3, 2))
        if tri_area(T) < 0.05:
            continue
        c = T.mean(0)
        for p in [c, c + rng.uniform(-0.2, 0.2, 2), rng.uniform(-3, 3, 2), T[trial % 3].copy()]:
            got = oracle.tri_r3(p, T)
            want = r3_numeric(p, T)
            assert got == pytest.approx(want, rel=1e-10, abs=1e-13), (trial, p)
    # orientation must not matter
    T = np.array([[0.0, 0.0], [1.0, 0.2], [0.3, 0.9]])
    p = np.array([0.1, 0.7])
    assert oracle.tri_r3(p, T) == pytest.approx(oracle.tri_r3(p, T[::-1].copy()), rel=1e-14)


def test_tri_r3_translation_scaling():
    T = np.array([[0.1, 0.0], [1.3, 0.4], [0.2, 1.1]])
    p = np.array([0.9, 0.9])
    base = oracle.tri_r3(p, T)
    s = 2.5
    assert oracle.tri_r3(s * p + 7.0, s * T + 7.0) == pytest.approx(s ** 5 * base, rel=1e-12)


def test_tri_mono_against_gauss(rng):
    for trial in range(10):
        T = rng.uniform(-2, 2, size=(3, 2))
        for a in range(0, 6):
            for b in range(0, 6 - a):
                f = lambda P: P[..., 0] ** a * P[..., 1] ** b
                want = abs(duffy(f, T[0], T[1], T[2], 12))
                # the monomial need not be positive: compare with the signed, CCW-oriented value
                sgn = np.sign(_cross2(T[1] - T[0], T[2] - T[0]))
                want = sgn * duffy(f, T[0], T[1], T[2], 12)
                assert oracle.tri_mono(a, b, T) == pytest.approx(want, rel=1e-11, abs=1e-12)
    assert oracle.tri_mono(0, 0, T) == pytest.approx(tri_area(T), rel=1e-14)


# ----------------------------------------------------------------------------------
# §3.2 one element: the weights integrate the local PHS+polynomial interpolant
# ----------------------------------------------------------------------------------

def _refined_integral(fun, T, levels=4, n=10):
    """Integral of fun over T by uniform 4^levels subdivision and a Gauss product rule."""
    tris = [T]
    for _ in range(levels):
        nxt = []
        for t in tris:
            m01, m12, m20 = (t[0] + t[1]) / 2, (t[1] + t[2]) / 2, (t[2] + t[0]) / 2
            nxt += [np.array([t[0], m01, m20]), np.array([m01, t[1], m12]),
                    np.array([m20, m12, t[2]]), np.array([m01, m12, m20])]
        tris = nxt
    return sum(abs(duffy(fun, t[0], t[1], t[2], n)) if False else
               np.sign(_cross2(t[1] - t[0], t[2] - t[0])) * duffy(fun, t[0], t[1], t[2], n) for t in tris)


@pytest.mark.parametrize("deg,k", [(1, 8), (2, 12), (3, 16), (4, 24)])
def test_element_weights_integrate_interpolant(deg, k, rng):
    from scipy.interpolate import RBFInterpolator
    T = np.array([[-0.3, -0.25], [0.35, -0.2], [0.0, 0.4]])
    xi = np.concatenate([T, rng.uniform(-1, 1, size=(k - 3, 2))])
    w = oracle.element_weights_local(xi, T, deg)
    data = np.sin(3 * xi[:, 0]) * np.cos(2 * xi[:, 1]) + xi[:, 0] ** 2
    s = RBFInterpolator(xi, data, kernel="cubic", degree=deg)
    want = _refined_integral(lambda P: s(P.reshape(-1, 2)).reshape(P.shape[:-1]), T)
    got = float(w @ data)
    assert got == pytest.approx(want, rel=1e-9, abs=1e-11)
    # polynomial reproduction (the moment conditions): exact for every monomial <= deg
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            assert w @ (xi[:, 0] ** a * xi[:, 1] ** b) == pytest.approx(oracle.tri_mono(a, b, T), abs=1e-13)


def test_element_weights_rigid_and_scale_invariance(rng):
    """Weights of a stencil transform as area: invariant under rotation/translation,
    scale by s^2 under uniform scaling (r^3 is homogeneous, P_deg is affine invariant)."""
    T = np.array([[-0.3, -0.25], [0.35, -0.2], [0.0, 0.4]])
    xi = np.concatenate([T, rng.uniform(-1, 1, size=(13, 2))])
    w = oracle.element_weights_local(xi, T, 3)
    a = 0.7
    Rm = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    s, sh = 0.37, np.array([0.1, -0.2])
    w2 = oracle.element_weights_local(s * xi @ Rm.T + sh, s * T @ Rm.T + sh, 3)
    np.testing.assert_allclose(w2, s * s * w, rtol=1e-9, atol=1e-13)


# ----------------------------------------------------------------------------------
# §3.2 flat quadrature weights
# ----------------------------------------------------------------------------------

def _flat(ns, k, deg):
    st = oracle.knn(ns.coords(), ns.tris, k)
    return oracle.quad_weights(ns.coords(), ns.tris, st, deg)


def test_flat_constants_and_polynomials_exact():
    ns = nodesets.square_halton(1500)
    x, y = ns.nodes[:, 0], ns.nodes[:, 1]
    for k, deg in [(24, 2), (21, 3)]:
        q = _flat(ns, k, deg)
        assert q.sum() == pytest.approx(1.0, abs=1e-13)
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                assert (q * x ** a * y ** b).sum() == pytest.approx(1.0 / ((a + 1) * (b + 1)), abs=1e-13)


def test_flat_regular_grid_interior_weights_equal_cell_area():
    """§4.2: on a regular triangular lattice interior stencils are rotated translates,
    so every interior weight equals the area per node (sqrt(3)/2 s^2)."""
    ns = nodesets.square_regular(30)
    s = ns.meta["s"]
    x, y = ns.nodes[:, 0], ns.nodes[:, 1]
    inner = np.minimum.reduce([x, y, 1 - x, 1 - y]) > 5 * s
    for k, deg in [(21, 3), (21, 2), (12, 2)]:
        q = _flat(ns, k, deg)
        np.testing.assert_allclose(q[inner], math.sqrt(3) / 2 * s * s, rtol=1e-12)


def test_regular_grid_supplement_polynomial_and_gaussian():
    """Supplement (regular triangular grid, r^3, k = 30): x^3 - y^4 is integrated exactly
    once degree-4 polynomials are appended (and not with degree 3), and the Gaussian
    exp(-10 |x - (1/2, 1/2)|^2), whose integral is (sqrt(pi/10) erf(sqrt(10)/2))^2, converges
    faster than the appended degree in n^-1/2."""
    from scipy.special import erf
    exact_g = (math.sqrt(math.pi / 10) * erf(math.sqrt(10) / 2)) ** 2
    exact_p = 0.25 - 0.2
    errs, ns_ = [], []
    for rows in (12, 40):
        ns = nodesets.square_regular(rows)
        x, y = ns.nodes[:, 0], ns.nodes[:, 1]
        q4 = _flat(ns, 30, 4)
        assert abs((q4 * (x ** 3 - y ** 4)).sum() - exact_p) < 1e-13
        q3 = _flat(ns, 30, 3)
        assert abs((q3 * (x ** 3 - y ** 4)).sum() - exact_p) > 1e-9
        errs.append(abs((q4 * np.exp(-10 * ((x - 0.5) ** 2 + (y - 0.5) ** 2))).sum() - exact_g) / exact_g)
        ns_.append(ns.n)
    assert math.log(errs[0] / errs[1]) / math.log(math.sqrt(ns_[1] / ns_[0])) > 4.0, errs


def test_flat_histogram_mode_near_one_over_n():
    """Fig. 3B: n = 2000 nodes on the unit square, r^3, k = 21, deg 3: the main mode of
    the weight histogram sits near 1/n = 0.0005 (the value printed in the caption)."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    fact = gold["flat_square_weight_mode"]
    ns = nodesets.square_halton(fact["n"])
    q = _flat(ns, fact["k"], fact["deg"])
    hist, edges = np.histogram(q, bins=60)
    mode = 0.5 * (edges[hist.argmax()] + edges[hist.argmax() + 1])
    assert mode == pytest.approx(fact["mode"], rel=0.25)


def test_flat_repulsion_nodes_weight_structure():
    """§4.2 on the paper's random node family (point repulsion, equispaced boundary;
    n = 2000, r^3, k = 21, deg 3): constants integrate exactly, the main histogram mode
    lies near 1/n, boundary weights are smaller than interior ones, and negative weights
    are few and small (the paper counts five)."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    fact = gold["flat_square_weight_mode"]
    ns = nodesets.square_repulsion(fact["n"])
    q = _flat(ns, fact["k"], fact["deg"])
    assert abs(q.sum() - 1.0) < 1e-12
    hist, edges = np.histogram(q, bins=60)
    mode = 0.5 * (edges[hist.argmax()] + edges[hist.argmax() + 1])
    assert mode == pytest.approx(fact["mode"], rel=0.25)
    nb = ns.meta["n_boundary"]
    assert np.median(q[:nb]) < 0.75 * np.median(q[nb:])
    assert (q < 0).sum() <= 5
    assert q.min() > -0.1 * np.median(q)


def test_flat_convergence_chebyshev():
    """§4.3: T5(2x-1) T4(2y-1) + 1 on the unit square (integral 1).  Random node sets
    make single errors noisy (§4.3 says so), so the RMS over three seeded node sets is
    used; it falls faster than O(h^deg) as n grows."""
    errs = []
    ns_list = [1000, 4000, 16000]
    for n in ns_list:
        e = []
        for seed in (0, 1000, 2000):
            ns = nodesets.square_halton(n, seed=seed)
            q = _flat(ns, 21, 3)
            x, y = ns.nodes[:, 0], ns.nodes[:, 1]
            f = (np.cos(5 * np.arccos(np.clip(2 * x - 1, -1, 1)))
                 * np.cos(4 * np.arccos(np.clip(2 * y - 1, -1, 1))) + 1)
            e.append((q * f).sum() - 1.0)
        errs.append(math.sqrt(np.mean(np.square(e))))
    order = math.log(errs[0] / errs[-1]) / math.log(math.sqrt(ns_list[-1] / ns_list[0]))
    assert order > 3.0, errs


# ----------------------------------------------------------------------------------
# §3.3 surfaces
# ----------------------------------------------------------------------------------

def _surf(ns, k, deg):
    st = oracle.knn(ns.nodes, ns.tris, k)
    return oracle.quad_weights(ns.nodes, ns.tris, st, deg, normals=ns.normals), st


def test_projection_point_lies_on_shared_cutting_planes():
    """§3.3: adjacent elements E, E' must send their shared edge to the same curved
    edge, so p_E and p_E' lie in the plane through that edge orthogonal to n_E - n_E'."""
    ns = nodesets.torus_lattice(4000, seed=3)
    nbr = oracle.tri_neighbors(ns.tris)
    assert (nbr >= 0).all()
    X = ns.nodes

    def normal(e):
        a, b, c = X[ns.tris[e]]
        nn = np.cross(b - a, c - a)
        nn /= np.linalg.norm(nn)
        return nn if nn @ ns.normals[ns.tris[e]].sum(0) > 0 else -nn

    checked = 0
    for e in range(0, ns.m, 97):
        pe = oracle.projection_point(X, ns.normals, ns.tris, nbr, e)
        if pe is None:
            continue
        for kk in range(3):
            f = nbr[e, kk]
            pf = oracle.projection_point(X, ns.normals, ns.tris, nbr, f)
            a = X[ns.tris[e, kk]]
            dn = normal(e) - normal(f)
            assert abs((pe - a) @ dn) < 1e-9 * max(1.0, np.linalg.norm(pe))
            if pf is not None:
                assert abs((pf - a) @ dn) < 1e-9 * max(1.0, np.linalg.norm(pf))
                checked += 1
    assert checked > 50


def test_surface_jacobian_matches_area_ratio_on_sphere():
    """J_E at each projected stencil node equals the ratio of surface area to plane area
    of the central projection mu_E (closed form on the unit sphere), measured by mapping
    a tiny triangle around the node."""
    ns = nodesets.sphere_fibonacci(800, seed=2)
    nbr = oracle.tri_neighbors(ns.tris)
    st = oracle.knn(ns.nodes, ns.tris, 12)
    X = ns.nodes
    for e in [0, 100, 333, 700]:
        p = oracle.projection_point(X, ns.normals, ns.tris, nbr, e)
        assert p is not None
        w, jac, central = oracle.surface_element_weights(X, ns.normals, ns.tris, nbr, e, st[e], 2)
        assert central
        a, b, c = X[ns.tris[e]]
        nE = np.cross(b - a, c - a)
        nE /= np.linalg.norm(nE)
        cE = (a + b + c) / 3

        def mu(xi):       # line p + s (xi - p), s > 0, hitting the unit sphere nearest to xi
            d = xi - p
            A, Bq, Cq = d @ d, 2 * p @ d, p @ p - 1
            roots = [(-Bq + sg * math.sqrt(Bq * Bq - 4 * A * Cq)) / (2 * A) for sg in (1, -1)]
            s = min(roots, key=lambda s: abs(s - 1))
            return p + s * d

        for r in range(12):
            x = X[st[e, r]]
            t = ((cE - p) @ nE) / ((x - p) @ nE)
            xi = p + t * (x - p)
            e1 = np.cross(nE, [0.3, 0.5, 0.7])
            e1 /= np.linalg.norm(e1)
            e2 = np.cross(nE, e1)
            h = 1e-4
            P = [xi, xi + h * e1, xi + h * e2]
            Q = [mu(v) for v in P]
            ratio = np.linalg.norm(np.cross(Q[1] - Q[0], Q[2] - Q[0])) / np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
            assert jac[r] == pytest.approx(ratio, rel=2e-4)


def test_sphere_area_and_monomial_convergence():
    """Supplementary (sphere): sum of weights -> 4 pi and x^2 y^2 z^4 (closed form
    2 G(3/2)^2 G(5/2) / G(11/2)) at least at the appended degree in n^{-1/2}; the
    integral of sin x cos 2y cos 3z is 0 (odd in x), and its error falls as fast."""
    exact_m = 2 * math.gamma(1.5) ** 2 * math.gamma(2.5) / math.gamma(5.5)
    ns_list = [1000, 4000, 16000]
    e_area, e_mono, e_odd = [], [], []
    for n in ns_list:
        ns = nodesets.sphere_fibonacci(n)
        q, _ = _surf(ns, 32, 3)
        x, y, z = ns.nodes.T
        e_area.append(abs(q.sum() - 4 * math.pi) / (4 * math.pi))
        e_mono.append(abs((q * (x ** 3 * y ** 2 * z ** 4 + 5)).sum() - 20 * math.pi) / (20 * math.pi))
        e_mono[-1] = max(e_mono[-1], abs((q * x ** 2 * y ** 2 * z ** 4).sum() - exact_m) / exact_m)
        e_odd.append(abs((q * np.sin(x) * np.cos(2 * y) * np.cos(3 * z)).sum()))
    span = math.log(math.sqrt(ns_list[-1] / ns_list[0]))
    assert math.log(e_odd[0] / e_odd[-1]) / span >= 3.0, e_odd
    assert math.log(e_area[0] / e_area[-1]) / span >= 3.0, e_area
    assert math.log(e_mono[0] / e_mono[-1]) / span >= 3.0, e_mono
    assert e_area[-1] < 1e-6


def test_torus_area_and_sin7x():
    """§4.4: torus R=3, r=1 quadrature of sin(7x)+1; area 4 pi^2 R r.  Reference value
    by the periodic trapezoid rule in (phi, theta), which is spectrally accurate."""
    R, r = 3.0, 1.0
    M = 600
    ph, th = np.meshgrid(np.arange(M) * 2 * np.pi / M, np.arange(M) * 2 * np.pi / M, indexing="ij")
    P = nodesets.torus_point(ph, th, R, r)
    ref = ((np.sin(7 * P[..., 0]) + 1) * r * (R + r * np.cos(th))).sum() * (2 * np.pi / M) ** 2
    errs = []
    ns_list = [4000, 16000]
    for n in ns_list:
        ns = nodesets.torus_lattice(n, R=R, r=r, jitter=0.0)  # spiral lattice, same aspect at both n
        q, _ = _surf(ns, 32, 3)
        assert q.sum() == pytest.approx(4 * math.pi ** 2 * R * r, rel=1e-4)
        errs.append(abs((q * (np.sin(7 * ns.nodes[:, 0]) + 1)).sum() - ref) / ref)
    order = math.log(errs[0] / errs[1]) / math.log(math.sqrt(ns_list[1] / ns_list[0]))
    assert order >= 3.0, errs


# ----------------------------------------------------------------------------------
# §2.2 Eq. (2.9): the nonlocal sum
# ----------------------------------------------------------------------------------

def test_nonlocal_sum_bruteforce(rng):
    n, B = 257, 3
    X = rng.uniform(-1, 1, size=(n, 3))
    q = rng.uniform(0.001, 0.01, n)
    u = rng.normal(0.2, 0.5, size=(B, n))
    kp = (1.0, 0.3, 0.5, 0.6)
    beta = np.array([20.0, 5.0, 50.0])
    theta = np.array([0.2, 0.5, 0.0])
    got = oracle.nonlocal_sum(X, q, u, kp, beta, theta)
    D2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    W = kp[0] * np.exp(-D2 / kp[1] ** 2) - kp[2] * np.exp(-D2 / kp[3] ** 2)
    F = 1 / (1 + np.exp(-beta[:, None] * (u - theta[:, None])))
    want = (W @ (q[None, :] * F).T).T
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)
    rows = np.array([5, 0, 256])
    np.testing.assert_allclose(oracle.nonlocal_sum(X, q, u, kp, beta, theta, rows=rows), want[:, rows], rtol=1e-14)


@pytest.mark.parametrize("period", [0.0, 1.0])
def test_nonlocal_operator_is_symmetric(rng, period):
    """w depends on the distance alone (§2.2), so W is symmetric: u.(Wv) = v.(Wu).  With
    f = 1 (u far above theta) the oracle's sum with weights v is Wv; this catches an index
    or a displacement taken the wrong way round, on the plain and the periodic distance."""
    n = 301
    X = rng.uniform(0, 1, size=(n, 3))
    X[:, 2] = 0.0 if period else X[:, 2]
    kp = (1.0, 0.15, 0.5, 0.3)
    one = np.full((1, n), 50.0)
    u, v = rng.normal(size=n), rng.normal(size=n)
    Wu = oracle.nonlocal_sum(X, u, one, kp, np.ones(1), np.zeros(1), period=period)[0]
    Wv = oracle.nonlocal_sum(X, v, one, kp, np.ones(1), np.zeros(1), period=period)[0]
    assert abs(u @ Wv - v @ Wu) < 1e-12 * np.abs(u) @ np.abs(Wv)


# ----------------------------------------------------------------------------------
# RK4 time stepping
# ----------------------------------------------------------------------------------

def test_rk4_linear_decay_closed_form(rng):
    """With w = 0 and no forcing du/dt = -u: RK4 multiplies by
    1 - dt + dt^2/2 - dt^3/6 + dt^4/24 per step exactly (up to rounding)."""
    n = 50
    X = rng.uniform(size=(n, 3))
    q = np.full(n, 0.02)
    u0 = rng.normal(size=(2, n))
    dt, N = 0.05, 37
    got = oracle.rk4(X, q, u0, (0.0, 0.1, 0.0, 0.2), 20.0, 0.2, 0.0, dt, N)
    g = 1 - dt + dt ** 2 / 2 - dt ** 3 / 6 + dt ** 4 / 24
    np.testing.assert_allclose(got, u0 * g ** N, rtol=1e-13)


def test_rk4_fourth_order_against_scipy(rng):
    """Halving dt shrinks the error against a tight-tolerance DOP853 solution ~16x."""
    from scipy.integrate import solve_ivp
    n = 40
    X = rng.uniform(size=(n, 3))
    q = rng.uniform(0.05, 0.1, n)
    u0 = rng.normal(0.3, 0.3, size=(1, n))
    kp = (1.0, 0.3, 0.5, 0.6)
    beta, theta = 8.0, 0.2
    D2 = ((X[:, None] - X[None]) ** 2).sum(-1)
    W = kp[0] * np.exp(-D2 / kp[1] ** 2) - kp[2] * np.exp(-D2 / kp[3] ** 2)
    rhs = lambda t, u: -u + W @ (q / (1 + np.exp(-beta * (u - theta))))
    T = 1.0
    ref = solve_ivp(rhs, (0, T), u0[0], method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    errs = []
    for N in (10, 20, 40):
        errs.append(np.abs(oracle.rk4(X, q, u0, kp, beta, theta, 0.0, T / N, N)[0] - ref).max())
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20, errs


# ----------------------------------------------------------------------------------
# Manufactured solution on the sphere (§4 Eq. (4.5) technique)
# ----------------------------------------------------------------------------------

def _fh_closed(kernel):
    """Funk-Hecke eigenvalues of exp(-r^2/s^2) on the unit sphere in closed form:
    r^2 = 2(1 - t); I_p = int_{-1}^1 exp(-a(1-t)) t^p dt by parts."""
    A1, s1, A2, s2 = kernel
    out = np.zeros(3)
    for amp, s in ((A1, s1), (-A2, s2)):
        a = 2.0 / s ** 2
        E = math.exp(-2 * a)
        I0 = (1 - E) / a
        I1 = (1 + E) / a - I0 / a
        I2 = (1 - E) / a - 2 * I1 / a
        out += amp * 2 * math.pi * np.array([I0, I1, 0.5 * (3 * I2 - I0)])
    return out


@pytest.mark.parametrize("kernel", [(1.0, 0.1, 0.5, 0.2), (1.2, 0.08, 0.6, 0.25), (1.0, 0.7, 0.3, 1.3)])
def test_funk_hecke_eigenvalues(kernel):
    np.testing.assert_allclose(oracle.mms_sphere_eigs(kernel), _fh_closed(kernel), rtol=1e-12)


def test_manufactured_sphere_solution_converges():
    """The discrete solution approaches the manufactured u* as n grows (the quadrature
    error drives the discrepancy), with an order above 2 in n^{-1/2}."""
    kernel = (1.0, 0.3, 0.5, 0.6)
    beta, theta = 20.0, 0.2
    F = oracle.mms_sphere_forcing(kernel)
    errs = []
    ns_list = [1000, 4000]
    for n in ns_list:
        ns = nodesets.sphere_fibonacci(n)
        q, _ = _surf(ns, 32, 3)
        u0 = oracle.mms_sphere_solution(ns.nodes, 0.0, beta, theta)
        uN = oracle.rk4(ns.nodes, q, u0, kernel, beta, theta, 0.0, 0.02, 10, forcing=F)
        ustar = oracle.mms_sphere_solution(ns.nodes, 0.2, beta, theta)
        errs.append(np.abs(uN[0] - ustar).max())
    assert errs[-1] < 1e-4
    order = math.log(errs[0] / errs[1]) / math.log(2.0)
    assert order > 2.0, errs


# ----------------------------------------------------------------------------------
# Discrete adjoint against FP64 central differences
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("period", [0.0, 2.0])
def test_adjoint_matches_central_differences(rng, period):
    """FP64 central differences (h = 1e-4) of L = |u(T) - target|^2 in the four kernel
    parameters and in entries of u0, on the plain and on the doubly periodic distance (nodes
    of the square of side 2, where the kernel reaches across the edges)."""
    n, B = 120, 2
    X = rng.uniform(-1, 1, size=(n, 3))
    if period:
        X[:, :2] += 1.0
        X[:, 2] = 0.0
    q = rng.uniform(0.01, 0.03, n)
    u0 = rng.normal(0.3, 0.3, size=(B, n))
    kp = np.array([1.0, 0.4, 0.5, 0.8])
    beta, theta = np.array([8.0, 12.0]), np.array([0.2, 0.3])
    dt, N = 0.05, 12
    target = rng.normal(0.1, 0.2, size=(B, n))
    uN = oracle.rk4(X, q, u0, kp, beta, theta, 0.0, dt, N, period=period)
    gu, gk = oracle.adjoint(X, q, u0, kp, beta, theta, 0.0, dt, N, 2 * (uN - target), period=period)
    loss = lambda u_, k_: oracle.loss(X, q, u_, k_, beta, theta, 0.0, dt, N, target, period=period)
    h = 1e-4
    for p in range(4):
        kp1, kp2 = kp.copy(), kp.copy()
        kp1[p] += h
        kp2[p] -= h
        fd = (loss(u0, kp1) - loss(u0, kp2)) / (2 * h)
        assert gk[:, p].sum() == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for (b, i) in [(0, 3), (1, 77), (0, 119)]:
        up, um = u0.copy(), u0.copy()
        up[b, i] += h
        um[b, i] -= h
        fd = (loss(up, kp) - loss(um, kp)) / (2 * h)
        assert gu[b, i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_oracle_thread_count_does_not_change_results():
    """The oracle's OpenMP loops reduce every output in a fixed order: one thread and all
    threads give bit-identical sums (the bench times both)."""
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, (700, 3))
    q = rng.uniform(0.5, 1.5, 700)
    u = rng.normal(size=(2, 700))
    a = oracle.nonlocal_sum(x, q, u, (1.0, 0.3, 0.5, 0.6), [10.0, 20.0], [0.1, 0.2])
    oracle.set_threads(1)
    try:
        b = oracle.nonlocal_sum(x, q, u, (1.0, 0.3, 0.5, 0.6), [10.0, 20.0], [0.1, 0.2])
    finally:
        oracle.set_threads(0)
    np.testing.assert_array_equal(a, b)
