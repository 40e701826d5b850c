"""FP64 CPU oracle for the RBF neural-field method (Shaw, Kilpatrick & Avitabile).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``nf_oracle.c`` (plain C, double precision, no contraction);
this module only marshals numpy arrays through ctypes.  Each function cites the
paper passage it follows:

* :func:`knn`              §3.1 stencil of an element: k nearest nodes to its centre
* :func:`tri_r3`, :func:`tri_mono`   §3.2 analytic integrals of the basis over a triangle
* :func:`element_weights_local`      §3.2 Eqs. (3.4)-(3.5) one element's RBF-QF weights
* :func:`quad_weights`     §3.2 Eq. (3.5) node weights (flat), §3.3 Eq. (3.6) (surfaces)
* :func:`nonlocal_sum`     §2.2 Eq. (2.9) I_i = sum_j w(x_i, x_j) mu_j f(u_j)
* :func:`rk4`              classical RK4 on Eq. (2.9)
* :func:`adjoint`          discrete adjoint of that RK4 map
* :func:`mms_sphere_eigs`  Funk-Hecke eigenvalues for the manufactured solution (§4, Eq. (4.5))
* :func:`rate`             §5 firing rates: sigmoid, C^4 smooth step (Eq. (smoothf))
* :func:`ab5_weights`      Adams-Bashforth 5 weights from their definition
* :func:`field_advance`    §5 models (neural field, synaptic depression, Eq. (nfsyndep)) by
                           RK4 or AB5
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_knn.argtypes = [_dp, C.c_int64, C.c_int, _ip, C.c_int64, _lp, C.c_int64, C.c_int, _ip]
        L.or_knn_at.argtypes = [_dp, C.c_int64, C.c_int, _dp, C.c_int64, C.c_int, _ip]
        L.or_tri_r3.argtypes = [_dp, _dp]
        L.or_tri_r3.restype = C.c_double
        L.or_tri_mono.argtypes = [C.c_int, C.c_int, _dp]
        L.or_tri_mono.restype = C.c_double
        L.or_element_weights_local.argtypes = [_dp, C.c_int, _dp, C.c_int, _dp]
        L.or_quad_weights.argtypes = [_dp, _dp, C.c_int64, C.c_int, _ip, C.c_int64, _ip, C.c_int, C.c_int,
                                      _dp, _dp, _lp]
        L.or_tri_neighbors.argtypes = [_ip, C.c_int64, _lp]
        L.or_projection_point.argtypes = [_dp, _dp, _ip, _lp, C.c_int64, _dp]
        L.or_surface_element_weights.argtypes = [_dp, _dp, _ip, _lp, C.c_int64, _ip, C.c_int, C.c_int, _dp, _dp,
                                                 C.POINTER(C.c_int)]
        L.or_nonlocal.argtypes = [_dp, _dp, C.c_int64, _dp, C.c_int, _dp, _dp, _dp, _lp, C.c_int64, _dp]
        L.or_rk4.argtypes = [_dp, _dp, C.c_int64, _dp, C.c_int, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp,
                             _dp, _dp]
        L.or_adjoint.argtypes = [_dp, _dp, C.c_int64, _dp, C.c_int, C.c_double, C.c_double, C.c_int, _dp, _dp,
                                 _dp, _dp, _dp, _dp, _dp]
        L.or_loss.argtypes = [_dp, _dp, C.c_int64, _dp, C.c_int, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp,
                              _dp, _dp]
        L.or_loss.restype = C.c_double
        L.or_mms_sphere_eigs.argtypes = [_dp, _dp]
        L.or_mms_sphere_solution.argtypes = [_dp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                             C.c_double, _dp]
        L.or_num_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or_set_threads.restype = None
        L.or_mms_flat_solution.argtypes = [_dp, C.c_int64, C.c_double, _dp, C.c_double, C.c_double, C.c_double,
                                           C.c_double, C.c_double, _dp]
        L.or_mms_flat_solution.restype = None
        L.or_mms_flat_forcing.argtypes = [_dp, C.c_int64, C.c_double, _dp, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_double, C.c_double, _dp]
        L.or_mms_flat_forcing.restype = None
        L.or_rate.argtypes = [_dp, C.c_double, C.c_double, C.c_double]
        L.or_rate.restype = C.c_double
        L.or_ab5_weights.argtypes = [_dp]
        L.or_field_advance.argtypes = [_dp, _dp, C.c_int64, _dp, _dp, C.c_int, C.c_double, C.c_double, C.c_int,
                                       _dp, _dp, _dp, _dp, C.c_int]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_lp)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int = 0) -> None:
    """Thread count of the oracle's OpenMP loops (0: the default); results do not depend on it."""
    lib().or_set_threads(int(n))


# ---------------------------------------------------------------------------- §3.1

def knn(nodes, tris, k, elems=None):
    """Stencils S(E): for each element (or each of ``elems``) the k nodes nearest to its
    centroid, ordered by (squared distance, index) ascending.  nodes: n x dim."""
    nodes, pn = _d(nodes)
    n, dim = nodes.shape
    tris, pt = _i32(tris)
    m = tris.shape[0]
    if elems is None:
        ne, pe = m, None
    else:
        elems, pe = _i64(elems)
        ne = elems.shape[0]
    out = np.empty((ne, k), dtype=np.int32)
    rc = lib().or_knn(pn, n, dim, pt, m, pe, ne, k, out.ctypes.data_as(_ip))
    if rc != 0:
        raise ValueError("or_knn: bad arguments")
    return out


def knn_at(nodes, centers, k):
    """The k nodes nearest to each of the given centres (m x dim), ordered by (squared
    distance, index) ascending: the selection of §3.1 around arbitrary points."""
    nodes, pn = _d(nodes)
    n, dim = nodes.shape
    centers, pc = _d(centers)
    m = centers.shape[0]
    out = np.empty((m, k), dtype=np.int32)
    if lib().or_knn_at(pn, n, dim, pc, m, k, out.ctypes.data_as(_ip)) != 0:
        raise ValueError("or_knn_at: bad arguments")
    return out


# ---------------------------------------------------------------------------- §3.2

def tri_r3(p, tri):
    """Integral over the planar triangle ``tri`` (3 x 2) of |x - p|^3."""
    p, pp = _d(p)
    tri, pt = _d(tri)
    return float(lib().or_tri_r3(pp, pt))


def tri_mono(a, b, tri):
    """Integral over the planar triangle ``tri`` (3 x 2) of x^a y^b."""
    tri, pt = _d(tri)
    return float(lib().or_tri_mono(int(a), int(b), pt))


def element_weights_local(xi, tri, deg):
    """RBF-QF weights of one element in its own (scaled) coordinates, Eq. (3.5)."""
    xi, px = _d(xi)
    tri, pt = _d(tri)
    k = xi.shape[0]
    w = np.empty(k)
    rc = lib().or_element_weights_local(px, k, pt, int(deg), w.ctypes.data_as(_dp))
    if rc != 0:
        raise np.linalg.LinAlgError(f"singular element system (rc={rc})")
    return w


def tri_neighbors(tris):
    tris, pt = _i32(tris)
    nbr = np.empty((tris.shape[0], 3), dtype=np.int64)
    lib().or_tri_neighbors(pt, tris.shape[0], nbr.ctypes.data_as(_lp))
    return nbr


def projection_point(nodes, normals, tris, nbr, e):
    """Projection point p_E of §3.3 (None when the cutting planes are near parallel)."""
    nodes, pn = _d(nodes)
    normals, pN = _d(normals)
    tris, pt = _i32(tris)
    nbr, pb = _i64(nbr)
    p = np.empty(3)
    ok = lib().or_projection_point(pn, pN, pt, pb, int(e), p.ctypes.data_as(_dp))
    return p if ok else None


def surface_element_weights(nodes, normals, tris, nbr, e, stencil, deg):
    """Weights (including the Jacobian of mu_E) and Jacobians of one surface element."""
    nodes, pn = _d(nodes)
    normals, pN = _d(normals)
    tris, pt = _i32(tris)
    nbr, pb = _i64(nbr)
    sten, ps = _i32(stencil)
    k = sten.shape[0]
    w = np.empty(k)
    jac = np.empty(k)
    central = C.c_int(0)
    rc = lib().or_surface_element_weights(pn, pN, pt, pb, int(e), ps, k, int(deg), w.ctypes.data_as(_dp),
                                          jac.ctypes.data_as(_dp), C.byref(central))
    if rc != 0:
        raise np.linalg.LinAlgError(f"singular element system (rc={rc})")
    return w, jac, bool(central.value)


def quad_weights(nodes, tris, stencils, deg, normals=None, return_elem=False):
    """Quadrature weights mu_j (Eq. (3.5) flat, §3.3 surfaces).  nodes: n x dim."""
    nodes, pn = _d(nodes)
    n, dim = nodes.shape
    tris, pt = _i32(tris)
    st, ps = _i32(stencils)
    m, k = st.shape
    if normals is not None:
        normals, pN = _d(normals)
    else:
        pN = None
    q = np.empty(n)
    W = np.empty((m, k))
    bad = C.c_int64(-1)
    rc = lib().or_quad_weights(pn, pN, n, dim, pt, m, ps, k, int(deg), q.ctypes.data_as(_dp),
                               W.ctypes.data_as(_dp), C.byref(bad))
    if rc < 0:
        raise ValueError("or_quad_weights: bad arguments")
    if rc > 0:
        raise np.linalg.LinAlgError(f"singular element system at element {bad.value}")
    return (q, W) if return_elem else q


# ---------------------------------------------------------------------------- §2.2

def _kern(kernel, period=0.0):
    """(A1, s1, A2, s2) plus the period L of the flat doubly periodic square (0: Euclidean
    distance).  A fifth entry of ``kernel`` is taken as the period when given."""
    k = [float(v) for v in kernel]
    if len(k) == 4:
        k.append(float(period))
    return _d(np.asarray(k[:5], dtype=np.float64))


def nonlocal_sum(x, q, u, kernel, beta, theta, rows=None, period=0.0):
    """I[b, i] = sum_j w(|x_i - x_j|) q_j f_b(u[b, j]) for all rows (or ``rows``).
    x: n x 3, u: B x n (or n), kernel: (A1, s1, A2, s2); period > 0 takes |x_i - x_j| as
    the doubly periodic distance of Eq. (dist) on the square of that side."""
    x, px = _d(x)
    q, pq = _d(q)
    u = np.atleast_2d(u)
    u, pu = _d(u)
    B, n = u.shape
    kp, pk = _kern(kernel, period)
    be, pbe = _d(np.broadcast_to(np.asarray(beta, dtype=np.float64), (B,)))
    th, pth = _d(np.broadcast_to(np.asarray(theta, dtype=np.float64), (B,)))
    if rows is None:
        I = np.empty((B, n))
        lib().or_nonlocal(px, pq, n, pu, B, pk, pbe, pth, None, 0, I.ctypes.data_as(_dp))
    else:
        rows, pr = _i64(rows)
        I = np.empty((B, rows.shape[0]))
        lib().or_nonlocal(px, pq, n, pu, B, pk, pbe, pth, pr, rows.shape[0], I.ctypes.data_as(_dp))
    return I


def _forcing_arr(forcing):
    if forcing is None:
        return None, None
    if forcing["kind"] == 2:
        f = np.asarray([2, forcing["c"], forcing["radius"], forcing["sigma"], forcing["scale"], 0.0],
                       dtype=np.float64)
    else:
        f = np.asarray([forcing["kind"], forcing["c"], forcing["a0"], *forcing["lam"]], dtype=np.float64)
    return _d(f)


def rk4(x, q, u0, kernel, beta, theta, t0, dt, nsteps, forcing=None, return_stages=False, period=0.0):
    """Classical RK4 for Eq. (2.9); returns u(t0 + nsteps dt) (B x n)."""
    x, px = _d(x)
    q, pq = _d(q)
    u = np.array(np.atleast_2d(u0), dtype=np.float64, order="C")
    B, n = u.shape
    kp, pk = _kern(kernel, period)
    be, pbe = _d(np.broadcast_to(np.asarray(beta, dtype=np.float64), (B,)))
    th, pth = _d(np.broadcast_to(np.asarray(theta, dtype=np.float64), (B,)))
    f, pf = _forcing_arr(forcing)
    st = np.empty((nsteps, 4, B, n)) if return_stages else None
    lib().or_rk4(px, pq, n, u.ctypes.data_as(_dp), B, t0, dt, nsteps, pk, pbe, pth, pf,
                 st.ctypes.data_as(_dp) if st is not None else None)
    return (u, st) if return_stages else u


def adjoint(x, q, u0, kernel, beta, theta, t0, dt, nsteps, lam_T, forcing=None, period=0.0):
    """Discrete RK4 adjoint: returns (dL/du0 (B x n), dL/d(A1,s1,A2,s2) (B x 4))."""
    x, px = _d(x)
    q, pq = _d(q)
    u0 = np.atleast_2d(u0)
    u0, pu = _d(u0)
    B, n = u0.shape
    kp, pk = _kern(kernel, period)
    be, pbe = _d(np.broadcast_to(np.asarray(beta, dtype=np.float64), (B,)))
    th, pth = _d(np.broadcast_to(np.asarray(theta, dtype=np.float64), (B,)))
    f, pf = _forcing_arr(forcing)
    lam, pl = _d(np.atleast_2d(lam_T))
    gu = np.empty((B, n))
    gk = np.empty((B, 4))
    lib().or_adjoint(px, pq, n, pu, B, t0, dt, nsteps, pk, pbe, pth, pf, pl, gu.ctypes.data_as(_dp),
                     gk.ctypes.data_as(_dp))
    return gu, gk


def loss(x, q, u0, kernel, beta, theta, t0, dt, nsteps, target, forcing=None, period=0.0):
    """L = sum (u_N - target)^2 after nsteps RK4 steps."""
    x, px = _d(x)
    q, pq = _d(q)
    u0 = np.atleast_2d(u0)
    u0, pu = _d(u0)
    B, n = u0.shape
    kp, pk = _kern(kernel, period)
    be, pbe = _d(np.broadcast_to(np.asarray(beta, dtype=np.float64), (B,)))
    th, pth = _d(np.broadcast_to(np.asarray(theta, dtype=np.float64), (B,)))
    f, pf = _forcing_arr(forcing)
    tg, ptg = _d(np.atleast_2d(target))
    return float(lib().or_loss(px, pq, n, pu, B, t0, dt, nsteps, pk, pbe, pth, pf, ptg))


def mms_sphere_eigs(kernel, period=0.0):
    """Funk-Hecke eigenvalues (lambda_0, lambda_1, lambda_2) of the radial kernel on the
    unit sphere, by composite Gauss-Legendre quadrature."""
    kp, pk = _kern(kernel, period)
    lam = np.empty(3)
    lib().or_mms_sphere_eigs(pk, lam.ctypes.data_as(_dp))
    return lam


def mms_sphere_forcing(kernel, c=0.5, a0=0.3):
    """Forcing descriptor for the manufactured sphere solution (kind 1)."""
    return {"kind": 1, "c": c, "a0": a0, "lam": tuple(mms_sphere_eigs(kernel))}


def mms_sphere_solution(x, t, beta, theta, c=0.5, a0=0.3):
    x, px = _d(x)
    u = np.empty(x.shape[0])
    lib().or_mms_sphere_solution(px, x.shape[0], t, c, a0, beta, theta, u.ctypes.data_as(_dp))
    return u


def mms_flat_forcing(c=0.1, radius=0.2, sigma=1.1, scale=1.0):
    """Forcing descriptor for the manufactured solution on the flat periodic square
    (kind 2): a Gaussian of width sigma whose centre circles the origin at ``radius``, plus
    c, as the firing rate; ``scale`` multiplies the convolution term (1 flat, r torus)."""
    return {"kind": 2, "c": c, "radius": radius, "sigma": sigma, "scale": scale}


def mms_flat_solution(x, t, kernel, period, beta, theta, c=0.1, radius=0.2, sigma=1.1):
    """u*(t, x) of the kind-2 manufactured solution at nodes (x, y, .) of the square."""
    x, px = _d(x)
    kp, pk = _kern(kernel, period)
    u = np.empty(x.shape[0])
    lib().or_mms_flat_solution(px, x.shape[0], t, pk, radius, sigma, c, beta, theta, u.ctypes.data_as(_dp))
    return u


def mms_flat_forcing_values(x, t, kernel, period, beta, theta, c=0.1, radius=0.2, sigma=1.1, scale=1.0):
    """gamma(t, x) of the kind-2 manufactured solution (the convolution by panel quadrature)."""
    x, px = _d(x)
    kp, pk = _kern(kernel, period)
    g = np.empty(x.shape[0])
    lib().or_mms_flat_forcing(px, x.shape[0], t, pk, radius, sigma, c, scale, beta, theta, g.ctypes.data_as(_dp))
    return g


def _model_arr(kind=0, rate=0, a=0.06, b=0.54, tau=1.0, beta_d=0.0):
    return np.array([kind, rate, a, b, tau, beta_d], dtype=np.float64)


def rate(u, beta=1.0, theta=0.0, kind=0, a=0.06, b=0.54):
    """Firing rate of the §5 models at every entry of u: kind 0 sigmoid (beta, theta),
    kind 1 the C^4 smooth step on [a, b] (Eq. (smoothf))."""
    m, pm = _d(_model_arr(0, kind, a, b))
    u = np.asarray(u, dtype=np.float64)
    return np.vectorize(lambda v: lib().or_rate(pm, float(v), float(beta), float(theta)))(u)


def ab5_weights():
    """Adams-Bashforth 5 weights c_0..c_4 (for F_n, F_{n-1}, ..., F_{n-4})."""
    c = np.empty(5)
    lib().or_ab5_weights(c.ctypes.data_as(_dp))
    return c


def field_advance(x, mu, u0, kernel, beta, theta, dt, nsteps, s0=None, kind=0, rate_kind=0, a=0.06, b=0.54,
                  tau=1.0, beta_d=0.0, integrator="rk4", period=0.0):
    """§5 models on the nodes: kind 0 the neural field of Eq. (2.9), kind 1 the
    synaptic-depression model (Eq. (nfsyndep), efficacy s); rate_kind 0 sigmoid, 1 smooth
    step on [a, b]; integrator "rk4" or "ab5" (started by four RK4 steps).
    Returns u (B x n), or (u, s) for kind 1."""
    x, px = _d(x)
    mu, pq = _d(mu)
    u = np.array(np.atleast_2d(u0), dtype=np.float64, order="C")
    B, n = u.shape
    s = np.array(np.atleast_2d(s0), dtype=np.float64, order="C") if kind == 1 else None
    kp, pk = _kern(kernel, period)
    be, pbe = _d(np.broadcast_to(np.asarray(beta, dtype=np.float64), (B,)))
    th, pth = _d(np.broadcast_to(np.asarray(theta, dtype=np.float64), (B,)))
    m, pm = _d(_model_arr(kind, rate_kind, a, b, tau, beta_d))
    lib().or_field_advance(px, pq, n, u.ctypes.data_as(_dp), s.ctypes.data_as(_dp) if s is not None else None, B,
                           0.0, dt, nsteps, pk, pbe, pth, pm, 1 if integrator == "ab5" else 0)
    return (u, s) if kind == 1 else u
