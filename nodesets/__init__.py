"""Seeded synthetic inputs for the RBF neural-field workloads.

This module is shared by the CPU oracle tests and the GPU path (tests, benchmark,
smoke check).  It produces *inputs only*: node sets, triangulations, node normals,
initial states and per-trajectory parameters.  It holds none of the method's
arithmetic (no stencils, no quadrature weights, no kernel sums, no time stepping);
those live, independently, in ``oracle/`` and in the CUDA library.

Workload shapes follow the paper's experiments (§4.1 node selection, §4.4 torus,
Supplementary sphere) and the five benchmark configurations:

* flat unit square: equispaced boundary nodes plus Halton interior nodes, Delaunay
  triangulation (§4.1 uses boundary nodes plus scattered interior nodes);
* unit sphere: Fibonacci nodes with seeded tangential jitter, convex-hull triangulation;
* torus (R, r): the paper's "spiral" triangular lattice in (phi, theta) (§4.1), with
  seeded jitter bounded well below the lattice spacing so the lattice connectivity
  remains a valid triangulation;
* ellipsoid: a Fibonacci sphere mapped by diag(axes) (hull connectivity is preserved
  by the affine map).

All triangles are returned counter-clockwise with respect to the outward normal
(flat domains: counter-clockwise in the plane).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "NodeSet", "halton", "square_halton", "square_regular", "sphere_fibonacci",
    "torus_lattice", "ellipsoid_fibonacci", "torus_point", "bump_u0",
    "spiral_bumps_u0", "random_bumps", "mexican_hat_cfg",
]


@dataclass
class NodeSet:
    """Nodes (n x 3, float64; z = 0 on flat domains), optional outward normals
    (n x 3) and a triangulation (m x 3 int32, CCW w.r.t. the outward normal)."""
    nodes: np.ndarray
    tris: np.ndarray
    normals: np.ndarray | None
    dim: int
    area: float | None = None          # exact area of the domain when known
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def m(self) -> int:
        return int(self.tris.shape[0])

    def coords(self) -> np.ndarray:
        """Coordinates with the domain's own dimension (n x dim)."""
        return np.ascontiguousarray(self.nodes[:, : self.dim])


# ----------------------------------------------------------------------------------
# low-level helpers
# ----------------------------------------------------------------------------------

def halton(index: np.ndarray, base: int) -> np.ndarray:
    """Radical inverse of integer ``index`` in ``base`` (the Halton sequence)."""
    index = np.asarray(index, dtype=np.int64).copy()
    out = np.zeros(index.shape, dtype=np.float64)
    f = 1.0
    while np.any(index > 0):
        f /= base
        out += f * (index % base)
        index //= base
    return out


def _orient_flat(nodes2: np.ndarray, tris: np.ndarray) -> np.ndarray:
    a, b, c = nodes2[tris[:, 0]], nodes2[tris[:, 1]], nodes2[tris[:, 2]]
    cr = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    t = tris.copy()
    flip = cr < 0
    t[flip, 1], t[flip, 2] = tris[flip, 2], tris[flip, 1]
    return t.astype(np.int32)


def _orient_outward(nodes: np.ndarray, tris: np.ndarray, outward: np.ndarray) -> np.ndarray:
    a, b, c = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    ref = outward[tris[:, 0]] + outward[tris[:, 1]] + outward[tris[:, 2]]
    t = tris.copy()
    flip = np.einsum("ij,ij->i", nrm, ref) < 0
    t[flip, 1], t[flip, 2] = tris[flip, 2], tris[flip, 1]
    return t.astype(np.int32)


def _pad3(x2: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([x2, np.zeros((x2.shape[0], 1))], axis=1))


# ----------------------------------------------------------------------------------
# flat unit square
# ----------------------------------------------------------------------------------

def _square_boundary(per_side: int) -> np.ndarray:
    t = np.arange(per_side, dtype=np.float64) / per_side
    z, o = np.zeros_like(t), np.ones_like(t)
    return np.concatenate([
        np.stack([t, z], 1), np.stack([o, t], 1),
        np.stack([1.0 - t, o], 1), np.stack([z, 1.0 - t], 1)])


def square_halton(n: int = 1500, seed: int = 0) -> NodeSet:
    """Unit square [0,1]^2: 4*floor(sqrt(n)) equispaced boundary nodes (corners
    included) and Halton (2,3) interior nodes starting at index 1+seed.  Interior
    candidates closer than a quarter of the boundary spacing to the boundary are
    skipped so no sliver elements form there.  Delaunay triangulation."""
    from scipy.spatial import Delaunay
    per_side = int(math.isqrt(n))
    bnd = _square_boundary(per_side)
    n_int = n - bnd.shape[0]
    h = 1.0 / per_side
    pts = []
    idx = 1 + seed
    while len(pts) < n_int:
        cand = np.arange(idx, idx + 2 * n_int, dtype=np.int64)
        idx += 2 * n_int
        xy = np.stack([halton(cand, 2), halton(cand, 3)], 1)
        keep = np.all((xy > 0.25 * h) & (xy < 1.0 - 0.25 * h), axis=1)
        pts.extend(xy[keep].tolist())
    interior = np.asarray(pts[:n_int], dtype=np.float64)
    x2 = np.concatenate([bnd, interior])
    tris = _orient_flat(x2, Delaunay(x2).simplices)
    return NodeSet(_pad3(x2), tris, None, 2, area=1.0,
                   meta={"kind": "square_halton", "n_boundary": bnd.shape[0], "seed": seed})


def square_repulsion(n: int = 2000, iters: int = 60, seed: int = 0) -> NodeSet:
    """Unit square with the paper's second node family (§4): interior nodes spread by a
    deterministic point-repulsion process, equispaced boundary nodes.  Starts from the
    nodes of ``square_halton``; each iteration moves every interior node by a tenth of the
    mean spacing s = n^-1/2 along the sum of the unit vectors away from its 8 nearest nodes,
    weighted (s / d)^3 (the step shrinks where that sum is below 1), boundary nodes fixed,
    and keeps it half a boundary spacing inside the square.  Delaunay triangulation."""
    from scipy.spatial import Delaunay, cKDTree
    base = square_halton(n, seed)
    x2 = base.coords().copy()
    nb = base.meta["n_boundary"]
    h = 1.0 / int(math.isqrt(n))
    s = math.sqrt(1.0 / n)
    for _ in range(iters):
        d, idx = cKDTree(x2).query(x2[nb:], 9)
        d, idx = d[:, 1:], idx[:, 1:]
        away = (x2[nb:, None, :] - x2[idx]) / d[..., None]
        f = (away * ((s / d) ** 3)[..., None]).sum(1)
        mag = np.linalg.norm(f, axis=1, keepdims=True)
        x2[nb:] += 0.1 * s * f / np.maximum(mag, 1e-300) * np.minimum(1.0, mag)
        x2[nb:] = np.clip(x2[nb:], 0.5 * h, 1.0 - 0.5 * h)
    tris = _orient_flat(x2, Delaunay(x2).simplices)
    return NodeSet(_pad3(x2), tris, None, 2, area=1.0,
                   meta={"kind": "square_repulsion", "n_boundary": nb, "iters": iters, "seed": seed})


def square_regular(rows: int = 24) -> NodeSet:
    """Unit square with interior nodes on an equilateral triangular lattice and
    equispaced boundary nodes (the paper's "regular grid", §4.1 and Supplementary).
    Returns the lattice spacing ``s`` in ``meta``; interior cell area is sqrt(3)/2 s^2."""
    from scipy.spatial import Delaunay
    s = 1.0 / rows
    dy = s * math.sqrt(3.0) / 2.0
    pts = []
    j = 1
    while j * dy < 1.0 - 0.5 * dy:
        off = 0.5 * s if (j % 2) else 0.0
        i = 0
        while True:
            x = off + i * s
            if x >= 1.0 - 0.25 * s:
                break
            if x > 0.25 * s:
                pts.append((x, j * dy))
            i += 1
        j += 1
    interior = np.asarray(pts)
    per_side = rows
    bnd = _square_boundary(per_side)
    x2 = np.concatenate([bnd, interior])
    tris = _orient_flat(x2, Delaunay(x2).simplices)
    return NodeSet(_pad3(x2), tris, None, 2, area=1.0,
                   meta={"kind": "square_regular", "s": s, "n_boundary": bnd.shape[0]})


# ----------------------------------------------------------------------------------
# curved closed surfaces
# ----------------------------------------------------------------------------------

def _fibonacci(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], 1)


def _tangent_frame(p: np.ndarray):
    ref = np.where(np.abs(p[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(ref, p)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(p, e1)
    return e1, e2


def _hull_tris(p: np.ndarray) -> np.ndarray:
    from scipy.spatial import ConvexHull
    return ConvexHull(p).simplices.astype(np.int32)


def sphere_fibonacci(n: int = 20000, jitter: float = 0.1, seed: int = 0) -> NodeSet:
    """Unit sphere: Fibonacci nodes, each moved by a seeded uniform tangential offset
    in [-jitter*h, jitter*h]^2 (h = sqrt(4 pi / n)) and re-projected to the sphere."""
    p = _fibonacci(n)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        h = math.sqrt(4.0 * math.pi / n)
        e1, e2 = _tangent_frame(p)
        off = rng.uniform(-jitter * h, jitter * h, size=(n, 2))
        p = p + off[:, :1] * e1 + off[:, 1:] * e2
        p /= np.linalg.norm(p, axis=1, keepdims=True)
    tris = _orient_outward(p, _hull_tris(p), p)
    return NodeSet(np.ascontiguousarray(p), tris, np.ascontiguousarray(p.copy()), 3,
                   area=4.0 * math.pi, meta={"kind": "sphere", "jitter": jitter, "seed": seed})


def ellipsoid_fibonacci(n: int, axes=(1.0, 0.8, 0.6), jitter: float = 0.1, seed: int = 0) -> NodeSet:
    """Ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 = 1: a jittered Fibonacci sphere mapped
    by diag(a, b, c).  Normals are the normalised gradients of the implicit form."""
    s = sphere_fibonacci(n, jitter, seed)
    ax = np.asarray(axes, dtype=np.float64)
    p = s.nodes * ax
    nrm = p / (ax * ax)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    tris = _orient_outward(p, s.tris, nrm)
    return NodeSet(np.ascontiguousarray(p), tris, np.ascontiguousarray(nrm), 3, area=None,
                   meta={"kind": "ellipsoid", "axes": tuple(axes), "seed": seed})


def torus_point(phi, theta, R: float, r: float) -> np.ndarray:
    """The torus parametrisation of §4, Eq. (4.1)."""
    phi = np.asarray(phi, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    return np.stack([(R + r * np.cos(theta)) * np.cos(phi),
                     (R + r * np.cos(theta)) * np.sin(phi),
                     r * np.sin(theta)], -1)


def _torus_rows(n: int, R: float, r: float) -> int:
    # near-equilateral lattice: rows of constant theta spaced (sqrt3/2) x node spacing
    target = math.sqrt(n / ((math.sqrt(3.0) / 2.0) * R / r))
    best = None
    for rows in range(4, n // 4 + 1, 2):
        if n % rows:
            continue
        if best is None or abs(rows - target) < abs(best - target):
            best = rows
    if best is None:
        raise ValueError(f"no even row count divides n={n}")
    return best


def _lattice_tris(rows: int, cols: int) -> np.ndarray:
    """Triangles of the doubly periodic staggered lattice (node t * cols + p; odd rows
    shifted by half a spacing)."""
    tris = []
    for t in range(rows):
        t1 = (t + 1) % rows
        p = np.arange(cols)
        p1 = (p + 1) % cols
        a = t * cols + p
        b = t * cols + p1
        c = t1 * cols + p
        d = t1 * cols + p1
        if t % 2 == 0:       # next row is shifted by +1/2
            tris.append(np.stack([a, b, c], 1))
            tris.append(np.stack([b, d, c], 1))
        else:                # this row is shifted by +1/2
            tris.append(np.stack([a, d, c], 1))
            tris.append(np.stack([a, b, d], 1))
    return np.concatenate(tris).astype(np.int32)


def torus_lattice(n: int = 100000, R: float = 1.0, r: float = 0.4, jitter: float = 0.15,
                  seed: int = 0) -> NodeSet:
    """Torus of major radius R and minor radius r sampled on the staggered triangular
    ("spiral") lattice of §4.1: an even number of rows of constant theta, equal phi
    spacing, alternate rows shifted by half a spacing.  Each node is then moved by a
    seeded uniform offset of at most ``jitter`` lattice spacings in (phi, theta)."""
    rows = _torus_rows(n, R, r)
    cols = n // rows
    t_idx = np.repeat(np.arange(rows), cols)
    p_idx = np.tile(np.arange(cols), rows)
    off = 0.5 * (t_idx % 2)
    dphi, dth = 2.0 * math.pi / cols, 2.0 * math.pi / rows
    phi = (p_idx + off) * dphi
    th = t_idx * dth
    if jitter > 0:
        rng = np.random.default_rng(seed)
        j = rng.uniform(-jitter, jitter, size=(n, 2))
        phi = phi + j[:, 0] * dphi
        th = th + j[:, 1] * dth
    x = torus_point(phi, th, R, r)
    nrm = np.stack([np.cos(th) * np.cos(phi), np.cos(th) * np.sin(phi), np.sin(th)], 1)
    tris = _orient_outward(x, _lattice_tris(rows, cols), nrm)
    return NodeSet(np.ascontiguousarray(x), tris, np.ascontiguousarray(nrm), 3,
                   area=4.0 * math.pi ** 2 * R * r,
                   meta={"kind": "torus", "R": R, "r": r, "rows": rows, "cols": cols,
                         "phi": phi, "theta": th, "seed": seed})


# ----------------------------------------------------------------------------------
# initial states and parameters
# ----------------------------------------------------------------------------------

@dataclass
class MexicanHat:
    """w(r) = A1 exp(-r^2/s1^2) - A2 exp(-r^2/s2^2) (lateral inhibition, §5 Eq. (5.1)
    in its unnormalised form)."""
    A1: float = 1.0
    s1: float = 0.1
    A2: float = 0.5
    s2: float = 0.2

    def astuple(self):
        return (self.A1, self.s1, self.A2, self.s2)


def mexican_hat_cfg() -> MexicanHat:
    return MexicanHat()


def bump_u0(nodes: np.ndarray, center, amp: float = 0.8, width: float = 0.1) -> np.ndarray:
    """amp * exp(-|x - center|^2 / (2 width^2))."""
    d = nodes - np.asarray(center, dtype=np.float64)[None, :]
    return amp * np.exp(-np.einsum("ij,ij->i", d, d) / (2.0 * width * width))


def spiral_bumps_u0(ns: NodeSet, count: int = 6, amp: float = 0.5, width: float = 0.15) -> np.ndarray:
    """Sum of phase-shifted bumps placed along a closed spiral on the torus:
    centres at (phi, theta) = (2 pi m / count, pi m / 3), m = 0..count-1."""
    R, r = ns.meta["R"], ns.meta["r"]
    u = np.zeros(ns.n)
    for m in range(count):
        c = torus_point(2.0 * math.pi * m / count, math.pi * m / 3.0, R, r)
        u += bump_u0(ns.nodes, c, amp, width)
    return u


def random_bumps(ns: NodeSet, B: int, seed: int, axes=(1.0, 1.0, 1.0)):
    """Per-trajectory random bump u0 and firing-rate parameters for batched runs:
    amplitude U[0.5, 1], width U[0.1, 0.3], centre uniform on the unit sphere mapped
    by diag(axes); beta U[10, 40], theta U[0.1, 0.3]."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.5, 1.0, B)
    wid = rng.uniform(0.1, 0.3, B)
    c = rng.normal(size=(B, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    c *= np.asarray(axes)[None, :]
    beta = rng.uniform(10.0, 40.0, B)
    theta = rng.uniform(0.1, 0.3, B)
    u0 = np.stack([bump_u0(ns.nodes, c[b], amp[b], wid[b]) for b in range(B)])
    return u0, beta, theta


# ----------------------------------------------------------------------------------
# further curved geometries of the paper (§5 deformed spheres; the ring Dupin cyclide of
# the convergence appendix)
# ----------------------------------------------------------------------------------

def _deformed_h(rho2, gamma):
    return np.sqrt(1.0 - gamma / (1.0 + rho2 / 2.89))


def deformed_sphere(n: int, gamma: float = 0.4, jitter: float = 0.1, seed: int = 0) -> NodeSet:
    """The one-parameter family D_gamma of §5: 1 = x^2 + y^2 + z^2 / (1 - gamma / (1 +
    (x^2 + y^2) / 2.89)).  A jittered Fibonacci sphere mapped by z -> z h(x^2 + y^2),
    h = sqrt(1 - gamma / (1 + rho^2 / 2.89)) (rho^2 = x^2 + y^2 is kept), with the sphere's
    hull connectivity; normals are the normalised gradients of the implicit form."""
    s = sphere_fibonacci(n, jitter, seed)
    p = s.nodes.copy()
    rho2 = p[:, 0] ** 2 + p[:, 1] ** 2
    p[:, 2] *= _deformed_h(rho2, gamma)
    g = 1.0 - gamma / (1.0 + rho2 / 2.89)
    dg = gamma / (2.89 * (1.0 + rho2 / 2.89) ** 2)        # dg / d(rho^2)
    z2 = p[:, 2] ** 2
    grad = np.stack([2 * p[:, 0] * (1 - z2 * dg / g ** 2), 2 * p[:, 1] * (1 - z2 * dg / g ** 2), 2 * p[:, 2] / g], 1)
    nrm = grad / np.linalg.norm(grad, axis=1, keepdims=True)
    tris = _orient_outward(p, s.tris, nrm)
    return NodeSet(np.ascontiguousarray(p), tris, np.ascontiguousarray(nrm), 3, area=deformed_sphere_area(gamma),
                   meta={"kind": "deformed_sphere", "gamma": gamma, "seed": seed})


def deformed_sphere_area(gamma: float) -> float:
    """Area of D_gamma: surface of revolution rho = sin t, z = cos t h(sin^2 t), integrated
    in t by 400-point Gauss-Legendre (the profile is smooth)."""
    x, w = np.polynomial.legendre.leggauss(400)
    t = 0.5 * math.pi * (x + 1.0)
    eps = 1e-6
    def prof(tt):
        return np.sin(tt), np.cos(tt) * _deformed_h(np.sin(tt) ** 2, gamma)
    r0, z0 = prof(t)
    rp, zp = prof(t + eps)
    rm, zm = prof(t - eps)
    ds = np.hypot((rp - rm) / (2 * eps), (zp - zm) / (2 * eps))
    return float(2.0 * math.pi * 0.5 * math.pi * np.sum(w * r0 * ds))


def cyclide_point(phi, theta, a=1.0, b=0.98, c=0.1983, d=0.5) -> np.ndarray:
    """Dupin cyclide, standard parametrisation over (phi, theta) in [0, 2 pi)^2 (ring case
    for c < d < a)."""
    phi = np.asarray(phi, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    den = a - c * np.cos(theta) * np.cos(phi)
    x = (d * (c - a * np.cos(theta) * np.cos(phi)) + b * b * np.cos(theta)) / den
    y = b * np.sin(theta) * (a - d * np.cos(phi)) / den
    z = b * np.sin(phi) * (c * np.cos(theta) - d) / den
    return np.stack([x, y, z], -1)


def _cyclide_frame(phi, theta, eps=1e-6, **kw):
    xp = (cyclide_point(phi + eps, theta, **kw) - cyclide_point(phi - eps, theta, **kw)) / (2 * eps)
    xt = (cyclide_point(phi, theta + eps, **kw) - cyclide_point(phi, theta - eps, **kw)) / (2 * eps)
    return np.cross(xp, xt)


def cyclide_area(a=1.0, b=0.98, c=0.1983, d=0.5, m: int = 600) -> float:
    """Area of the cyclide by the periodic trapezoid rule on an m x m parameter grid
    (spectrally accurate for the smooth periodic area element)."""
    g = 2.0 * math.pi * np.arange(m) / m
    P, T = np.meshgrid(g, g, indexing="ij")
    J = np.linalg.norm(_cyclide_frame(P, T, a=a, b=b, c=c, d=d), axis=-1)
    return float(J.sum() * (2.0 * math.pi / m) ** 2)


def cyclide_integral(f, a=1.0, b=0.98, c=0.1983, d=0.5, m: int = 600) -> float:
    """Integral of f(x, y, z) over the cyclide (periodic trapezoid rule, m x m grid)."""
    g = 2.0 * math.pi * np.arange(m) / m
    P, T = np.meshgrid(g, g, indexing="ij")
    X = cyclide_point(P, T, a=a, b=b, c=c, d=d)
    J = np.linalg.norm(_cyclide_frame(P, T, a=a, b=b, c=c, d=d), axis=-1)
    return float((f(X[..., 0], X[..., 1], X[..., 2]) * J).sum() * (2.0 * math.pi / m) ** 2)


def cyclide_lattice(n: int, a=1.0, b=0.98, c=0.1983, d=0.5, rows: int | None = None) -> NodeSet:
    """Ring Dupin cyclide on a non-random staggered triangular lattice in (phi, theta)
    parameter space (the appendix's mesh): rows of constant theta, odd rows shifted by
    half a spacing.  Normals from the parametrisation's tangent vectors, oriented outward
    (positive enclosed volume)."""
    if rows is None:
        # near-equilateral triangles: the theta circles are about twice as long as the phi
        # circles (mean 2 pi vs pi for these parameters), so theta gets rows spaced
        # sqrt(3)/2 of the phi spacing: cols / rows = (sqrt(3)/2) (1 / 2)
        rows = max(4, int(round(math.sqrt(n / (0.25 * math.sqrt(3.0))) / 2.0)) * 2)
    cols = n // rows
    t_idx = np.repeat(np.arange(rows), cols)
    p_idx = np.tile(np.arange(cols), rows)
    th = t_idx * (2.0 * math.pi / rows)
    ph = (p_idx + 0.5 * (t_idx % 2)) * (2.0 * math.pi / cols)
    x = cyclide_point(ph, th, a=a, b=b, c=c, d=d)
    nrm = _cyclide_frame(ph, th, a=a, b=b, c=c, d=d)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    tris = _lattice_tris(rows, cols)
    # orient normals outward: the triangulated surface must enclose a positive volume
    tri_n = np.cross(x[tris[:, 1]] - x[tris[:, 0]], x[tris[:, 2]] - x[tris[:, 0]])
    align = np.sign(np.einsum("ij,ij->i", tri_n, nrm[tris[:, 0]]))
    vol = np.sum(np.einsum("ij,ij->i", x[tris[:, 0]], tri_n) * align) / 6.0
    if vol < 0:
        nrm = -nrm
    tris = _orient_outward(x, tris, nrm)
    return NodeSet(np.ascontiguousarray(x), tris, np.ascontiguousarray(nrm), 3, area=cyclide_area(a, b, c, d),
                   meta={"kind": "cyclide", "abcd": (a, b, c, d), "rows": rows, "cols": cols})
