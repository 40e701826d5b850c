"""The seeded input generators: deterministic, inside their domains, triangulations that
cover the domain with consistently oriented triangles.  CPU only."""
import math

import numpy as np
from scipy.spatial import cKDTree

import nodesets


def _tri_areas2(x2, tris):
    a, b, c = x2[tris[:, 0]], x2[tris[:, 1]], x2[tris[:, 2]]
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])


def test_square_families_cover_the_square():
    for ns in (nodesets.square_halton(2000), nodesets.square_repulsion(2000), nodesets.square_regular(30)):
        x2 = ns.coords()
        assert x2.min() >= 0.0 and x2.max() <= 1.0
        area2 = _tri_areas2(x2, ns.tris)
        assert (area2 > 0).all()                        # counter-clockwise, no degenerate triangle
        assert abs(0.5 * area2.sum() - 1.0) < 1e-12     # the triangles tile the square


def test_square_repulsion_is_deterministic_and_spread():
    a, b = nodesets.square_repulsion(2000), nodesets.square_repulsion(2000)
    np.testing.assert_array_equal(a.nodes, b.nodes)
    np.testing.assert_array_equal(a.tris, b.tris)
    halton = nodesets.square_halton(2000)
    nb = a.meta["n_boundary"]
    np.testing.assert_array_equal(a.nodes[:nb], halton.nodes[:nb])  # the boundary stays put
    s = math.sqrt(1.0 / a.n)
    d_rep = cKDTree(a.coords()).query(a.coords(), 2)[0][:, 1].min()
    d_hal = cKDTree(halton.coords()).query(halton.coords(), 2)[0][:, 1].min()
    assert d_rep > 0.5 * s > d_hal                    # repulsion removes the close pairs


def test_surface_sets_have_unit_outward_normals():
    for ns in (nodesets.sphere_fibonacci(3000), nodesets.ellipsoid_fibonacci(3000),
               nodesets.torus_lattice(4000)):
        nrm = ns.normals
        np.testing.assert_allclose(np.linalg.norm(nrm, axis=1), 1.0, atol=1e-12)
        a, b, c = (ns.nodes[ns.tris[:, i]] for i in range(3))
        face = np.cross(b - a, c - a)
        vert = nrm[ns.tris].sum(1)
        assert ((face * vert).sum(1) > 0).all()         # faces oriented along the node normals
