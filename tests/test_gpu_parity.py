"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the
same seeded inputs.

Bars: stencil indices bit-exact; quadrature weights within 1e-12 relative
(max-norm); FP32 nonlocal sums and trajectories within 1e-5 relative L2 per
trajectory.  The oracle always receives the FP32-rounded values the GPU sees.
"""

import numpy as np
import pytest
import torch

import nodesets
import oracle
from nodesets import workloads as W

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
Q_REL = 1e-12


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_13379_gb300 as nf
    nf.lib()
    return nf


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel_l2(got, want):
    got, want = np.atleast_2d(got), np.atleast_2d(want)
    return max(np.linalg.norm(g - w) / np.linalg.norm(w) for g, w in zip(got, want))


# ------------------------------------------------------------------ §3.1 stencils

@pytest.mark.parametrize("case", ["square", "sphere", "torus", "ties2d", "ties3d"])
def test_stencils_bit_exact(nf, case):
    if case == "square":
        ns, k = nodesets.square_halton(1500), 24
        X = ns.coords()
    elif case == "sphere":
        ns, k = nodesets.sphere_fibonacci(3000, seed=4), 32
        X = ns.nodes
    elif case == "torus":
        ns, k = nodesets.torus_lattice(6000, seed=5), 48
        X = ns.nodes
    else:  # quantised coordinates: many exact distance ties
        rng = np.random.default_rng(7)
        d = 2 if case == "ties2d" else 3
        X = np.round(rng.uniform(0, 1, size=(2000, d)) * 16) / 16
        tris = rng.integers(0, 2000, size=(3000, 3)).astype(np.int32)
        ns = nodesets.NodeSet(X, tris, None, d)
        k = 40
    got = nf.nf_build_stencils(dev(X, torch.float64), dev(ns.tris, torch.int32), k).cpu().numpy()
    want = oracle.knn(X, ns.tris, k)
    np.testing.assert_array_equal(got, want)


def test_stencils_k_equals_n(nf):
    rng = np.random.default_rng(3)
    X = rng.uniform(size=(40, 2))
    tris = rng.integers(0, 40, size=(7, 3)).astype(np.int32)
    got = nf.nf_build_stencils(dev(X, torch.float64), dev(tris, torch.int32), 40).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.knn(X, tris, 40))


# ------------------------------------------------------------------ §3.2-3.3 weights

def _weights_pair(nf, ns, k, deg):
    X = ns.coords()
    st = oracle.knn(X, ns.tris, k)
    want = oracle.quad_weights(X, ns.tris, st, deg, normals=ns.normals if ns.dim == 3 else None)
    normals = dev(ns.normals, torch.float64) if ns.dim == 3 else None
    got = nf.nf_quad_weights(dev(X, torch.float64), dev(ns.tris, torch.int32), dev(st, torch.int32), deg,
                             normals=normals).cpu().numpy()
    return got, want


@pytest.mark.parametrize("case", ["flat", "sphere", "torus", "ellipsoid", "regular", "deformed", "cyclide"])
def test_quad_weights_match_oracle(nf, case):
    if case == "flat":
        ns, k, deg = nodesets.square_halton(1500), 24, 2
    elif case == "sphere":
        ns, k, deg = nodesets.sphere_fibonacci(4000, seed=1), 32, 3
    elif case == "torus":
        ns, k, deg = nodesets.torus_lattice(8000, seed=2), 48, 4
    elif case == "ellipsoid":
        ns, k, deg = nodesets.ellipsoid_fibonacci(5000, seed=3), 32, 3
    elif case == "deformed":
        ns, k, deg = nodesets.deformed_sphere(4000, 0.8, seed=6), 32, 3
    elif case == "cyclide":
        ns, k, deg = nodesets.cyclide_lattice(4000), 32, 3
    else:
        ns, k, deg = nodesets.square_regular(24), 21, 3
    got, want = _weights_pair(nf, ns, k, deg)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < Q_REL, err


def test_quad_weights_singular_stencil_reported(nf):
    """A stencil whose nodes are collinear cannot carry the degree-1 polynomial
    moments (§3.1 unisolvency): the call reports NF_ERR_SINGULAR."""
    X = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [3.0, 0.0], [0.5, 1.0]])
    tris = np.array([[0, 1, 4]], dtype=np.int32)
    st = np.array([[0, 1, 2, 3]], dtype=np.int32)  # collinear stencil
    with pytest.raises(nf.NFError) as ei:
        nf.nf_quad_weights(dev(X, torch.float64), dev(tris, torch.int32), dev(st, torch.int32), 1)
    assert ei.value.name == "NF_ERR_SINGULAR"


# ------------------------------------------------------------------ §2.2 nonlocal sum

def _op(nf, X, q, kernel, path):
    return nf.Operator(dev(X, torch.float32), dev(q, torch.float32), kernel, path)


@pytest.mark.parametrize("path", [0, 1, 2, 4, 5])
@pytest.mark.parametrize("n,B", [(3001, 1), (2500, 3), (1100, 7), (5, 2), (1, 1), (2048, 2), (1500, 19), (1100, 35)])
def test_nonlocal_apply_matches_oracle(nf, path, n, B):
    rng = np.random.default_rng(n + B)
    X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    q = rng.uniform(0.5, 1.5, n).astype(np.float32) / n
    u = rng.normal(0.3, 0.4, size=(B, n)).astype(np.float32)
    beta = rng.uniform(10, 40, B).astype(np.float32)
    theta = rng.uniform(0.1, 0.3, B).astype(np.float32)
    kern = (1.0, 0.3, 0.5, 0.6)
    op = _op(nf, X, q, kern, path)
    got = nf.nf_nonlocal_apply(op, dev(u, torch.float32), dev(beta, torch.float32), dev(theta, torch.float32))
    op.check()
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), f32(beta), f32(theta))
    assert rel_l2(got.cpu().numpy(), want) < REL_L2


@pytest.mark.parametrize("s1", [0.02, 0.3, 3.0])
def test_nonlocal_apply_row_order_forms(nf, s1):
    """The matrix-free kernel takes rows in Morton order; a warp whose rows lie within
    s1 / sqrt(log2 e) of their centre expands the squared distance about that centre,
    any other warp uses coordinate differences.  Nodes in six blobs, listed in random
    order, with a narrow, a medium and a wide kernel mix both forms; every row must
    match the oracle."""
    rng = np.random.default_rng(int(s1 * 100))
    n = 4099
    centres = rng.uniform(-5, 5, size=(6, 3))
    X = (centres[rng.integers(0, 6, n)] + rng.normal(0, 0.5, size=(n, 3))).astype(np.float32)
    q = rng.uniform(0.5, 1.5, n).astype(np.float32) / n
    u = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
    kern = (1.0, s1, 0.5, 2 * s1)
    op = _op(nf, X, q, kern, 0).mf_schedule(nf.MF_SYMMETRIC)
    got = nf.nf_nonlocal_apply(op, dev(u, torch.float32), 20.0, 0.2).cpu().numpy()
    op.check()
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)))
    assert rel_l2(got, want) < REL_L2
    assert np.abs(got - want).max() / np.abs(want).max() < REL_L2


@pytest.mark.parametrize("sched", [1, 2, 3])
@pytest.mark.parametrize("ratio,n", [(2.0, 2048), (2 ** 0.5, 1024), (3 ** 0.5, 1025), (1.7, 3073), (2.0, 1023),
                                     (None, 3073), (None, 1025)])
def test_nonlocal_apply_width_ratios_and_blocks(nf, ratio, n, sched):
    """One trajectory, every schedule (symmetric block pairs of 1,024 or 512 nodes; packed
    row blocks x column splits): the forms for s2^2 / s1^2 = 4, 2, 3 (e1 = e2^m by squaring) and a non-integer
    ratio (two exponentials), and a single Gaussian (A2 = 0, one accumulator per sum; ratio
    None), on node counts at and just past the 1024-node block boundaries (one block, a
    ragged second block, exact blocks)."""
    rng = np.random.default_rng(int((ratio or 5.0) * 1000) + n)
    X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    q = rng.uniform(0.5, 1.5, n).astype(np.float32) / n
    u = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
    s1 = 0.15
    kern = (1.0, s1, 0.5, float(np.float32(s1) * np.float32(ratio))) if ratio else (1.3, s1, 0.0, 0.3)
    op = _op(nf, X, q, kern, 0).mf_schedule(sched)
    got = nf.nf_nonlocal_apply(op, dev(u, torch.float32), 20.0, 0.2).cpu().numpy()
    op.check()
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)))
    assert rel_l2(got, want) < REL_L2
    assert np.abs(got - want).max() / np.abs(want).max() < REL_L2


@pytest.mark.parametrize("A1,A2", [(1.0, 1e-35), (1e-30, 1.0), (-0.7, 0.3), (0.0, 0.8), (2.0, -0.5)])
def test_nonlocal_apply_amplitude_extremes(nf, A1, A2):
    """The symmetric kernel with an integer width ratio combines the two Gaussians through
    the per-row ratio -A1 f1 / (A2 f2); amplitude ratios far outside FP32's range (here
    1e35) take the general form instead.  Both sides of that limit, a vanishing ratio, an
    A1 of zero and signs flipped, against the oracle."""
    rng = np.random.default_rng(77)
    n = 3000
    X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    q = rng.uniform(0.5, 1.5, n).astype(np.float32) / n
    u = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
    s1 = 0.15
    kern = (A1, s1, A2, float(np.float32(s1) * np.float32(2.0)))
    op = _op(nf, X, q, kern, 0).mf_schedule(nf.MF_SYMMETRIC)
    got = nf.nf_nonlocal_apply(op, dev(u, torch.float32), 20.0, 0.2).cpu().numpy()
    op.check()
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)))
    assert np.isfinite(got).all()
    assert rel_l2(got, want) < REL_L2


def test_nonlocal_apply_paper_kernel_torus_sampled_full_size(nf):
    """Full precision-workload size (n = 100,000 torus nodes), the launch
    configuration the benchmark times; the oracle evaluates 384 sampled rows."""
    wl = W.precision()
    X = wl.ns.nodes.astype(np.float32)
    rng = np.random.default_rng(11)
    q = (wl.ns.area / wl.n * rng.uniform(0.8, 1.2, wl.n)).astype(np.float32)
    u = wl.u0.astype(np.float32)
    rows = np.sort(rng.choice(wl.n, 384, replace=False))
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(wl.kernel), f32(wl.beta), f32(wl.theta), rows=rows)
    for path in (0, 2, 1, 4):
        op = _op(nf, X, q, wl.kernel, path)
        got = nf.nf_nonlocal_apply(op, dev(u, torch.float32), float(wl.beta[0]), float(wl.theta[0]))
        op.check()
        assert rel_l2(got.cpu().numpy()[:, rows], want) < REL_L2, path
        op.close()
        del op
        torch.cuda.empty_cache()


# ------------------------------------------------------------------ RK4 trajectories

def _rk4_pair(nf, X, q, u0, kernel, beta, theta, dt, nsteps, path, forcing=None, extra=None):
    op = _op(nf, X, q, kernel, path)
    u = dev(u0, torch.float32)
    F = None
    Fo = None
    if forcing is not None:
        lam = nf.nf_mms_sphere_eigs(kernel)
        F = nf.Forcing(1, dev(extra["Y1"], torch.float32), dev(extra["Y2"], torch.float32), forcing["c"],
                       forcing["a0"], lam)
        Fo = oracle.mms_sphere_forcing(f32(kernel), forcing["c"], forcing["a0"])
    nf.nf_rk4_advance(op, u, 0.0, dt, nsteps, dev(beta, torch.float32), dev(theta, torch.float32), forcing=F)
    op.check()
    want = oracle.rk4(f32(X), f32(q), f32(u0), f32(kernel), f32(beta), f32(theta), 0.0, dt, nsteps, forcing=Fo)
    return u.cpu().numpy(), want


@pytest.mark.parametrize("path", [0, 1, 2, 4, 5])
def test_rk4_flat_workload_full(nf, path):
    """The flat unit-square workload end to end: oracle stencils and weights, then
    100 RK4 steps (t = 0..5) on the GPU vs the FP64 oracle."""
    wl = W.flat()
    X2 = wl.ns.coords()
    st = oracle.knn(X2, wl.ns.tris, wl.k)
    q = oracle.quad_weights(X2, wl.ns.tris, st, wl.deg)
    X = wl.ns.nodes.astype(np.float32)
    got, want = _rk4_pair(nf, X, q.astype(np.float32), wl.u0.astype(np.float32), wl.kernel,
                          wl.beta.astype(np.float32), wl.theta.astype(np.float32), wl.dt, wl.nsteps, path)
    assert rel_l2(got, want) < REL_L2


@pytest.mark.parametrize("n,nsteps,C", [(1, 3, 1), (7, 5, 2), (1500, 30, 7), (4000, 12, 5), (8192, 6, 3), (8193, 6, 3)])
def test_rk4_small_sets_checkpoints(nf, n, nsteps, C):
    """Small node sets (1 and 7 nodes in a padded block, up to one past 8,192) on the
    automatic and the packed schedule: trajectory and every checkpoint against the oracle,
    and the two schedules' checkpoints against each other."""
    rng = np.random.default_rng(n + 17)
    X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    q = rng.uniform(0.5, 1.5, n).astype(np.float32) / max(n, 1) * 8.0
    u0 = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
    kern = (1.0, 0.15, 0.5, 0.3)
    dt = 0.05
    want = oracle.rk4(f32(X), f32(q), f32(u0), f32(kern), f32([20.0]), f32([0.2]), 0.0, dt, nsteps)
    res = {}
    for sched in (nf.MF_AUTO, nf.MF_PACKED):
        op = _op(nf, X, q, kern, 0).mf_schedule(sched)
        u = dev(u0, torch.float32)
        ck = torch.zeros((nsteps // C + 1, 1, n), dtype=torch.float32, device="cuda")
        nf.nf_rk4_advance(op, u, 0.0, dt, nsteps, 20.0, 0.2, ckpt=ck, C_every=C)
        op.check()
        res[sched] = (u.cpu().numpy(), ck.cpu().numpy())
        assert rel_l2(res[sched][0], want) < REL_L2
    for c in range(1, nsteps // C + 1):
        wc = oracle.rk4(f32(X), f32(q), f32(u0), f32(kern), f32([20.0]), f32([0.2]), 0.0, dt, c * C)
        assert rel_l2(res[nf.MF_AUTO][1][c], wc) < REL_L2
        assert rel_l2(res[nf.MF_AUTO][1][c], res[nf.MF_PACKED][1][c]) < REL_L2


def test_rk4_sphere_manufactured_forcing(nf):
    wl = W.sphere(3000)
    st = oracle.knn(wl.ns.nodes, wl.ns.tris, wl.k)
    q = oracle.quad_weights(wl.ns.nodes, wl.ns.tris, st, wl.deg, normals=wl.ns.normals)
    X = wl.ns.nodes.astype(np.float32)
    extra = {"Y1": f32(0.5 * X[:, 2]), "Y2": f32(X[:, 0]) * f32(X[:, 1])}
    got, want = _rk4_pair(nf, X, q.astype(np.float32), wl.u0.astype(np.float32), wl.kernel,
                          wl.beta.astype(np.float32), wl.theta.astype(np.float32), wl.dt, 40, 0,
                          forcing=wl.forcing, extra=extra)
    assert rel_l2(got, want) < REL_L2


def test_rk4_sphere_manufactured_forcing_from_operator(nf):
    """The same manufactured problem with the forcing kind that takes Y1, Y2 and the
    eigenvalues from the operator (the caller passes only c and a0)."""
    wl = W.sphere(3000)
    st = oracle.knn(wl.ns.nodes, wl.ns.tris, wl.k)
    q = oracle.quad_weights(wl.ns.nodes, wl.ns.tris, st, wl.deg, normals=wl.ns.normals).astype(np.float32)
    X = wl.ns.nodes.astype(np.float32)
    op = _op(nf, X, q, wl.kernel, 0)
    u = dev(wl.u0.astype(np.float32), torch.float32)
    beta, theta = wl.beta.astype(np.float32), wl.theta.astype(np.float32)
    F = nf.Forcing.sphere(wl.forcing["c"], wl.forcing["a0"])
    nf.nf_rk4_advance(op, u, 0.0, wl.dt, 40, dev(beta, torch.float32), dev(theta, torch.float32), forcing=F)
    op.check()
    Fo = oracle.mms_sphere_forcing(f32(wl.kernel), wl.forcing["c"], wl.forcing["a0"])
    want = oracle.rk4(f32(X), f32(q), f32(wl.u0), f32(wl.kernel), f32(beta), f32(theta), 0.0, wl.dt, 40, forcing=Fo)
    assert rel_l2(u.cpu().numpy(), want) < REL_L2
    ck = torch.zeros((3, 1, X.shape[0]), dtype=torch.float32, device="cuda")
    with pytest.raises(nf.NFError) as ei:
        nf.nf_adjoint(op, ck, 1, 0.0, wl.dt, 2, 20.0, 0.2, torch.zeros((1, X.shape[0]), device="cuda"), forcing=F)
    assert ei.value.name == "NF_ERR_UNSUPPORTED"


def test_stencils_at_given_centres(nf):
    """nf_build_stencils_at: bit-exact against the oracle for arbitrary centres (quantised,
    with exact ties, some outside the nodes' bounding box), and equal to nf_build_stencils
    at the triangle centroids."""
    rng = np.random.default_rng(77)
    for dim in (2, 3):
        n = 3000
        X = np.round(rng.uniform(0, 1, size=(n, dim)) * 32) / 32
        Cq = np.round(rng.uniform(-0.3, 1.3, size=(700, dim)) * 64) / 64
        k = 21
        got = nf.nf_build_stencils_at(dev(X, torch.float64), dev(Cq, torch.float64), k).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.knn_at(X, Cq, k))
        tris = rng.integers(0, n, size=(500, 3)).astype(np.int32)
        cent = ((X[tris[:, 0]] + X[tris[:, 1]]) + X[tris[:, 2]]) / 3.0
        a = nf.nf_build_stencils_at(dev(X, torch.float64), dev(cent, torch.float64), k).cpu().numpy()
        b = nf.nf_build_stencils(dev(X, torch.float64), dev(tris, torch.int32), k).cpu().numpy()
        np.testing.assert_array_equal(a, b)


def test_quad_weights_options_struct(nf):
    """nf_quad_weights_opts gives the same weights as nf_quad_weights; other spline orders
    are refused."""
    wl = W.sphere(2000)
    nodes = dev(wl.ns.nodes, torch.float64)
    tris = dev(wl.ns.tris, torch.int32)
    normals = dev(wl.ns.normals, torch.float64)
    st = nf.nf_build_stencils(nodes, tris, wl.k)
    a = nf.nf_quad_weights(nodes, tris, st, wl.deg, normals=normals)
    b = nf.nf_quad_weights_opts(nodes, tris, st, {"dim": 3, "phs_order": 3, "poly_deg": wl.deg, "curved": 1},
                                normals=normals)
    assert torch.equal(a, b)
    with pytest.raises(nf.NFError) as ei:
        nf.nf_quad_weights_opts(nodes, tris, st, {"dim": 3, "phs_order": 5, "poly_deg": wl.deg, "curved": 1},
                                normals=normals)
    assert ei.value.name == "NF_ERR_UNSUPPORTED"


def test_rk4_batched_trajectories(nf):
    rng = np.random.default_rng(5)
    ns = nodesets.ellipsoid_fibonacci(2000, seed=9)
    q = np.full(ns.n, 3.0 / ns.n, dtype=np.float32)
    u0, beta, theta = nodesets.random_bumps(ns, 6, 17, (1.0, 0.8, 0.6))
    X = ns.nodes.astype(np.float32)
    got, want = _rk4_pair(nf, X, q, u0.astype(np.float32), W.KERNEL, beta.astype(np.float32),
                          theta.astype(np.float32), 0.05, 20, 0)
    assert rel_l2(got, want) < REL_L2


def test_rk4_linear_decay_full_size(nf):
    """Property at the full precision-workload size: with w = 0, RK4 multiplies u by
    (1 - dt + dt^2/2 - dt^3/6 + dt^4/24) per step."""
    wl = W.precision()
    X = wl.ns.nodes.astype(np.float32)
    q = np.full(wl.n, wl.ns.area / wl.n, dtype=np.float32)
    op = _op(nf, X, q, (0.0, 0.1, 0.0, 0.2), 0)
    u = dev(wl.u0, torch.float32)
    u0 = u.clone()
    dt, N = wl.dt, 4
    nf.nf_rk4_advance(op, u, 0.0, dt, N, 50.0, 0.2)
    op.check()
    g = 1 - dt + dt ** 2 / 2 - dt ** 3 / 6 + dt ** 4 / 24
    want = u0.double().cpu().numpy() * g ** N
    assert rel_l2(u.cpu().numpy(), want) < 1e-6


def test_rk4_checkpoints(nf):
    rng = np.random.default_rng(2)
    n = 700
    X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    q = np.full(n, 1.0 / n, dtype=np.float32)
    u0 = rng.normal(0.2, 0.3, size=(2, n)).astype(np.float32)
    op = _op(nf, X, q, (1.0, 0.3, 0.5, 0.6), 0)
    u = dev(u0, torch.float32)
    ck = torch.zeros((4, 2, n), dtype=torch.float32, device="cuda")
    nf.nf_rk4_advance(op, u, 0.0, 0.05, 9, 20.0, 0.2, ckpt=ck, C_every=3)
    op.check()
    ck = ck.cpu().numpy()
    np.testing.assert_array_equal(ck[0], u0)
    np.testing.assert_array_equal(ck[3], u.cpu().numpy())
    for c in (1, 2):
        want = oracle.rk4(f32(X), f32(q), f32(u0), (1.0, 0.3, 0.5, 0.6), 20.0, np.float32(0.2), 0.0, 0.05, 3 * c)
        assert rel_l2(ck[c], want) < REL_L2


def test_mf_schedule_switch_and_auto(nf):
    """The automatic schedule picks the packed kernel for a small node set and the
    symmetric one at n = 20,000 (210 block pairs of 1,024 nodes); switching schedules on a live operator
    (also between captured RK4 steps) keeps the results."""
    for n, want_tile in ((3000, None), (20000, 1024)):
        rng = np.random.default_rng(n)
        X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
        q = np.full(n, 1.0 / n, dtype=np.float32)
        u0 = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
        op = _op(nf, X, q, (1.0, 0.3, 0.5, 0.6), 0)
        shape = op.launch_shape()
        if want_tile is not None:  # symmetric, 1,024- or (autotuned) 512-node blocks
            assert shape["tile_cols"] in (512, 1024) and shape["splits"] == -(-n // 1024) * (1024 // shape["tile_cols"])
        else:
            assert shape["tile_cols"] in (512, 1024) and shape["splits"] <= 64
        res = []
        for sched in (0, 1, 2, 0):
            op.mf_schedule(sched)
            u = dev(u0, torch.float32)
            nf.nf_rk4_advance(op, u, 0.0, 0.05, 3, 20.0, 0.2)
            op.check()
            res.append(u.cpu().numpy())
        want = oracle.rk4(f32(X), f32(q), f32(u0), (1.0, 0.3, 0.5, 0.6), 20.0, float(np.float32(0.2)), 0.0, 0.05, 3)
        for r in res:
            assert rel_l2(r, want) < REL_L2


@pytest.mark.parametrize("B", [2, 3])
def test_symmetric_kernel_several_trajectories(nf, B):
    """Up to three trajectories share one symmetric launch (a grid z per trajectory); their
    sums and RK4 steps match the oracle, with and without block-pair culling."""
    rng = np.random.default_rng(B)
    ns = nodesets.torus_lattice(16000, seed=B)
    X = ns.nodes.astype(np.float32)
    n = ns.n
    q = np.full(n, ns.area / n, dtype=np.float32)
    u = rng.normal(0.3, 0.4, size=(B, n)).astype(np.float32)
    beta = rng.uniform(10, 40, B).astype(np.float32)
    theta = rng.uniform(0.1, 0.3, B).astype(np.float32)
    kern = (1.0, 0.02, 0.5, 0.04)  # narrow enough that far block pairs cull on this torus
    rows = np.sort(rng.choice(n, 300, replace=False))
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), f32(beta), f32(theta), rows=rows)
    op = _op(nf, X, q, kern, 0).mf_schedule(nf.MF_SYMMETRIC)
    got = nf.nf_nonlocal_apply(op, dev(u, torch.float32), dev(beta, torch.float32), dev(theta, torch.float32))
    op.check()
    got = got.cpu().numpy()
    assert rel_l2(got[:, rows], want) < REL_L2
    live, total = op.mf_cull(True)
    assert live < total
    got_c = nf.nf_nonlocal_apply(op, dev(u, torch.float32), dev(beta, torch.float32), dev(theta, torch.float32))
    np.testing.assert_array_equal(got_c.cpu().numpy(), got)
    ua, ub = dev(u, torch.float32), dev(u, torch.float32)
    nf.nf_rk4_advance(op, ua, 0.0, 0.02, 2, dev(beta, torch.float32), dev(theta, torch.float32))
    op.mf_cull(False)
    nf.nf_rk4_advance(op, ub, 0.0, 0.02, 2, dev(beta, torch.float32), dev(theta, torch.float32))
    op.check()
    np.testing.assert_array_equal(ua.cpu().numpy(), ub.cpu().numpy())


@pytest.mark.parametrize("n,B", [(1000, 8), (3000, 64), (2100, 65), (1500, 130), (6000, 256)])
def test_dense_fp32_gemm_several_trajectories(nf, n, B):
    """Dense FP32 operators with eight or more trajectories run the SIMT FP32 GEMM (tiles
    of 64 or 128 trajectories, split K on small node sets, ragged trajectory tiles)."""
    rng = np.random.default_rng(n + 7 * B)
    X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    q = rng.uniform(0.5, 1.5, n).astype(np.float32) / n
    u = rng.normal(0.3, 0.4, size=(B, n)).astype(np.float32)
    beta = rng.uniform(10, 40, B).astype(np.float32)
    theta = rng.uniform(0.1, 0.3, B).astype(np.float32)
    kern = (1.0, 0.3, 0.5, 0.6)
    op = nf.Operator(dev(X, torch.float32), dev(q, torch.float32), kern, nf.DENSE_FP32)
    got = nf.nf_nonlocal_apply(op, dev(u, torch.float32), dev(beta, torch.float32), dev(theta, torch.float32))
    op.check()
    sel = np.unique(np.concatenate([[0, B - 1], rng.choice(B, min(B, 6), replace=False)]))
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u[sel]), f32(kern), f32(beta[sel]), f32(theta[sel]))
    assert rel_l2(got.cpu().numpy()[sel], want) < REL_L2
    op.close()


def test_dense_fp32_gemm_rk4(nf):
    """RK4 through the GEMM path (24 trajectories) against the oracle."""
    ns = nodesets.ellipsoid_fibonacci(2500, seed=4)
    q = np.full(ns.n, 3.0 / ns.n, dtype=np.float32)
    u0, beta, theta = nodesets.random_bumps(ns, 24, 5, (1.0, 0.8, 0.6))
    X = ns.nodes.astype(np.float32)
    got, want = _rk4_pair(nf, X, q, u0.astype(np.float32), W.KERNEL, beta.astype(np.float32),
                          theta.astype(np.float32), 0.05, 10, nf.DENSE_FP32)
    assert rel_l2(got, want) < REL_L2
