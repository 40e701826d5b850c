"""GPU parity for the doubly periodic distance (§4, Eq. (dist)) and the flat manufactured
forcing of the convergence studies (§4.3 on the square, §4.4 on the torus in (phi, theta)
coordinates), against the FP64 oracle (pinned in tests/test_oracle_periodic.py).

Bar: 1e-5 relative L2 per trajectory (FP32 sums), as for the Euclidean paths."""
import math

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
L = float(np.float32(2.0 * math.pi))


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_13379_gb300 as nf
    nf.lib()
    return nf


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def rel_l2(got, want):
    got, want = np.atleast_2d(got), np.atleast_2d(want)
    return max(np.linalg.norm(g - w) / np.linalg.norm(w) for g, w in zip(got, want))


def _square(n, seed, z_noise=0.0):
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.uniform(0, L, (n, 2)), z_noise * rng.normal(size=(n, 1))], 1).astype(np.float32)
    q = (rng.uniform(0.5, 1.5, n) * L * L / n).astype(np.float32)
    return rng, X, q


# a kernel wide enough that every node sees wrapped neighbours, one width ratio per form
KERNELS = {
    "m4": (1.0, 0.6, 0.5, 1.2, L),            # s2 = 2 s1: e1 = e2^4
    "general": (1.3, 0.5, 0.45, 1.1, L),     # two exponentials per pair
    "paper": (1.0 / (2 * math.pi / 40 ** 2), math.sqrt(2) / 40, 0.0, math.sqrt(2) / 40 * 1.7, L),
    "mixed": (1.0, 0.2, 0.45, 0.25, L),      # narrow enough that far images flush to zero
}


@pytest.mark.parametrize("kname", sorted(KERNELS))
@pytest.mark.parametrize("path", [0, 1, 2, 4, 5])
@pytest.mark.parametrize("n,B", [(3001, 1), (2500, 3), (1100, 7), (5, 2)])
def test_periodic_nonlocal_apply(nf, kname, path, n, B):
    """Every path (symmetric matrix-free for one trajectory; scalar and packed pair kernels
    for several; dense FP32, bf16 hi+lo and symmetric blocks) on random nodes of the square,
    several 1024-node blocks plus a ragged tail."""
    kern = KERNELS[kname]
    rng, X, q = _square(n, n + B + path)
    u = rng.normal(0.3, 0.4, size=(B, n)).astype(np.float32)
    beta = rng.uniform(10, 40, B).astype(np.float32)
    theta = rng.uniform(0.1, 0.3, B).astype(np.float32)
    op = nf.Operator(dev(X), dev(q), kern, path)
    got = nf.nf_nonlocal_apply(op, dev(u), dev(beta), dev(theta)).cpu().numpy()
    op.check()
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), f32(beta), f32(theta))
    assert rel_l2(got, want) < REL_L2


@pytest.mark.parametrize("kern", [(1.0, 0.2, 0.45, 0.25, L), (1.0, 0.05, 0.5, 0.1, L), (1.0, 0.3, 0.5, 0.6, L)])
def test_periodic_forms_blobs(nf, kern):
    """Nodes in tight blobs centred on the square's edges and corners (each blob wraps
    around), listed in random order: the symmetric kernel's passes mix the expanded form,
    centred differences with columns at their nearest image of the pass centre, and (wide
    kernels) per-pair nearest images; every row must match the oracle."""
    rng = np.random.default_rng(int(kern[1] * 1000))
    n = 5000
    centres = np.array([[0.0, 0.0], [L / 2, 0.0], [0.0, L / 3], [L - 0.1, L / 2], [2.0, 2.5]])
    xy = centres[rng.integers(0, len(centres), n)] + rng.normal(0, 0.3, size=(n, 2))
    X = np.concatenate([np.mod(xy, L), np.zeros((n, 1))], 1).astype(np.float32)
    q = (rng.uniform(0.5, 1.5, n) / n).astype(np.float32)
    u = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
    op = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(nf.MF_SYMMETRIC)
    got = nf.nf_nonlocal_apply(op, dev(u), 20.0, 0.2).cpu().numpy()
    op.check()
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)))
    assert rel_l2(got, want) < REL_L2
    assert np.abs(got - want).max() / np.abs(want).max() < REL_L2


@pytest.mark.parametrize("sched", [4, 3])
@pytest.mark.parametrize("kname", sorted(KERNELS))
@pytest.mark.parametrize("n", [3001, 1025])
def test_periodic_symmetric_schedule(nf, kname, n, sched):
    """The symmetric kernel's periodic forms on small node sets (the automatic schedule
    would take the packed kernel there), with 1,024- and 512-node blocks."""
    kern = KERNELS[kname]
    rng, X, q = _square(n, 40 + n)
    u = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
    op = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(sched)
    got = nf.nf_nonlocal_apply(op, dev(u), 20.0, 0.2).cpu().numpy()
    op.check()
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)))
    assert rel_l2(got, want) < REL_L2


def test_periodic_z_is_not_wrapped(nf):
    """Only x and y differences wrap: nodes slightly off the plane keep their z distance."""
    kern = KERNELS["m4"]
    rng, X, q = _square(2300, 5, z_noise=0.4)
    u = rng.normal(0.3, 0.4, size=(1, 2300)).astype(np.float32)
    for path in (0, 1):
        op = nf.Operator(dev(X), dev(q), kern, path)
        got = nf.nf_nonlocal_apply(op, dev(u), 20.0, 0.2).cpu().numpy()
        op.check()
        want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)))
        assert rel_l2(got, want) < REL_L2


def test_periodic_nodes_outside_the_cell(nf):
    """Nodes given in any cell (coordinates shifted by multiples of L) give the same sums."""
    kern = KERNELS["general"]
    rng, X, q = _square(1500, 8)
    u = rng.normal(0.3, 0.4, size=(1, 1500)).astype(np.float32)
    Y = X.copy()
    Y[:, :2] += (L * rng.integers(-3, 4, size=(1500, 2))).astype(np.float32)
    a = nf.Operator(dev(X), dev(q), kern, 0)
    b = nf.Operator(dev(Y), dev(q), kern, 0)
    ga = nf.nf_nonlocal_apply(a, dev(u), 20.0, 0.2).cpu().numpy()
    gb = nf.nf_nonlocal_apply(b, dev(u), 20.0, 0.2).cpu().numpy()
    assert rel_l2(gb, ga) < 1e-5


def test_periodic_noalloc(nf):
    kern = KERNELS["m4"]
    rng, X, q = _square(4000, 9)
    u = rng.normal(0.3, 0.4, size=4000).astype(np.float32)
    out = torch.empty(4000, dtype=torch.float32, device="cuda")
    got = nf.nf_nonlocal_apply_noalloc(dev(X), dev(q), dev(u), kern, 20.0, 0.2, out).cpu().numpy()
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)))
    assert rel_l2(got, want) < REL_L2


def test_periodic_grouped_tensor_core(nf):
    """Grouped bf16 hi+lo operators (tcgen05 path) over periodic members."""
    kern = KERNELS["m4"]
    data, ops = [], []
    for n, B, seed in ((1500, 12, 1), (900, 5, 2)):
        rng, X, q = _square(n, seed)
        u = rng.normal(0.3, 0.4, size=(B, n)).astype(np.float32)
        be = rng.uniform(10, 40, B).astype(np.float32)
        th = rng.uniform(0.1, 0.3, B).astype(np.float32)
        data.append((X, q, u, be, th))
        ops.append(nf.Operator(dev(X), dev(q), kern, nf.DENSE_BF16X2))
    grp = nf.GroupedOperator(ops, [d[2].shape[0] for d in data])
    u = torch.cat([dev(d[2]).reshape(-1) for d in data])
    I = nf.nf_nonlocal_apply(grp, u, torch.cat([dev(d[3]) for d in data]), torch.cat([dev(d[4]) for d in data]))
    grp.check()
    for (X, q, u0, be, th), got in zip(data, grp.split(I)):
        want = oracle.nonlocal_sum(f32(X), f32(q), f32(u0), f32(kern), f32(be), f32(th))
        assert rel_l2(got.cpu().numpy(), want) < REL_L2


@pytest.mark.parametrize("kname", ["m4", "general"])
def test_periodic_adjoint(nf, kname):
    kern = KERNELS[kname]
    n, B, nsteps, C, dt = 1700, 2, 8, 4, 0.02
    rng, X, q = _square(n, 21)
    u0 = rng.normal(0.3, 0.3, size=(B, n)).astype(np.float32)
    beta = np.array([20.0, 12.0], dtype=np.float32)
    theta = np.array([0.2, 0.25], dtype=np.float32)
    target = (0.9 * u0 + 0.05 * rng.normal(size=u0.shape)).astype(np.float32)
    op = nf.Operator(dev(X), dev(q), kern, 0)
    u = dev(u0)
    ck = torch.zeros((nsteps // C + 1, B, n), dtype=torch.float32, device="cuda")
    nf.nf_rk4_advance(op, u, 0.0, dt, nsteps, dev(beta), dev(theta), ckpt=ck, C_every=C)
    gu, gk = nf.nf_adjoint(op, ck, C, 0.0, dt, nsteps, dev(beta), dev(theta), 2.0 * (u - dev(target)))
    op.check()
    uN = oracle.rk4(f32(X), f32(q), f32(u0), f32(kern), f32(beta), f32(theta), 0.0, dt, nsteps)
    gu_o, gk_o = oracle.adjoint(f32(X), f32(q), f32(u0), f32(kern), f32(beta), f32(theta), 0.0, dt, nsteps,
                                2.0 * (uN - f32(target)))
    gu, gk = gu.cpu().numpy(), gk.cpu().numpy()
    for b in range(B):
        assert np.linalg.norm(gu[b] - gu_o[b]) / np.linalg.norm(gu_o[b]) < 1e-5
        np.testing.assert_allclose(gk[b], gk_o[b], rtol=1e-4, atol=1e-6 * np.abs(gk_o[b]).max())


# ------------------------------------------------------------------ manufactured forcing

C0, RAD, SIG, BETA, THETA = 0.1, 0.2, 1.1, 20.0, 0.3


def _periodic_grid(m):
    t = (np.arange(m) + 0.5) * (L / m)
    X, Y = np.meshgrid(t, t, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.zeros(m * m)], 1).astype(np.float32)


@pytest.mark.parametrize("kname,scale", [("m4", 1.0), ("general", 0.7), ("paper", 1.0)])
@pytest.mark.parametrize("path", [0, 2])
def test_rk4_flat_manufactured_forcing(nf, kname, scale, path):
    """RK4 with the moving-Gaussian forcing: the GPU evaluates the convolution term in
    closed form (erf), the oracle by panel quadrature; the trajectories agree."""
    kern = KERNELS[kname]
    m = 48
    X = _periodic_grid(m)
    q = np.full(m * m, (L / m) ** 2, dtype=np.float32)
    u0 = oracle.mms_flat_solution(f32(X), 0.0, f32(kern[:4]), L, BETA, THETA, C0, RAD, SIG)[None, :]
    u0 = u0.astype(np.float32)
    op = nf.Operator(dev(X), dev(q), kern, path)
    u = dev(u0)
    dt, nsteps = 0.01, 10
    nf.nf_rk4_advance(op, u, 0.0, dt, nsteps, BETA, THETA, forcing=nf.Forcing.flat(C0, RAD, SIG, scale))
    op.check()
    want = oracle.rk4(f32(X), f32(q), f32(u0), f32(kern), BETA, float(np.float32(THETA)), 0.0, dt, nsteps,
                      forcing=oracle.mms_flat_forcing(C0, RAD, SIG, scale))
    assert rel_l2(u.cpu().numpy(), want) < REL_L2


def test_flat_forcing_needs_a_periodic_kernel(nf):
    X = _periodic_grid(8)
    op = nf.Operator(dev(X), dev(np.ones(64)), (1.0, 0.5, 0.5, 1.0), 0)
    with pytest.raises(nf.NFError):
        nf.nf_rk4_advance(op, dev(np.zeros((1, 64))), 0.0, 0.01, 1, 20.0, 0.3, forcing=nf.Forcing.flat())
    opp = nf.Operator(dev(X), dev(np.ones(64)), (1.0, 0.5, 0.5, 1.0, L), 0)
    with pytest.raises(nf.NFError):  # z = G + c leaves (0, 1)
        nf.nf_rk4_advance(opp, dev(np.zeros((1, 64))), 0.0, 0.01, 1, 20.0, 0.3,
                          forcing=nf.Forcing.flat(c=0.1, sigma=0.2))


def test_periodic_models(nf):
    """The §5 models on a periodic operator (depression, smooth step, AB5)."""
    kern = KERNELS["m4"]
    rng, X, q = _square(2000, 31)
    u0 = rng.uniform(0.0, 0.6, size=(1, 2000)).astype(np.float32)
    s0 = rng.uniform(0.5, 1.0, size=(1, 2000)).astype(np.float32)
    op = nf.Operator(dev(X), dev(q), kern, 0)
    u, s = dev(u0), dev(s0)
    nf.nf_field_advance(op, u, 0.02, 20, dev(np.array([20.0])), dev(np.array([0.2])), s=s, rate=1, tau=3.0,
                        beta_d=0.6, integrator="ab5")
    op.check()
    wu, ws = oracle.field_advance(f32(X), f32(q), f32(u0), f32(kern), 20.0, float(np.float32(0.2)),
                                  float(np.float32(0.02)), 20, s0=f32(s0), kind=1, rate_kind=1,
                                  a=float(np.float32(0.06)), b=float(np.float32(0.54)), tau=3.0,
                                  beta_d=float(np.float32(0.6)), integrator="ab5")
    assert rel_l2(u.cpu().numpy(), wu) < REL_L2
    assert rel_l2(s.cpu().numpy(), ws) < REL_L2


@pytest.mark.parametrize("path", [0, 1, 2, 4, 5])
def test_spatial_error_map_unit_square(nf, path):
    """§4.2, Eq. (flat_spatial_error) on the unit square (period 1): the oracle's weights on
    point-repulsion nodes (n = 2000, r^3, k = 21, deg 3), a 64 x 64 grid of centres x0
    appended as nodes of weight 0, f = 1, so that row x0 of the sum is Q_n f_x0 for the
    periodic Gaussian of sigma = 1/10.  Every path against the oracle on the grid rows, and
    the mean of E(x0) = 1 - Q_n f_x0 / Q f_x0 near zero, as the exactness for constants
    requires."""
    import nodesets
    from scipy.special import erf
    ns = nodesets.square_repulsion(2000)
    x2 = ns.coords()
    q = oracle.quad_weights(x2, ns.tris, oracle.knn(x2, ns.tris, 21), 3)
    m = 64
    t = (np.arange(m) + 0.5) / m
    c = np.stack(np.meshgrid(t, t, indexing="ij"), -1).reshape(-1, 2)
    X = np.concatenate([ns.nodes, np.concatenate([c, np.zeros((m * m, 1))], 1)]).astype(np.float32)
    qa = np.concatenate([q, np.zeros(m * m)]).astype(np.float32)
    s = math.sqrt(2.0) * 0.1
    kern = (1.0, s, 0.0, s, 1.0)
    u = np.full((1, X.shape[0]), 50.0, dtype=np.float32)
    op = nf.Operator(dev(X), dev(qa), kern, path)
    got = nf.nf_nonlocal_apply(op, dev(u), 1.0, 0.0).cpu().numpy()[0, ns.n:].astype(np.float64)
    op.check()
    rows = np.arange(ns.n, X.shape[0])
    want = oracle.nonlocal_sum(f32(X), f32(qa), f32(u), f32(kern[:4]), 1.0, 0.0, rows=rows, period=1.0)[0]
    assert rel_l2(got, want) < REL_L2
    Qf = (s * math.sqrt(math.pi) * erf(0.5 / s)) ** 2
    rms = math.sqrt((((Qf - want) / Qf) ** 2).mean())
    assert abs(((Qf - got) / Qf).mean()) < 0.1 * rms
