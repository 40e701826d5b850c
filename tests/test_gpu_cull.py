"""Block-pair culling of the symmetric matrix-free kernel: block pairs whose every node pair
contributes exactly zero in FP32 are skipped.  The culled sums must be bit-identical to the
full symmetric sums (same nonzero terms, same order) and match the FP64 oracle within the
1e-5 relative L2 bar."""
import math

import numpy as np
import pytest
import torch

import nodesets
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


def _torus(n, seed):
    ns = nodesets.torus_lattice(n, seed=seed)
    return ns.nodes.astype(np.float32), np.full(ns.n, ns.area / ns.n, dtype=np.float32), ns


def _square(n, seed):
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.uniform(0, L, (n, 2)), np.zeros((n, 1))], 1).astype(np.float32)
    return X, np.full(n, L * L / n, dtype=np.float32)


CASES = {
    # narrow Mexican hat on the torus (R = 1, r = 0.4): far blocks cull
    "torus_narrow": ("torus", (1.0, 0.02, 0.5, 0.04)),
    # the §4.3 kernel Gauss(1/40) on the periodic square: almost every block pair culls
    "square_paper": ("square", (1.0 / (2 * math.pi / 40 ** 2), math.sqrt(2) / 40, 0.0, 0.1, L)),
    # general width ratio, periodic, moderate width
    "square_general": ("square", (1.0, 0.08, 0.4, 0.13, L)),
    # wide kernel: nothing culls
    "torus_wide": ("torus", (1.0, 0.6, 0.5, 1.2)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_cull_bit_identical_and_oracle(nf, case):
    geom, kern = CASES[case]
    n = 20000
    if geom == "torus":
        X, q, ns = _torus(n, 5)
        u = (0.8 * nodesets.spiral_bumps_u0(ns))[None, :].astype(np.float32)
    else:
        X, q = _square(n, 6)
        rng = np.random.default_rng(7)
        u = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
    full = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(nf.MF_SYMMETRIC)
    cull = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(nf.MF_SYMMETRIC)
    live, total = cull.mf_cull(True)
    assert 0 < live <= total
    if case == "torus_wide":
        assert live == total
    else:
        assert live < total, (live, total)
    a = nf.nf_nonlocal_apply(full, dev(u), 20.0, 0.2).cpu().numpy()
    b = nf.nf_nonlocal_apply(cull, dev(u), 20.0, 0.2).cpu().numpy()
    full.check()
    cull.check()
    np.testing.assert_array_equal(a, b)
    rows = np.sort(np.random.default_rng(8).choice(n, 400, replace=False))
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)), rows=rows)
    assert rel_l2(b[:, rows], want) < REL_L2
    # RK4 steps through the captured graph, then culling switched off again
    ua, ub = dev(u), dev(u)
    nf.nf_rk4_advance(full, ua, 0.0, 0.02, 3, 20.0, 0.2)
    nf.nf_rk4_advance(cull, ub, 0.0, 0.02, 3, 20.0, 0.2)
    np.testing.assert_array_equal(ua.cpu().numpy(), ub.cpu().numpy())
    cull.mf_cull(False)
    c = nf.nf_nonlocal_apply(cull, dev(u), 20.0, 0.2).cpu().numpy()
    np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("case", ["square_paper", "torus_narrow"])
def test_cull_512_blocks(nf, case):
    """Culling over 512-node blocks: bit-identical to the unculled 512-node sum."""
    geom, kern = CASES[case]
    n = 20000
    if geom == "torus":
        X, q, ns = _torus(n, 5)
    else:
        X, q = _square(n, 6)
    u = np.random.default_rng(9).normal(0.3, 0.4, size=(1, len(q))).astype(np.float32)
    full = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(nf.MF_SYMMETRIC_512)
    cull = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(nf.MF_SYMMETRIC_512)
    live, total = cull.mf_cull(True)
    assert live < total and total == (-(-len(q) // 1024) * 2) * ((-(-len(q) // 1024) * 2) + 1) // 2
    a = nf.nf_nonlocal_apply(full, dev(u), 20.0, 0.2).cpu().numpy()
    b = nf.nf_nonlocal_apply(cull, dev(u), 20.0, 0.2).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    rows = np.sort(np.random.default_rng(8).choice(len(q), 300, replace=False))
    want = oracle.nonlocal_sum(f32(X), f32(q), f32(u), f32(kern), 20.0, float(np.float32(0.2)), rows=rows)
    assert rel_l2(b[:, rows], want) < REL_L2


def test_cull_separated_clusters(nf):
    """Two clusters far apart: every cross pair culls and each cluster sums only itself."""
    rng = np.random.default_rng(3)
    n = 16000
    X = np.concatenate([rng.normal(0, 0.2, (n // 2, 3)), rng.normal(0, 0.2, (n // 2, 3)) + 50.0]).astype(np.float32)
    q = np.full(n, 1.0 / n, dtype=np.float32)
    u = rng.normal(0.3, 0.4, size=(1, n)).astype(np.float32)
    kern = (1.0, 0.1, 0.5, 0.2)
    full = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(nf.MF_SYMMETRIC)
    cull = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(nf.MF_SYMMETRIC)
    live, total = cull.mf_cull(True)
    assert live < total
    a = nf.nf_nonlocal_apply(full, dev(u), 20.0, 0.2).cpu().numpy()
    b = nf.nf_nonlocal_apply(cull, dev(u), 20.0, 0.2).cpu().numpy()
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("kern", [(1.0, 0.02, 0.5, 0.04), (3.0, 0.02, 0.0, 0.05)])
def test_cull_adjoint_bit_identical(nf, kern):
    """The adjoint pass culls with its own live pairs (both Gaussians count: the A2 and s2
    parameter sums need e2 even when A2 = 0): gradients bit-identical to the unculled ones."""
    n, B, nsteps, C, dt = 20000, 1, 4, 2, 0.02
    X, q, ns = _torus(n, 11)
    u0 = (0.8 * nodesets.spiral_bumps_u0(ns))[None, :].astype(np.float32)
    target = (0.9 * u0).astype(np.float32)
    res = []
    for cull in (False, True):
        op = nf.Operator(dev(X), dev(q), kern, 0).mf_schedule(nf.MF_SYMMETRIC_1024)
        if cull:
            live, total = op.mf_cull(True)
            assert live < total
        u = dev(u0)
        ck = torch.zeros((nsteps // C + 1, B, n), dtype=torch.float32, device="cuda")
        nf.nf_rk4_advance(op, u, 0.0, dt, nsteps, 20.0, 0.2, ckpt=ck, C_every=C)
        gu, gk = nf.nf_adjoint(op, ck, C, 0.0, dt, nsteps, 20.0, 0.2, 2.0 * (u - dev(target)))
        op.check()
        res.append((u.cpu().numpy(), gu.cpu().numpy(), gk.cpu().numpy()))
    for a, b in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, b)
    assert np.abs(res[1][2]).max() > 0
