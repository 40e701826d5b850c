"""Batched tensor-core path (grouped tcgen05 GEMM, bf16 x 3 split, FP32 accumulate)
against the FP64 oracle.  Groups cover ragged row tiles (n not a multiple of 128),
ragged K (n not a multiple of 32) and trajectory counts that are not multiples of 16.

Tolerance.  hi + lo bf16 pairs carry 16 significant bits, so W diag(q) / s_i and
F = f(U) each differ from their FP32 values by at most 2^-17 relative per entry, and
the dropped lo x lo product is at most 2^-18 relative: a per-term bound of
2^-17 + 2^-17 + 2^-18 ~= 1.9e-5.  Small node sets (few significant terms per sum)
are held to 2e-5 relative L2; the batched workload's own sizes are held to the 1e-5
bar of the FP32 paths (more terms per sum, errors average out)."""
import numpy as np
import pytest
import torch

import nodesets
import oracle
from nodesets import workloads as W

pytestmark = pytest.mark.gpu

REL_L2 = 2e-5


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


def _members(nf, specs, kern):
    data = []
    for n, B, seed in specs:
        ns = nodesets.ellipsoid_fibonacci(n, seed=seed)
        X = ns.nodes.astype(np.float32)
        q = np.full(n, 3.0 / n, dtype=np.float32)
        u0, beta, theta = nodesets.random_bumps(ns, B, seed + 7, (1.0, 0.8, 0.6))
        data.append((ns, X, q, u0.astype(np.float32), beta.astype(np.float32), theta.astype(np.float32)))
    ops = [nf.Operator(dev(X), dev(q), kern, nf.DENSE_BF16X2) for (_, X, q, _, _, _) in data]
    return data, ops


SPECS = [
    [(1000, 20, 1), (1500, 7, 2)],
    [(2100, 64, 3), (531, 16, 4), (1283, 3, 5), (777, 33, 6)],
    [(3000, 256, 8)],
]


@pytest.mark.parametrize("specs", SPECS)
def test_grouped_nonlocal_apply(nf, specs):
    kern = (1.0, 0.1, 0.5, 0.2)
    data, ops = _members(nf, specs, kern)
    grp = nf.GroupedOperator(ops, [s[1] for s in specs])
    u = torch.cat([dev(d[3]).reshape(-1) for d in data])
    beta = torch.cat([dev(d[4]) for d in data])
    theta = torch.cat([dev(d[5]) for d in data])
    I = nf.nf_nonlocal_apply(grp, u, beta, theta)
    grp.check()
    for (ns, X, q, u0, be, th), got in zip(data, grp.split(I)):
        want = oracle.nonlocal_sum(f32(X), f32(q), f32(u0), f32(kern), f32(be), f32(th))
        g = got.cpu().numpy()
        for b in range(want.shape[0]):
            assert np.linalg.norm(g[b] - want[b]) / np.linalg.norm(want[b]) < REL_L2, b


@pytest.mark.parametrize("specs", SPECS[:2])
def test_grouped_rk4(nf, specs):
    kern = (1.0, 0.1, 0.5, 0.2)
    data, ops = _members(nf, specs, kern)
    grp = nf.GroupedOperator(ops, [s[1] for s in specs])
    u = torch.cat([dev(d[3]).reshape(-1) for d in data])
    beta = torch.cat([dev(d[4]) for d in data])
    theta = torch.cat([dev(d[5]) for d in data])
    nsteps, dt = 10, 0.05
    nf.nf_rk4_advance(grp, u, 0.0, dt, nsteps, beta, theta)
    grp.check()
    for (ns, X, q, u0, be, th), got in zip(data, grp.split(u)):
        want = oracle.rk4(f32(X), f32(q), f32(u0), f32(kern), f32(be), f32(th), 0.0, dt, nsteps)
        g = got.cpu().numpy()
        for b in range(want.shape[0]):
            assert np.linalg.norm(g[b] - want[b]) / np.linalg.norm(want[b]) < REL_L2, b


def test_grouped_full_batched_workload_sampled(nf):
    """The batched workload at full size (sphere 40,000 x 256 trajectories, ellipsoids
    8,000 / 15,000 / 30,000 x 64), launched as the benchmark launches it; the oracle
    evaluates 48 sampled rows of every trajectory."""
    wls = W.batched()
    kern = W.KERNEL
    ops, data = [], []
    for wl in wls:
        X = wl.ns.nodes.astype(np.float32)
        q = np.full(wl.n, (wl.ns.area or 4 * np.pi * 0.8) / wl.n, dtype=np.float32)
        ops.append(nf.Operator(dev(X), dev(q), kern, nf.DENSE_BF16X2))
        data.append((X, q, wl.u0.astype(np.float32), wl.beta.astype(np.float32), wl.theta.astype(np.float32)))
    grp = nf.GroupedOperator(ops, [wl.B for wl in wls])
    u = torch.cat([dev(d[2]).reshape(-1) for d in data])
    beta = torch.cat([dev(d[3]) for d in data])
    theta = torch.cat([dev(d[4]) for d in data])
    I = nf.nf_nonlocal_apply(grp, u, beta, theta)
    grp.check()
    rng = np.random.default_rng(5)
    worst = 0.0
    for (X, q, u0, be, th), got in zip(data, grp.split(I)):
        rows = np.sort(rng.choice(X.shape[0], 48, replace=False))
        want = oracle.nonlocal_sum(f32(X), f32(q), f32(u0), f32(kern), f32(be), f32(th), rows=rows)
        g = got.cpu().numpy()[:, rows]
        err = np.linalg.norm(g - want, axis=1) / np.linalg.norm(want, axis=1)
        worst = max(worst, float(err.max()))
    print(f"batched workload: worst per-trajectory relative L2 error {worst:.3e}")
    assert worst < 1e-5


def test_group_rejects_non_bf16_members(nf):
    X = np.random.default_rng(0).uniform(size=(64, 3)).astype(np.float32)
    op = nf.Operator(dev(X), dev(np.full(64, 1 / 64)), (1.0, 0.3, 0.5, 0.6), nf.MATRIX_FREE)
    with pytest.raises(nf.NFError) as ei:
        nf.GroupedOperator([op], [4])
    assert ei.value.name == "NF_ERR_ARG"


@pytest.mark.parametrize("specs", [
    [(1200, 40, 11), (900, 17, 12), (2000, 64, 13), (700, 5, 14), (1500, 130, 15), (1100, 33, 16)],  # six node sets
    [(1800, 300, 21), (1000, 20, 22)],   # 300 trajectories: two sub-groups of one node set
])
def test_grouped_more_sets_and_trajectories(nf, specs):
    """Grouped operators beyond four node sets and beyond 256 trajectories per set, after the
    autotuner has picked the launch configuration: nonlocal sums and 5 RK4 steps against the
    oracle on sampled trajectories of every set."""
    kern = (1.0, 0.1, 0.5, 0.2)
    data, ops = _members(nf, specs, kern)
    grp = nf.GroupedOperator(ops, [s[1] for s in specs])
    t = grp.tuning()
    assert t["ring_depth"] in (2, 3) and t["traj_split"] in (1, 2) and t["lpt_coef"] in (4.0, 8.0, 12.0)
    assert len(specs) <= t["subgroups"] <= 8 and t["ms_per_launch"] > 0
    u = torch.cat([dev(d[3]).reshape(-1) for d in data])
    beta = torch.cat([dev(d[4]) for d in data])
    theta = torch.cat([dev(d[5]) for d in data])
    I = nf.nf_nonlocal_apply(grp, u, beta, theta)
    nsteps, dt = 5, 0.05
    nf.nf_rk4_advance(grp, u, 0.0, dt, nsteps, beta, theta)
    grp.check()
    rng = np.random.default_rng(len(specs))
    for (ns, X, q, u0, be, th), gI, gu in zip(data, grp.split(I), grp.split(u)):
        B = u0.shape[0]
        sel = np.unique(np.concatenate([[0, B - 1], rng.choice(B, min(B, 3), replace=False)]))
        wI = oracle.nonlocal_sum(f32(X), f32(q), f32(u0[sel]), f32(kern), f32(be[sel]), f32(th[sel]))
        wu = oracle.rk4(f32(X), f32(q), f32(u0[sel]), f32(kern), f32(be[sel]), f32(th[sel]), 0.0, dt, nsteps)
        for got, want in ((gI.cpu().numpy()[sel], wI), (gu.cpu().numpy()[sel], wu)):
            err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
            assert err.max() < REL_L2, err.max()
    grp.close()
    for op in ops:
        op.close()


def test_group_limits(nf):
    """Nine node sets, or trajectories needing more than eight sub-groups of 256, are refused."""
    X = np.random.default_rng(1).uniform(size=(256, 3)).astype(np.float32)
    op = nf.Operator(dev(X), dev(np.full(256, 1 / 256)), (1.0, 0.3, 0.5, 0.6), nf.DENSE_BF16X2)
    with pytest.raises(nf.NFError) as ei:
        nf.GroupedOperator([op] * 9, [4] * 9)
    assert ei.value.name == "NF_ERR_ARG"
    with pytest.raises(nf.NFError) as ei:
        nf.GroupedOperator([op, op], [1800, 300])   # 8 + 2 sub-groups
    assert ei.value.name == "NF_ERR_UNSUPPORTED"
    op.close()


def test_grouped_every_configuration_matches(nf):
    """Every launch configuration the autotuner chooses from (ring depth 2 or 3, a member of
    128+ trajectories whole or in two, LPT weights 4 / 8 / 12) gives sums within the oracle's
    bar, and the same sums: ring depth and schedule only reorder work, the split only the
    tile a column belongs to."""
    specs = [(2100, 160, 31), (1300, 24, 32), (900, 64, 33)]
    kern = (1.0, 0.1, 0.5, 0.2)
    data, ops = _members(nf, specs, kern)
    grp = nf.GroupedOperator(ops, [s[1] for s in specs])
    u = torch.cat([dev(d[3]).reshape(-1) for d in data])
    beta = torch.cat([dev(d[4]) for d in data])
    theta = torch.cat([dev(d[5]) for d in data])
    wants = [oracle.nonlocal_sum(f32(X), f32(q), f32(u0), f32(kern), f32(be), f32(th))
             for (ns, X, q, u0, be, th) in data]
    ref = None
    for depth in (3, 2):
        for split in (1, 2):
            for coef in (4.0, 8.0, 12.0):
                grp.configure(depth, split, coef)
                t = grp.tuning()
                assert (t["ring_depth"], t["traj_split"], t["lpt_coef"]) == (depth, split, coef)
                I = nf.nf_nonlocal_apply(grp, u, beta, theta)
                u2 = u.clone()
                nf.nf_rk4_advance(grp, u2, 0.0, 0.05, 2, beta, theta)
                grp.check()
                for got, want in zip(grp.split(I), wants):
                    err = np.linalg.norm(got.cpu().numpy() - want, axis=1) / np.linalg.norm(want, axis=1)
                    assert err.max() < REL_L2, (depth, split, coef, err.max())
                cur = (I.cpu().numpy(), u2.cpu().numpy())
                if ref is None:
                    ref = cur
                else:
                    np.testing.assert_allclose(cur[0], ref[0], rtol=1e-6, atol=1e-7 * np.abs(ref[0]).max())
                    np.testing.assert_allclose(cur[1], ref[1], rtol=1e-6, atol=1e-7 * np.abs(ref[1]).max())
    with pytest.raises(nf.NFError):
        grp.configure(4, 1, 8.0)
    grp.close()
    for op in ops:
        op.close()
