"""Parity at the time shapes the benchmark times, on reduced node counts the FP64 oracle
finishes in seconds.

* The differentiation workload: 200 RK4 steps of dt = 0.02 with a checkpoint every 20 steps
  (ten recomputed segments), the target trajectory from the hidden kernel (1.2, 0.08, 0.6,
  0.25), gradients at (1, 0.1, 0.5, 0.2); on a torus of a few thousand nodes, for the
  width-ratio-4 kernel (e1 = e2^4 inside the kernels) and a general two-exponential kernel,
  one and two trajectories.  The GPU adjoint is compared with the oracle's discrete adjoint
  (same terminal gradient lambda_T), and its directional derivative with an FP64 central
  difference of the oracle's loss (h = 1e-4).
* The batched workload's trajectory counts (256 on one node set, 64 on each of three more),
  10 RK4 steps through the grouped tensor-core path, against the oracle's RK4 on sampled
  trajectories of every node set.

Tolerances (relative L2 unless stated): dL/du0 1e-5; dL/d(A1, s1, A2, s2) 1e-5 as a vector
and 1e-4 per component, since a single small component is a sum over 4 x 200 stages of FP32
pair sums whose cancellation (the Mexican hat's two Gaussians of opposite sign) FP32 cannot
avoid (measured on GB300: 4e-7 and 9e-8 as vectors); the directional derivative 1e-4; the
bf16 x 3 grouped trajectories 1e-5, the bar of the FP32 paths: the split's per-term bound is
2^-17 + 2^-17 + 2^-18 ~= 1.9e-5, but with thousands of terms per sum the errors average out
(measured 1.1e-7 after 10 steps)."""
import numpy as np
import pytest
import torch

import nodesets
import oracle
from nodesets import workloads as W

pytestmark = pytest.mark.gpu

EVAL = (1.0, 0.1, 0.5, 0.2)        # the differentiation workload's evaluation point (ratio 4)
HIDDEN = (1.2, 0.08, 0.6, 0.25)    # its target kernel
GENERAL = (1.1, 0.09, 0.55, 0.23)  # non-integer width ratio: two exponentials per pair
DT, NSTEPS, C = 0.02, 200, 20


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


def _torus_case(n, B, seed):
    ns = nodesets.torus_lattice(n, 1.0, 0.4, 0.15, seed)
    n = ns.n
    X = ns.nodes.astype(np.float32)
    q = np.full(n, ns.area / n, dtype=np.float32)
    u0 = np.stack([nodesets.spiral_bumps_u0(ns, count=6 - b) for b in range(B)]).astype(np.float32)
    beta = np.array([20.0, 14.0][:B], dtype=np.float32)
    theta = np.array([0.2, 0.25][:B], dtype=np.float32)
    return X, q, u0, beta, theta


def _gpu_gradient(nf, X, q, u0, kern, beta, theta, lamT):
    B, n = u0.shape
    op = nf.Operator(dev(X), dev(q), kern, nf.MATRIX_FREE)
    u = dev(u0)
    ck = torch.zeros((NSTEPS // C + 1, B, n), dtype=torch.float32, device="cuda")
    nf.nf_rk4_advance(op, u, 0.0, DT, NSTEPS, dev(beta), dev(theta), ckpt=ck, C_every=C)
    gu, gk = nf.nf_adjoint(op, ck, C, 0.0, DT, NSTEPS, dev(beta), dev(theta), dev(lamT))
    op.check()
    out = u.cpu().numpy(), gu.cpu().numpy().astype(np.float64), gk.cpu().numpy().astype(np.float64)
    op.close()
    return out


@pytest.mark.parametrize("n,B,kern", [(3000, 1, EVAL), (2000, 2, EVAL), (2000, 1, GENERAL)])
def test_adjoint_200_steps_checkpoints_every_20(nf, n, B, kern):
    X, q, u0, beta, theta = _torus_case(n, B, seed=n + B)
    target = oracle.rk4(f32(X), f32(q), f32(u0), HIDDEN, f32(beta), f32(theta), 0.0, DT, NSTEPS)
    uN = oracle.rk4(f32(X), f32(q), f32(u0), f32(kern), f32(beta), f32(theta), 0.0, DT, NSTEPS)
    lamT = (2.0 * (uN - target)).astype(np.float32)
    uN_gpu, gu, gk = _gpu_gradient(nf, X, q, u0, kern, beta, theta, lamT)
    for b in range(B):
        assert np.linalg.norm(uN_gpu[b] - uN[b]) / np.linalg.norm(uN[b]) < 1e-5
    gu_o, gk_o = oracle.adjoint(f32(X), f32(q), f32(u0), f32(kern), f32(beta), f32(theta), 0.0, DT, NSTEPS,
                                f32(lamT))
    for b in range(B):
        e_u = np.linalg.norm(gu[b] - gu_o[b]) / np.linalg.norm(gu_o[b])
        e_k = np.linalg.norm(gk[b] - gk_o[b]) / np.linalg.norm(gk_o[b])
        print(f"n={X.shape[0]} B={B} kern={kern} traj {b}: dL/du0 rel L2 {e_u:.2e}, dL/dkernel rel L2 {e_k:.2e}")
        assert e_u < 1e-5
        assert e_k < 1e-5  # the four gradients as a vector
        np.testing.assert_allclose(gk[b], gk_o[b], rtol=1e-4, atol=1e-6 * np.abs(gk_o[b]).max())


def test_adjoint_200_steps_directional_derivative_vs_central_difference(nf):
    """<grad L, d> from the GPU adjoint against (L(p + h d) - L(p - h d)) / 2h of the
    oracle's FP64 loss, for one random direction d over (A1, s1, A2, s2) and u0."""
    X, q, u0, beta, theta = _torus_case(2000, 1, seed=17)
    target = oracle.rk4(f32(X), f32(q), f32(u0), HIDDEN, f32(beta), f32(theta), 0.0, DT, NSTEPS)
    uN = oracle.rk4(f32(X), f32(q), f32(u0), EVAL, f32(beta), f32(theta), 0.0, DT, NSTEPS)
    lamT = (2.0 * (uN - target)).astype(np.float32)
    _, gu, gk = _gpu_gradient(nf, X, q, u0, EVAL, beta, theta, lamT)
    rng = np.random.default_rng(23)
    dk = rng.normal(size=4) * np.abs(EVAL)            # relative to each parameter's size
    du = rng.normal(size=u0.shape) * 0.1
    gpu = float(gk[0] @ dk + np.sum(gu * du))
    h = 1e-4
    p = np.asarray(f32(EVAL))
    base = f32(u0)

    def L(s):
        return oracle.loss(f32(X), f32(q), base + s * du, p + s * dk, f32(beta), f32(theta), 0.0, DT, NSTEPS,
                           target)

    fd = (L(h) - L(-h)) / (2 * h)
    parts = abs(float(gk[0] @ dk)) + abs(float(np.sum(gu * du)))
    print(f"directional derivative: GPU adjoint {gpu:.9e}, FP64 central difference {fd:.9e}, "
          f"kernel part {float(gk[0] @ dk):.3e}, u0 part {float(np.sum(gu * du)):.3e}")
    assert abs(fd) > 0.1 * parts  # the direction does not cancel to noise
    assert abs(gpu - fd) <= 1e-4 * abs(fd)


def test_grouped_rk4_at_batched_trajectory_counts(nf):
    """256 trajectories on a sphere and 64 on each of three ellipsoids (1 : 0.8 : 0.6), node
    sets of 2,000-6,000 nodes, 10 RK4 steps of dt = 0.05 on the grouped tensor-core path;
    the oracle integrates 6 sampled trajectories of every node set (first, last, random)."""
    wls = W.batched(sizes=(6000, 2000, 3000, 4000), seed=3)
    kern = W.KERNEL
    ops, data = [], []
    for wl in wls:
        X = wl.ns.nodes.astype(np.float32)
        q = np.full(wl.n, (wl.ns.area or 4 * np.pi * 0.8) / wl.n, dtype=np.float32)
        ops.append(nf.Operator(dev(X), dev(q), kern, nf.DENSE_BF16X2))
        data.append((X, q, wl.u0.astype(np.float32), wl.beta.astype(np.float32), wl.theta.astype(np.float32)))
    assert [wl.B for wl in wls] == [256, 64, 64, 64]
    grp = nf.GroupedOperator(ops, [wl.B for wl in wls])
    u = torch.cat([dev(d[2]).reshape(-1) for d in data])
    beta = torch.cat([dev(d[3]) for d in data])
    theta = torch.cat([dev(d[4]) for d in data])
    nsteps, dt = 10, 0.05
    nf.nf_rk4_advance(grp, u, 0.0, dt, nsteps, beta, theta)
    grp.check()
    rng = np.random.default_rng(9)
    worst = 0.0
    for (X, q, u0, be, th), got in zip(data, grp.split(u)):
        B = u0.shape[0]
        sel = np.unique(np.concatenate([[0, B - 1], rng.choice(B, 4, replace=False)]))
        want = oracle.rk4(f32(X), f32(q), f32(u0[sel]), f32(kern), f32(be[sel]), f32(th[sel]), 0.0, dt, nsteps)
        g = got.cpu().numpy()[sel]
        err = np.linalg.norm(g - want, axis=1) / np.linalg.norm(want, axis=1)
        worst = max(worst, float(err.max()))
    print(f"grouped RK4 at the batched trajectory counts: worst relative L2 {worst:.3e}")
    assert worst < 1e-5
    grp.close()
    for op in ops:
        op.close()
