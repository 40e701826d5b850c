"""Full-size checks of the sphere and differentiation workloads in the launch
configuration the benchmark times, against the FP64 oracle on the same inputs.

* Unit sphere, n = 20,000 (k = 32, degree 3), manufactured forcing of §4 Eq. (4.5):
  one RK4 step against the oracle on every node (1e-5 relative L2), then the full
  200 steps against the manufactured solution u*.
* Torus, n = 40,000: the discrete RK4 adjoint (gradients in u0 and in the four
  kernel parameters) over one step against the oracle's adjoint.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from nodesets import workloads as W

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


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


def test_sphere_workload_full_size(nf):
    wl = W.sphere()
    st = oracle.knn(wl.ns.nodes, wl.ns.tris, wl.k)
    q = oracle.quad_weights(wl.ns.nodes, wl.ns.tris, st, wl.deg, normals=wl.ns.normals).astype(np.float32)
    X = wl.ns.nodes.astype(np.float32)
    u0 = wl.u0.astype(np.float32)
    c, a0 = wl.forcing["c"], wl.forcing["a0"]
    beta, theta = float(wl.beta[0]), float(wl.theta[0])
    F = nf.Forcing(nf.FORCE_MMS_EIGEN, dev(0.5 * X[:, 2]), dev(f32(X[:, 0]) * f32(X[:, 1])), c, a0,
                   nf.nf_mms_sphere_eigs(wl.kernel))
    op = nf.Operator(dev(X), dev(q), wl.kernel, nf.MATRIX_FREE)
    u = dev(u0)
    nf.nf_rk4_advance(op, u, 0.0, wl.dt, 1, beta, theta, forcing=F)
    op.check()
    Fo = oracle.mms_sphere_forcing(f32(wl.kernel), c, a0)
    want = oracle.rk4(f32(X), f32(q), f32(u0), f32(wl.kernel), f32(wl.beta), f32(wl.theta), 0.0, wl.dt, 1,
                      forcing=Fo)
    got = u.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < REL_L2
    # the whole run (t = 0 .. 2): the semi-discrete solution tracks u*, to 1.8e-5 of
    # max |u*| at this n; a wrong sign or eigenvalue in the forcing gives errors of 1e-2
    u = dev(u0)
    nf.nf_rk4_advance(op, u, 0.0, wl.dt, wl.nsteps, beta, theta, forcing=F)
    op.check()
    T = wl.dt * wl.nsteps
    Xd = wl.ns.nodes
    z = c + a0 * math.cos(T) * (0.5 * Xd[:, 2] + Xd[:, 0] * Xd[:, 1])
    ustar = theta + np.log(z / (1.0 - z)) / beta
    err = np.abs(u.double().cpu().numpy().ravel() - ustar).max() / np.abs(ustar).max()
    assert err < 1e-4, err
    op.close()


def test_adjoint_workload_full_size(nf):
    wl = W.adjoint()
    n = wl.n
    X = wl.ns.nodes.astype(np.float32)
    q = np.full(n, wl.ns.area / n, dtype=np.float32)
    u0 = wl.u0.astype(np.float32)
    rng = np.random.default_rng(40000)
    target = (0.9 * u0 + 0.05 * rng.normal(size=u0.shape)).astype(np.float32)
    beta, theta = float(wl.beta[0]), float(wl.theta[0])
    nsteps, C = 1, 1
    op = nf.Operator(dev(X), dev(q), wl.kernel, nf.MATRIX_FREE)
    u = dev(u0)
    ck = torch.zeros((nsteps // C + 1, 1, n), dtype=torch.float32, device="cuda")
    nf.nf_rk4_advance(op, u, 0.0, wl.dt, nsteps, beta, theta, ckpt=ck, C_every=C)
    gu, gk = nf.nf_adjoint(op, ck, C, 0.0, wl.dt, nsteps, beta, theta, 2.0 * (u - dev(target)))
    op.check()
    op.close()
    uN = oracle.rk4(f32(X), f32(q), f32(u0), f32(wl.kernel), f32(wl.beta), f32(wl.theta), 0.0, wl.dt, nsteps)
    gu_o, gk_o = oracle.adjoint(f32(X), f32(q), f32(u0), f32(wl.kernel), f32(wl.beta), f32(wl.theta), 0.0,
                                wl.dt, nsteps, 2.0 * (uN - f32(target)))
    gu = gu.cpu().numpy()
    gk = gk.cpu().numpy()
    assert np.linalg.norm(gu[0] - gu_o[0]) / np.linalg.norm(gu_o[0]) < REL_L2
    np.testing.assert_allclose(gk[0], gk_o[0], rtol=1e-4, atol=1e-6 * np.abs(gk_o[0]).max())
