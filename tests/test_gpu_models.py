"""GPU parity of nf_field_advance (the §5 models: neural field or synaptic depression,
sigmoid or C^4 smooth-step rate, RK4 or AB5) against the FP64 oracle, which is pinned in
tests/test_oracle_models.py.  Bar: 1e-5 relative L2 per trajectory for u and s."""
import numpy as np
import pytest
import torch

import nodesets
import oracle

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


def rel_l2(got, want):
    return max(np.linalg.norm(g - w) / np.linalg.norm(w) for g, w in zip(np.atleast_2d(got), np.atleast_2d(want)))


def _case(n=1600, B=1, seed=0):
    ns = nodesets.torus_lattice(n, seed=seed)
    X = ns.nodes.astype(np.float32)
    mu = np.full(ns.n, ns.area / ns.n, dtype=np.float32)
    u0 = np.stack([(0.7 + 0.2 * b) * nodesets.spiral_bumps_u0(ns, count=3 + b) for b in range(B)]).astype(np.float32)
    rng = np.random.default_rng(seed)
    s0 = rng.uniform(0.5, 1.0, size=u0.shape).astype(np.float32)
    return ns, X, mu, u0, s0


def _run(nf, path, kind, rate, integ, B=1, nsteps=30, dt=0.02, n=1600):
    ns, X, mu, u0, s0 = _case(n, B)
    kern = (5.0, 0.3, 7.0, 0.6)
    beta = np.array([20.0, 12.0, 30.0][:B], dtype=np.float32)
    theta = np.array([0.2, 0.25, 0.15][:B], dtype=np.float32)
    tau, bd = 3.0, 0.6
    op = nf.Operator(dev(X), dev(mu), kern, path)
    u = dev(u0)
    s = dev(s0) if kind == 1 else None
    nf.nf_field_advance(op, u, dt, nsteps, dev(beta), dev(theta), s=s, rate=rate, tau=tau, beta_d=bd,
                        integrator=integ)
    op.check()
    want = oracle.field_advance(f32(X), f32(mu), f32(u0), f32(kern), f32(beta), f32(theta), float(np.float32(dt)),
                                nsteps, s0=f32(s0), kind=kind, rate_kind=rate, a=float(np.float32(0.06)),
                                b=float(np.float32(0.54)), tau=float(np.float32(tau)), beta_d=float(np.float32(bd)),
                                integrator=integ)
    if kind == 1:
        wu, ws = want
        assert rel_l2(u.cpu().numpy(), wu) < REL_L2
        assert rel_l2(s.cpu().numpy(), ws) < REL_L2
    else:
        assert rel_l2(u.cpu().numpy(), want) < REL_L2


@pytest.mark.parametrize("integ", ["rk4", "ab5"])
@pytest.mark.parametrize("rate", [0, 1])
@pytest.mark.parametrize("kind", [0, 1])
def test_models_matrix_free(nf, kind, rate, integ):
    _run(nf, 0, kind, rate, integ)


@pytest.mark.parametrize("path", [1, 2, 4, 5])
def test_depression_ab5_dense_paths(nf, path):
    """The dense paths (W diag(mu) FP32 and bf16 hi+lo; symmetric K with mu on the vector
    side) under the depression model with the smooth step and AB5."""
    _run(nf, path, 1, 1, "ab5")


@pytest.mark.parametrize("integ", ["rk4", "ab5"])
def test_models_several_trajectories(nf, integ):
    """Three trajectories with their own sigmoid parameters (multi-trajectory kernels)."""
    _run(nf, 0, 1, 0, integ, B=3, nsteps=12)


def test_ab5_fewer_steps_than_its_start(nf):
    """nsteps <= 4: AB5 is all start-up RK4 steps, identical to RK4."""
    ns, X, mu, u0, s0 = _case(1200)
    kern = (5.0, 0.3, 7.0, 0.6)
    op = nf.Operator(dev(X), dev(mu), kern, 0)
    ua, ub = dev(u0), dev(u0)
    nf.nf_field_advance(op, ua, 0.02, 3, 20.0, 0.2, integrator="ab5")
    nf.nf_field_advance(op, ub, 0.02, 3, 20.0, 0.2, integrator="rk4")
    op.check()
    np.testing.assert_array_equal(ua.cpu().numpy(), ub.cpu().numpy())


def test_field_advance_rejects_bad_arguments(nf):
    ns, X, mu, u0, s0 = _case(500)
    op = nf.Operator(dev(X), dev(mu), (1.0, 0.1, 0.5, 0.2), 0)
    u = dev(u0)
    with pytest.raises(nf.NFError):
        nf.nf_field_advance(op, u, 0.02, 5, 20.0, 0.2, s=dev(s0), tau=0.0)  # depression needs tau > 0
    with pytest.raises(nf.NFError):
        nf.nf_field_advance(op, u, 0.02, 5, 20.0, 0.2, rate=1, a=0.5, b=0.1)  # empty transition
