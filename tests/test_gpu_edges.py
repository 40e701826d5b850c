"""Edge and degenerate cases of the operator paths: argument checks, zero steps, a kernel
that is identically zero, and node sets collapsed to one point (every pair at r = 0, so
I_i = w(0) sum_j q_j f(u_j) in closed form)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

PATHS = [0, 1, 2, 4, 5]


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_13379_gb300 as nf
    nf.lib()
    return nf


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def test_operator_rejects_bad_arguments(nf):
    X = dev(np.zeros((10, 3)))
    q = dev(np.ones(10))
    for kern, path in (((1.0, 0.0, 0.5, 0.2), 0), ((1.0, 0.1, 0.5, -0.2), 0), ((1.0, 0.1, 0.5, 0.2, -1.0), 0),
                       ((float("nan"), 0.1, 0.5, 0.2), 0), ((1.0, 0.1, 0.5, 0.2), 3), ((1.0, 0.1, 0.5, 0.2), 7)):
        with pytest.raises(nf.NFError) as ei:
            nf.Operator(X, q, kern, path)
        assert ei.value.name == "NF_ERR_ARG"
    with pytest.raises(nf.NFError):
        nf.Operator(dev(np.zeros((0, 3))), dev(np.zeros(0)), (1.0, 0.1, 0.5, 0.2), 0)
    op = nf.Operator(X, q, (1.0, 0.1, 0.5, 0.2), 0)
    with pytest.raises(nf.NFError):
        op.mf_schedule(9)
    dense = nf.Operator(X, q, (1.0, 0.1, 0.5, 0.2), 1)
    with pytest.raises(nf.NFError):
        dense.mf_schedule(1)
    with pytest.raises(nf.NFError):
        dense.mf_cull(True)


@pytest.mark.parametrize("path", PATHS)
def test_zero_steps_and_checkpoint(nf, path):
    rng = np.random.default_rng(path)
    n = 1500
    X = rng.uniform(-1, 1, (n, 3))
    op = nf.Operator(dev(X), dev(np.full(n, 1.0 / n)), (1.0, 0.2, 0.5, 0.4), path)
    u0 = rng.normal(size=(2, n)).astype(np.float32)
    u = dev(u0)
    ck = torch.full((1, 2, n), -7.0, device="cuda")
    nf.nf_rk4_advance(op, u, 0.0, 0.05, 0, dev(np.array([20.0, 10.0])), dev(np.array([0.2, 0.3])), ckpt=ck,
                      C_every=1)
    op.check()
    np.testing.assert_array_equal(u.cpu().numpy(), u0)
    np.testing.assert_array_equal(ck[0].cpu().numpy(), u0)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("B", [1, 3, 17])
def test_zero_kernel_gives_zero_sums(nf, path, B):
    rng = np.random.default_rng(B + path)
    n = 2100
    X = rng.uniform(-1, 1, (n, 3))
    op = nf.Operator(dev(X), dev(rng.uniform(0.5, 1.5, n) / n), (0.0, 0.2, 0.0, 0.4), path)
    u = dev(rng.normal(size=(B, n)))
    I = nf.nf_nonlocal_apply(op, u, dev(np.full(B, 20.0)), dev(np.full(B, 0.2)))
    op.check()
    assert torch.count_nonzero(I).item() == 0


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("B", [1, 2, 5])
def test_collapsed_node_set_closed_form(nf, path, B):
    """All nodes at one point: every pair has r = 0, so every row sum equals
    (A1 - A2) sum_j q_j f(u_j) -- the same for all i, known in closed form."""
    rng = np.random.default_rng(10 * B + path)
    n = 3000
    X = np.tile(np.array([[0.3, -0.2, 0.7]]), (n, 1))
    q = rng.uniform(0.5, 1.5, n) / n
    u = rng.normal(0.2, 0.5, (B, n))
    beta, theta = rng.uniform(5, 30, B), rng.uniform(0.0, 0.4, B)
    kern = (1.3, 0.2, 0.45, 0.4)
    q32, u32 = q.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64)
    b32, t32 = beta.astype(np.float32).astype(np.float64), theta.astype(np.float32).astype(np.float64)
    f = 1.0 / (1.0 + np.exp(-b32[:, None] * (u32 - t32[:, None])))
    want = (np.float64(np.float32(1.3)) - np.float64(np.float32(0.45))) * (f * q32).sum(1)
    op = nf.Operator(dev(X), dev(q), kern, path)
    if path == 0:
        op.mf_schedule(nf.MF_SYMMETRIC)
    I = nf.nf_nonlocal_apply(op, dev(u), dev(beta), dev(theta)).cpu().numpy().astype(np.float64)
    op.check()
    np.testing.assert_allclose(I, np.repeat(want[:, None], n, 1), rtol=1e-5)


@pytest.mark.parametrize("path", PATHS)
def test_nonfinite_state_is_reported(nf, path):
    """A NaN in the initial state spreads through the sums; the RK4 step records it on the
    operator and the check reports NF_ERR_NONFINITE (a finite run on another operator of
    the same nodes reports nothing)."""
    rng = np.random.default_rng(40 + path)
    n = 1500
    X = dev(rng.uniform(-1, 1, (n, 3)))
    q = dev(np.full(n, 1.0 / n))
    u0 = rng.normal(size=(1, n)).astype(np.float32)
    ok = nf.Operator(X, q, (1.0, 0.2, 0.5, 0.4), path)
    nf.nf_rk4_advance(ok, dev(u0), 0.0, 0.05, 2, 20.0, 0.2)
    ok.check()
    u0[0, 7] = np.nan
    bad = nf.Operator(X, q, (1.0, 0.2, 0.5, 0.4), path)
    nf.nf_rk4_advance(bad, dev(u0), 0.0, 0.05, 2, 20.0, 0.2)
    with pytest.raises(nf.NFError) as ei:
        bad.check()
    assert ei.value.name == "NF_ERR_NONFINITE"


def test_pipe_probe_rates_are_plausible(nf):
    """The instruction-rate probe behind the pair kernels' roofline: FP32 FMA lanes per
    clock per SM (scalar and f32x2) and SFU ex2 per clock per SM within the range any
    recent NVIDIA SM can have, and the implied SM clock within the part's range."""
    for kind, lo, hi in ((nf.PROBE_FMA, 32.0, 260.0), (nf.PROBE_FMA2, 32.0, 260.0), (nf.PROBE_EX2, 4.0, 64.0)):
        rate, mhz, ms = nf.nf_probe_pipe(kind, 2000)
        assert lo <= rate <= hi, (kind, rate)
        assert 300.0 <= mhz <= 2500.0, (kind, mhz)
        assert ms > 0.0


def test_profiling_ring_keeps_every_step(nf):
    """With a ring of K event sets, the last K RK4 steps keep their own stage timings; the
    most recent step's timings equal nf_operator_kernel_ms."""
    rng = np.random.default_rng(3)
    n = 5000
    X = dev(rng.uniform(-1, 1, (n, 3)))
    q = dev(np.full(n, 1.0 / n))
    for path in (0, 1):
        op = nf.Operator(X, q, (1.0, 0.3, 0.5, 0.6), path)
        op.profile(True, ring=5)
        u = dev(rng.normal(0.2, 0.3, n)).view(1, -1)
        for _ in range(3):
            nf.nf_rk4_advance(op, u, 0.0, 0.05, 1, 20.0, 0.2)
        nf.nf_rk4_advance(op, u, 0.0, 0.05, 4, 20.0, 0.2)
        hist = op.kernel_ms_history(5)
        assert len(hist) == 5 and all(len(h) == 4 and min(h) > 0.0 for h in hist)
        assert op.kernel_ms() == hist[-1]
        with pytest.raises(nf.NFError):
            op.kernel_ms_history(6)
        op.check()
        op.close()
