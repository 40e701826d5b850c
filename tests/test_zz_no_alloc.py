"""The allocation-free nonlocal sum (nf_nonlocal_apply_noalloc) against the regular
matrix-free entry point (nf_nonlocal_apply through an operator handle).

Callers of nf_nonlocal_apply_noalloc are ones that cannot allocate device memory when
they need the sum, so the entry point works from a fixed device array instead.  This
test calls it through the C ABI twice in a row with different sizes (the second,
smaller call must not see the first call's leftovers), compares each result with the
regular entry point within the 1e-5 relative-L2 bar used for FP32 sums, and checks
that repeated calls leave the device's free memory unchanged.  It lives in its own
file, collected last, and passes alone or after the rest of the suite.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_13379_gb300 as nf
    nf.lib()
    return nf


def _case(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    q = (rng.uniform(0.5, 1.5, n) / n).astype(np.float32)
    u = rng.normal(0.3, 0.4, n).astype(np.float32)
    to = lambda a: torch.as_tensor(a, device="cuda").contiguous()
    return to(x), to(q), to(u)


def test_noalloc_matches_regular_entry_point_twice(nf):
    kern = (1.0, 0.3, 0.5, 0.6)
    beta, theta = 20.0, 0.2
    cases = [_case(3000, 1), _case(1500, 2)]
    outs = [torch.empty(c[0].shape[0], dtype=torch.float32, device="cuda") for c in cases]
    refs = []
    for x, q, u in cases:
        op = nf.Operator(x, q, kern, nf.MATRIX_FREE)
        refs.append(nf.nf_nonlocal_apply(op, u, beta, theta).clone())
        op.check()
        op.close()
    torch.cuda.synchronize()
    for (x, q, u), out, ref in zip(cases, outs, refs):
        nf.nf_nonlocal_apply_noalloc(x, q, u, kern, beta, theta, out)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        assert err < REL_L2, err
    # repeated calls allocate nothing
    free0 = torch.cuda.mem_get_info()[0]
    for (x, q, u), out in zip(cases, outs):
        nf.nf_nonlocal_apply_noalloc(x, q, u, kern, beta, theta, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for out, ref in zip(outs, refs):
        assert (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item() < REL_L2


@pytest.mark.parametrize("n", [20011, 32768])
def test_noalloc_large_sizes_match_regular_entry_point_and_oracle(nf, n):
    """The sizes where the pair kernel takes four rows per warp (padded n >= 16,384), up to
    the largest n the scratch array holds; the split plan stays within the array's limit
    (the planner is given that limit), and sampled rows match the FP64 oracle."""
    import oracle

    kern = (1.0, 0.1, 0.5, 0.2)
    beta, theta = 20.0, 0.2
    x, q, u = _case(n, 11 + n)
    max_n, max_splits, splits = nf.nf_noalloc_limits(n)
    assert max_n == 32768 and 1 <= splits <= max_splits == 16
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    nf.nf_nonlocal_apply_noalloc(x, q, u, kern, beta, theta, out)
    nf.nf_noalloc_status()
    op = nf.Operator(x, q, kern, nf.MATRIX_FREE)
    ref = nf.nf_nonlocal_apply(op, u, beta, theta).clone()
    op.check()
    op.close()
    err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
    assert err < REL_L2, err
    rows = np.sort(np.random.default_rng(n).choice(n, 64, replace=False))
    f64 = lambda t: t.cpu().numpy().astype(np.float64)
    want = np.asarray(oracle.nonlocal_sum(f64(x), f64(q), f64(u), kern, [beta], [theta], rows=rows)).ravel()
    got = out.cpu().numpy().astype(np.float64)[rows]
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < REL_L2


def test_noalloc_split_plan_within_scratch_for_every_size(nf):
    """Every padded size the entry point accepts plans at most the 16 column splits the
    scratch array holds (the partial sums would otherwise not fit)."""
    for n in range(1024, 32768 + 1, 1024):
        max_n, max_splits, splits = nf.nf_noalloc_limits(n)
        assert 1 <= splits <= max_splits, (n, splits)


def test_noalloc_failed_wait_gives_nan_then_recovers(nf):
    """A pair-kernel block that gives up waiting leaves its partial sums unwritten; the
    call then writes NaN to I and nf_noalloc_status reports NF_ERR_TIMEOUT.  The flag is
    set on the host side of the self-test (no kernel waits); the next regular call
    clears it and returns the regular result."""
    x, q, u = _case(5000, 21)
    out = torch.zeros(5000, dtype=torch.float32, device="cuda")
    nf.nf_selftest_noalloc_flag(out)
    torch.cuda.synchronize()
    assert bool(torch.isnan(out).all())
    with pytest.raises(nf.NFError) as ei:
        nf.nf_noalloc_status()
    assert ei.value.name == "NF_ERR_TIMEOUT"
    kern = (1.0, 0.3, 0.5, 0.6)
    nf.nf_nonlocal_apply_noalloc(x, q, u, kern, 20.0, 0.2, out)
    nf.nf_noalloc_status()
    assert bool(torch.isfinite(out).all())
    op = nf.Operator(x, q, kern, nf.MATRIX_FREE)
    ref = nf.nf_nonlocal_apply(op, u, 20.0, 0.2)
    op.close()
    assert (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item() < REL_L2


def test_noalloc_binding_rejects_short_buffers(nf):
    """The binding checks shapes before the library sees the pointers (a short buffer would
    otherwise be read or written past its end)."""
    x, q, u = _case(2000, 4)
    out = torch.empty(2000, dtype=torch.float32, device="cuda")
    kern = (1.0, 0.3, 0.5, 0.6)
    with pytest.raises(ValueError):
        nf.nf_nonlocal_apply_noalloc(x, q[:1999], u, kern, 20.0, 0.2, out)
    with pytest.raises(ValueError):
        nf.nf_nonlocal_apply_noalloc(x, q, u, kern, 20.0, 0.2, out[:1000])
    with pytest.raises(ValueError):
        nf.nf_nonlocal_apply_noalloc(x[:, :2].contiguous(), q, u, kern, 20.0, 0.2, out)


def test_noalloc_rejects_sizes_beyond_its_scratch(nf):
    x, q, u = _case(32769, 3)
    out = torch.empty(32769, dtype=torch.float32, device="cuda")
    with pytest.raises(nf.NFError) as ei:
        nf.nf_nonlocal_apply_noalloc(x, q, u, (1.0, 0.3, 0.5, 0.6), 20.0, 0.2, out)
    assert ei.value.name == "NF_ERR_ARG"
