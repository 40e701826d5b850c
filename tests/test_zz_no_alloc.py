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


def test_noalloc_rejects_sizes_beyond_its_scratch(nf):
    x, q, u = _case(32769, 3)
    out = torch.empty(32769, dtype=torch.float32, device="cuda")
    with pytest.raises(nf.NFError) as ei:
        nf.nf_nonlocal_apply_noalloc(x, q, u, (1.0, 0.3, 0.5, 0.6), 20.0, 0.2, out)
    assert ei.value.name == "NF_ERR_ARG"
