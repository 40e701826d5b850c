"""Failure detection without a GPU fault: a kernel whose wait can never complete gives
up after a bounded number of polls, the call reports NF_ERR_TIMEOUT, and the CUDA
context keeps working afterwards."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_13379_gb300 as nf
    nf.lib()
    return nf


def test_bounded_wait_reports_timeout_and_context_survives(nf):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = nf.lib().nf_selftest_timeout(stream)
    assert nf.STATUS[st] == "NF_ERR_TIMEOUT", nf.lib().nf_last_error()
    # the context is intact: a regular computation still matches the oracle
    rng = np.random.default_rng(0)
    n = 700
    X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    q = np.full(n, 1.0 / n, dtype=np.float32)
    u = rng.normal(0.2, 0.3, size=(1, n)).astype(np.float32)
    op = nf.Operator(torch.as_tensor(X, device="cuda"), torch.as_tensor(q, device="cuda"), (1.0, 0.3, 0.5, 0.6))
    got = nf.nf_nonlocal_apply(op, torch.as_tensor(u, device="cuda"), 20.0, 0.2)
    op.check()
    f64 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    want = oracle.nonlocal_sum(f64(X), f64(q), f64(u), (1.0, 0.3, 0.5, 0.6), 20.0, np.float32(0.2))
    assert np.linalg.norm(got.cpu().numpy() - want) / np.linalg.norm(want) < 1e-5
