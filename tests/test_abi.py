"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol include/nf.h declares, and rejects bad arguments on the host side (no GPU
work is launched by these calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "nf.h")).read()
    return sorted(set(re.findall(r"NF_API\s+[\w\s\*]*?\b(nf_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def nf():
    import paper_2504_13379_gb300 as nf
    nf.lib()
    return nf


def test_header_declares_the_paper_calls():
    syms = header_symbols()
    for name in ["nf_build_stencils", "nf_quad_weights", "nf_nonlocal_apply", "nf_rk4_advance", "nf_adjoint"]:
        assert name in syms


def test_library_exports_every_declared_symbol(nf):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", nf._build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(nf_\w+)", out))
    missing = [s for s in header_symbols() if s not in exported]
    assert not missing, missing
    assert sorted(header_symbols()) == sorted(nf.EXPORTS)


def test_version(nf):
    assert nf.lib().nf_version() >> 16 == 1


def test_host_side_argument_errors(nf):
    L = nf.lib()
    h = C.c_void_p()
    kern = nf._Kernel(1.0, 0.1, 0.5, 0.2)
    assert L.nf_operator_create(None, None, 10, kern, 0, None, C.byref(h)) == 1
    assert b"non-NULL" in L.nf_last_error()
    bad = nf._Kernel(1.0, -0.1, 0.5, 0.2)
    assert L.nf_operator_create(C.c_void_p(16), C.c_void_p(16), 10, bad, 0, None, C.byref(h)) == 1
    assert L.nf_operator_create(C.c_void_p(16), C.c_void_p(16), 10, kern, 9, None, C.byref(h)) == 1
    assert L.nf_build_stencils(None, 10, 2, None, 5, 3, None, None) == 1
    assert L.nf_build_stencils(C.c_void_p(16), 10, 4, C.c_void_p(16), 5, 3, C.c_void_p(16), None) == 1
    assert L.nf_build_stencils(C.c_void_p(16), 10, 2, C.c_void_p(16), 5, 11, C.c_void_p(16), None) == 1
    bad_el = C.c_int64(0)
    # deg 3 needs 10 polynomial terms: k = 8 violates unisolvency
    assert L.nf_quad_weights(C.c_void_p(16), None, 100, 2, C.c_void_p(16), 50, C.c_void_p(16), 8, 3,
                             C.c_void_p(16), C.byref(bad_el), None) == 1
    assert b"unisolvency" in L.nf_last_error()
    assert bad_el.value == -1
    assert L.nf_nonlocal_apply(None, None, 1, None, None, None, None) == 1
    assert L.nf_rk4_advance(None, None, 1, 0.0, 0.1, 1, None, None, None, None, 1, None) == 1
    assert L.nf_operator_destroy(None) == 0


def test_mms_eigenvalues_match_oracle_quadrature(nf):
    import numpy as np
    import oracle
    for kp in [(1.0, 0.1, 0.5, 0.2), (1.2, 0.08, 0.6, 0.25), (1.0, 0.3, 0.5, 0.6)]:
        k32 = tuple(float(np.float32(v)) for v in kp)
        np.testing.assert_allclose(nf.nf_mms_sphere_eigs(kp), oracle.mms_sphere_eigs(k32), rtol=1e-12)
