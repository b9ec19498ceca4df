"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/vms.h declares.
These run without a GPU: no compute call is made."""
import os
import re
import ctypes

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vms_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0809_4802_gb300 import build, vms
    build.build()
    return vms.load_library()


def test_header_declares_the_boundary_calls():
    syms = declared_symbols()
    for name in ("vms_create", "vms_mesh_upload", "vms_state_upload", "vms_assemble_newton_schur",
                 "vms_apply", "vms_solve", "vms_newton_step", "vms_residual"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_0809_4802_gb300 import vms
    syms = declared_symbols()
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(vms.EXPORTS) == syms


def test_version_string(lib):
    assert b"sm_103a" in lib.vms_version()


def test_bad_arguments_return_codes_without_a_device(lib):
    from paper_0809_4802_gb300 import vms
    assert lib.vms_create(None, 0, 0) == vms.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.vms_create(ctypes.byref(h), 0, 7) == vms.ERR_INVALID_ARG
    assert lib.vms_destroy(None) == vms.OK
    assert lib.vms_set_stream(None, None) == vms.ERR_INVALID_ARG
    assert lib.vms_residual(None, None, None) == vms.ERR_INVALID_ARG
    assert lib.vms_last_error(None) == b"null context"


def test_library_is_built_for_sm_103a_only():
    from paper_0809_4802_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_library_tet_rule_matches_the_oracle(n):
    """The library's conical-product rule (Gauss-Jacobi points by Golub-Welsch in C++) against the
    oracle's (scipy's Gauss-Jacobi roots): same points and weights (host code, no GPU)."""
    import oracle
    from paper_0809_4802_gb300 import vms
    pts, wts = vms.tet_rule(n)
    opts, owts = oracle.tet_rule(n)
    order = np.lexsort(pts.T[::-1])
    oorder = np.lexsort(opts.T[::-1])
    np.testing.assert_allclose(pts[order], opts[oorder], rtol=0, atol=1e-14)
    np.testing.assert_allclose(wts[order], owts[oorder], rtol=1e-13, atol=1e-17)
