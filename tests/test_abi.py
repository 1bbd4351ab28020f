"""CPU checks of the C ABI: the library loads (no GPU call) and exports every
function include/ovl.h declares; the Python binding knows all of them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ovl.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ovl_[a-z_0-9A-Z]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0810_4228_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("ovl_apply_Dw", "ovl_sign_krylov", "ovl_set_deflation", "ovl_set_gauge", "ovl_create"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_0810_4228_gb300 import ovl
    assert sorted(ovl.EXPORTS) == _declared()


def test_create_rejects_bad_dims_without_gpu(lib):
    """Argument checks happen before any CUDA call."""
    h = ctypes.c_void_p()
    for dims, bc in (((4, 4, 4, 3), -1), ((1, 4, 4, 4), -1), ((4, 4, 4, 4), 0)):
        arr = (ctypes.c_int * 4)(*dims)
        assert lib.ovl_create(ctypes.byref(h), arr, bc, None) == 1  # OVL_EINVAL


def test_flags_match_header():
    from paper_0810_4228_gb300 import ovl
    with open(os.path.join(ROOT, "include", "ovl.h")) as f:
        src = f.read()
    for name in ("ARNOLDI", "LANCZOS2", "GAMMA5", "DAGGER", "NATIVE", "HOST", "F32", "F32_FULL",
                 "OVERLAP", "MIXED", "TWO_PASS", "INNER_NEWTON", "NO_GRAPH", "PROFILE",
                 "STENCIL_SITE", "STENCIL_SPLIT", "REPROJ", "STEPWISE", "PASS2_F64", "PASS2_DF", "NO_TUNE",
                 "ARNOLDI_CGS2"):
        m = re.search(r"#define\s+OVL_%s\s+(0x[0-9a-fA-F]+|\d+)" % name, src)
        assert m, name
        assert int(m.group(1), 0) == getattr(ovl, name), name


def test_reprojection_period_matches_header():
    """OVL_REPROJ_PERIOD(p) of the header (re-projection every p-th step) and the binding's
    REPROJ_PERIOD encode p the same way, in bits 24-30 beside the OVL_REPROJ bit."""
    from paper_0810_4228_gb300 import ovl
    with open(os.path.join(ROOT, "include", "ovl.h")) as f:
        src = f.read()
    m = re.search(r"#define\s+OVL_REPROJ_PERIOD\(p\)\s+\(OVL_REPROJ \| \(\(\(p\) & 0x7f\) << 24\)\)", src)
    assert m
    for p in (1, 2, 5, 127):
        assert ovl.REPROJ_PERIOD(p) == ovl.REPROJ | (p << 24)
        assert ovl.REPROJ_PERIOD(p) < 2 ** 31  # a non-negative C int
    for bad in (0, 128):
        with pytest.raises(ValueError):
            ovl.REPROJ_PERIOD(bad)
