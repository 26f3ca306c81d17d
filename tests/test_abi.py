"""CPU checks of the C ABI: the library builds, loads, exports every function
declared in include/otm.h, and rejects bad arguments on the host (no GPU work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1309_0787_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(otm_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("otm_whiten_topic", "otm_whiten_community", "otm_project", "otm_sgd_step",
                     "otm_sgd_run", "otm_unwhiten", "otm_recon_error", "otm_topic_moments"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_1309_0787_gb300 import otm
    assert set(_declared()) == set(otm.ENTRY_POINTS)


def test_version_and_empty_error(lib):
    lib.otm_version.restype = ctypes.c_int
    assert lib.otm_version() >= 100
    lib.otm_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.otm_last_error(), bytes)


def test_host_side_argument_errors(lib):
    """Invalid arguments return OTM_EINVAL (1) before any CUDA call."""
    lib.otm_last_error.restype = ctypes.c_char_p
    vp = ctypes.c_void_p
    f = lib.otm_sgd_step
    f.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_double,
                  ctypes.c_double, ctypes.c_double, vp, ctypes.c_size_t, vp]
    # k = 0
    assert f(vp(16), vp(16), vp(16), vp(16), 8, 0, vp(16), 1.0, 0.1, 1.0, None, 0, None) == 1
    assert b"k=0" in lib.otm_last_error()
    # k too large for the FP32 kernel
    assert f(vp(16), vp(16), vp(16), vp(16), 8, 129, vp(16), 1.0, 0.1, 1.0, None, 0, None) == 1
    # null pointer
    assert f(None, vp(16), vp(16), vp(16), 8, 4, vp(16), 1.0, 0.1, 1.0, None, 0, None) == 1
    g = lib.otm_syev
    g.argtypes = [vp, ctypes.c_int64, vp, vp, vp, ctypes.c_size_t, vp]
    assert g(vp(16), 200, vp(16), vp(16), vp(16), 1 << 30, None) == 1
    lib.otm_syev_workspace.restype = ctypes.c_size_t
    lib.otm_syev_workspace.argtypes = [ctypes.c_int64]
    assert g(vp(16), 10, vp(16), vp(16), vp(16), lib.otm_syev_workspace(10) - 1, None) == 1


def test_csr_validation(lib):
    from paper_1309_0787_gb300 import otm
    vp = ctypes.c_void_p
    lib.otm_project.argtypes = [ctypes.POINTER(otm.OtmCsr), vp, ctypes.c_int64, vp, vp, vp]
    bad = otm.OtmCsr(-1, 4, 0, 16, 16, 16)
    assert lib.otm_project(ctypes.byref(bad), vp(16), 4, None, vp(16), None) == 1
    nullrp = otm.OtmCsr(3, 4, 0, 0, 0, 0)
    assert lib.otm_project(ctypes.byref(nullrp), vp(16), 4, None, vp(16), None) == 1


def test_workspace_sizes_monotone(lib):
    lib.otm_whiten_topic_workspace.restype = ctypes.c_size_t
    lib.otm_whiten_topic_workspace.argtypes = [ctypes.c_int64] * 5
    a = lib.otm_whiten_topic_workspace(100, 50, 400, 5, 10)
    b = lib.otm_whiten_topic_workspace(1000, 500, 400, 5, 10)
    c = lib.otm_whiten_topic_workspace(1000, 500, 4000, 5, 10)
    assert 0 < a < b < c


def test_host_side_errors_of_membership_validation_and_nystrom(lib):
    """The newer entry points reject bad sizes on the host (OTM_EINVAL) before
    any CUDA call, so these run without a GPU."""
    from paper_1309_0787_gb300 import otm
    lib.otm_last_error.restype = ctypes.c_char_p
    vp, i64, f64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    m = lib.otm_membership
    m.argtypes = [vp, i64, i64, vp, f64, f64, vp, vp, sz, vp]
    assert m(vp(16), 10, 0, vp(16), 1.0, 0.0, vp(16), vp(16), 1 << 20, None) == 1   # k = 0
    assert m(vp(16), 10, 1025, vp(16), 1.0, 0.0, vp(16), vp(16), 1 << 20, None) == 1
    assert m(vp(16), -1, 4, vp(16), 1.0, 0.0, vp(16), vp(16), 1 << 20, None) == 1
    assert m(vp(16), 10, 4, None, 1.0, 0.0, vp(16), vp(16), 1 << 20, None) == 1    # V null
    assert m(vp(16), 10, 4, vp(16), 1.0, 0.0, vp(16), vp(16), 0, None) == 1        # workspace
    assert b"workspace" in lib.otm_last_error()
    p = lib.otm_pvalue_match
    p.argtypes = [vp, i64, vp, i64, i64, f64, vp, vp, vp, vp, sz, vp]
    assert p(vp(16), 3, vp(16), 3, 2, 0.01, vp(16), vp(16), vp(16), vp(16), 1 << 20, None) == 1
    assert b"n >= 3" in lib.otm_last_error()
    assert p(vp(16), 3, vp(16), 1025, 10, 0.01, vp(16), vp(16), vp(16), vp(16), 1 << 20,
             None) == 1
    assert p(vp(16), 3, None, 3, 10, 0.01, vp(16), vp(16), vp(16), vp(16), 1 << 20, None) == 1
    w = lib.otm_whiten_topic_nystrom
    w.argtypes = [ctypes.POINTER(otm.OtmCsr), vp, i64, i64, f64] + [vp] * 9 + [sz, vp]
    X = otm.OtmCsr(10, 40, 20, 16, 16, 16)
    outs = [vp(16)] * 8                          # S (vp(32)) must not alias O
    assert w(ctypes.byref(X), vp(32), 5, 5, 1.0, *outs, vp(16), 1 << 30, None) == 1   # kt = k
    assert w(ctypes.byref(X), vp(32), 5, 161, 1.0, *outs, vp(16), 1 << 30, None) == 1
    assert w(ctypes.byref(X), vp(32), 5, 41, 1.0, *outs, vp(16), 1 << 30, None) == 1  # kt > d
    assert w(ctypes.byref(X), vp(32), 5, 10, -1.0, *outs, vp(16), 1 << 30, None) == 1
    assert w(ctypes.byref(X), vp(32), 5, 10, 1.0, *outs, vp(16), 0, None) == 1
    assert b"workspace" in lib.otm_last_error()
    assert w(ctypes.byref(X), vp(16), 5, 10, 1.0, *outs, vp(16), 1 << 30, None) == 1
    assert b"alias" in lib.otm_last_error()
    lib.otm_whiten_topic_nystrom_workspace.restype = sz
    lib.otm_whiten_topic_nystrom_workspace.argtypes = [i64] * 4
    assert 0 < lib.otm_whiten_topic_nystrom_workspace(10, 40, 5, 10) < \
        lib.otm_whiten_topic_nystrom_workspace(1000, 4000, 5, 10)
