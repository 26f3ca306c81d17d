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
    lib.otm_whiten_topic_workspace.argtypes = [ctypes.c_int64] * 4
    a = lib.otm_whiten_topic_workspace(100, 50, 5, 10)
    b = lib.otm_whiten_topic_workspace(1000, 500, 5, 10)
    assert 0 < a < b
