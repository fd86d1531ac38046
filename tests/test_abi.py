"""The C-ABI library builds, loads and exports every function include/wgw.h declares (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libwgw():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2203_05623_gb300 import build
    return ctypes.CDLL(build.build())


def declared_functions():
    text = open(os.path.join(ROOT, "include", "wgw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wgw_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(libwgw):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(libwgw, n)]
    assert missing == []


def test_host_only_entry_points(libwgw):
    import paper_2203_05623_gb300 as W
    o = W.wgw_default_options()
    assert o.precision == W.WGW_FP64 and o.cg_tol == 1e-12 and o.dav_factor == 4
    libwgw.wgw_status_string.restype = ctypes.c_char_p
    assert libwgw.wgw_status_string(W.WGW_ERR_NOCONV) == b"Sternheimer solve did not converge"
    # Argument validation happens before any device work.
    h = ctypes.c_void_p()
    assert W.lib().wgw_setup(ctypes.byref(h), -1.0, 5.0, 24, None, 0, None, None, None, None, 4, None) == W.WGW_ERR_ARG
    assert b"invalid" in W.lib().wgw_last_error()
