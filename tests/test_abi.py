"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/lbm.h.  Host-only calls (no device work) are checked too."""
import ctypes
import os
import re

import pytest

from paper_1903_01168_gb300 import build as B
from paper_1903_01168_gb300 import lbm as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
            if f.endswith(".h")]
    names = set()
    for h in hdrs:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_abi():
    names = declared_symbols()
    assert set(L.ABI_SYMBOLS) <= set(names)


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls():
    p = L.lbm_default_params()
    assert p.alpha_b == 0.2 and p.delta == 0.1 and p.beta == 0.99 and abs(p.mrt_lambda - 0.8) < 1e-15
    # 2 buffers x (2 FP32 density planes + 16 deviation planes) x ny x pitch,
    # pitch = nx + 2 * 8 ghost columns rounded to 16 bytes
    assert L.lbm_bytes_required(64, 32, p) == 2 * 2 * 32 * 80 * 4 + 2 * 16 * 32 * 80 * 4
    p.storage = L.LBM_F16DEV
    assert L.lbm_bytes_required(64, 32, p) == 2 * 5 * 32 * 80 * 4 + 2 * 16 * 32 * 80 * 2
    bad = L.lbm_default_params()
    bad.tau_r = 0.5
    assert L.lbm_bytes_required(64, 32, bad) == 0
    bad = L.lbm_default_params()
    bad.bc_x = L.LBM_BC_WALL
    assert L.lbm_bytes_required(64, 32, bad) == 0
    assert L.lbm_bytes_required(4, 32, L.lbm_default_params()) == 0


def test_batch_options_are_checked_before_any_device_call():
    lib = L.load()
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(None)
    opts = L.lbm_batch_opts(rows_per_item=0, row_overhead=1.0)
    assert lib.lbm_batch_create_ex(arr, 0, ctypes.byref(opts), ctypes.byref(h)) == L.LBM_EINVAL
    assert lib.lbm_batch_create_ex(arr, 1, None, ctypes.byref(h)) == L.LBM_EINVAL
    bad = L.lbm_batch_opts(rows_per_item=0, row_overhead=1.0, plan=7)
    assert lib.lbm_batch_create_ex(arr, 1, ctypes.byref(bad), ctypes.byref(h)) == L.LBM_EINVAL
    assert h.value is None


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(B, "LIB", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        L.load()
