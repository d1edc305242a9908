"""The C-ABI library builds, loads and exports every function include/hq.h
declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

from paper_2605_25149_gb300 import build, hq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hq_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(hq.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 20
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(hq.EXPORTED) == declared


def test_config_struct_layout_and_defaults():
    c = hq.default_config(16, 8)
    assert (c.m, c.nev, c.lo, c.hi) == (16, 8, -6.0, 6.0)
    assert c.precision == hq.FP64 and c.mg_nu1 == 2 and c.mg_coarsest == 4
    assert c.shift != c.shift  # NaN: automatic shift


def test_workspace_sizing_and_config_validation():
    ok = hq.workspace_bytes(hq.default_config(64, 64))
    assert ok > 9 * 64 ** 3 * 64 * 8
    mixed = hq.workspace_bytes(hq.default_config(64, 64, precision="mixed"))
    assert 0 < mixed < ok
    assert hq.workspace_bytes(hq.default_config(2, 1)) == 0          # m < 3
    assert hq.workspace_bytes(hq.default_config(4, 65)) == 0         # N > n
    assert hq.workspace_bytes(hq.default_config(8, 4, tau=-1.0)) == 0
    assert hq.workspace_bytes(hq.default_config(8, 4, mg_nu1=0)) == 0


def test_status_strings():
    assert hq.status_string(0) == "ok"
    assert "breakdown" in hq.status_string(5)


def test_init_rejects_null_workspace_without_touching_a_device():
    lib = hq.load()
    c = hq.default_config(8, 4)
    ctx = ctypes.c_void_p()
    st = lib.hq_init(ctypes.byref(c), None, 0, None, ctypes.byref(ctx))
    assert st == 4 and not ctx.value
