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
    assert c.tau_safety == 0.8  # last field: the struct layouts agree to the end


def test_workspace_sizing_and_config_validation():
    ok = hq.workspace_bytes(hq.default_config(64, 64))
    assert ok > 9 * 64 ** 3 * 64 * 8
    mixed = hq.workspace_bytes(hq.default_config(64, 64, precision="mixed"))
    assert 0 < mixed < ok
    assert hq.workspace_bytes(hq.default_config(2, 1)) == 0          # m < 3
    assert hq.workspace_bytes(hq.default_config(4, 65)) == 0         # N > n
    assert hq.workspace_bytes(hq.default_config(8, 4, tau=-1.0)) == 0
    assert hq.workspace_bytes(hq.default_config(8, 4, mg_nu1=0)) == 0
    for c in (0.0, -0.5, 1.5):
        assert hq.workspace_bytes(hq.default_config(8, 4, tau_safety=c)) == 0
    assert hq.workspace_bytes(hq.default_config(8, 4, tau_safety=1.0)) > 0


def test_status_strings():
    assert hq.status_string(0) == "ok"
    assert "breakdown" in hq.status_string(5)


def test_init_rejects_null_workspace_without_touching_a_device():
    lib = hq.load()
    c = hq.default_config(8, 4)
    ctx = ctypes.c_void_p()
    st = lib.hq_init(ctypes.byref(c), None, 0, None, ctypes.byref(ctx))
    assert st == 4 and not ctx.value


def test_batch_create_rejects_bad_arguments_without_touching_a_device():
    lib = hq.load()
    out = ctypes.c_void_p()
    assert lib.hq_batch_create(None, 1, None, ctypes.byref(out)) == 1 and not out.value
    fake = (ctypes.c_void_p * 2)(0x1000, 0x1000)          # repeated context
    assert lib.hq_batch_create(fake, 2, None, ctypes.byref(out)) == 1 and not out.value
    assert lib.hq_batch_create(fake, 0, None, ctypes.byref(out)) == 1
    assert lib.hq_batch_create(fake, 65, None, ctypes.byref(out)) == 1
    assert lib.hq_batch_last_error(None) == b"null batch"


def test_launch_shape_fields_and_tuner_workspace():
    lib = hq.load()
    c = hq.default_config(32, 16, precision="mixed")
    assert c.grid_block == 0 and c.grid_ctas == 0
    base = hq.workspace_bytes(c)
    tune_ws = int(lib.hq_tune_workspace_bytes(ctypes.byref(c)))
    assert tune_ws >= base > 0
    for b in (64, 128, 256):
        for k in (4, 8, 16, 32):
            t = hq.default_config(32, 16, precision="mixed", grid_block=b, grid_ctas=k)
            assert 0 < hq.workspace_bytes(t) <= tune_ws
    assert hq.workspace_bytes(hq.default_config(32, 16, grid_block=96)) == 0
    assert hq.workspace_bytes(hq.default_config(32, 16, grid_block=512)) == 0
    assert hq.workspace_bytes(hq.default_config(32, 16, grid_ctas=65)) == 0
    out = hq.Config()
    assert lib.hq_tune(ctypes.byref(c), None, 0, None, ctypes.byref(out), None) == 4


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the built libhq.so, loading raises."""
    monkeypatch.setattr(hq, "_lib", None)
    monkeypatch.setattr(hq, "LIB_PATH", "/nonexistent/libhq.so")
    with pytest.raises(RuntimeError, match="not built"):
        hq.load()


def test_device_operands_must_be_cuda_tensors():
    """Host tensors are refused before any call reaches the library."""
    import torch
    with pytest.raises(ValueError, match="CUDA tensor"):
        hq._dptr(torch.zeros(4, dtype=torch.float64))
    assert hq._dptr(None) is None
