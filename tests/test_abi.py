"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/kg.h declares.  No CUDA compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2507_13204_gb300 import _lib as L
from paper_2507_13204_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kg_[a-z_]+)\s*\(", src)))


def test_header_matches_binding_list():
    assert declared_functions() == sorted(L.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a(lib):
    # the device code in the fatbin is sm_103a (checked through the build flags we pass)
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
    assert os.path.dirname(L.LIB_PATH).endswith("paper_2507_13204_gb300")


def test_options_default_and_struct_layout(lib):
    o = L.kg_options()
    o.dtype = 7
    lib.kg_options_default(ctypes.byref(o))
    assert (o.dtype, o.strategy, o.mode, o.arith, o.check) == (L.KG_F64, 0, 0, 0, 0)
    assert ctypes.sizeof(L.kg_options) == 40


@pytest.mark.parametrize("sizes,nsizes", [((0,), 1), ((-5,), 1), ((1 << 31,), 1)])
def test_create_rejects_bad_sizes_before_touching_the_device(lib, sizes, nsizes):
    h = ctypes.c_void_p()
    sz = (ctypes.c_int64 * len(sizes))(*sizes)
    data = (ctypes.c_void_p * 1)(16)
    rc = lib.kg_create(ctypes.byref(h), L.KG_QUADFORM, sz, nsizes, data, 1, None, None)
    assert rc == L.KG_ERR_INVALID_ARG
    assert "size" in lib.kg_last_error().decode()
    assert not h.value


def test_create_rejects_bad_enums(lib):
    h = ctypes.c_void_p()
    sz = (ctypes.c_int64 * 1)(8)
    data = (ctypes.c_void_p * 1)(16)
    for field, bad in [("dtype", 5), ("strategy", 9), ("mode", 4), ("arith", 3), ("block", 33)]:
        o = L.kg_options()
        lib.kg_options_default(ctypes.byref(o))
        setattr(o, field, bad)
        rc = lib.kg_create(ctypes.byref(h), L.KG_QUADFORM, sz, 1, data, 1, ctypes.byref(o), None)
        assert rc == L.KG_ERR_INVALID_ARG, field


def test_null_handles_are_rejected(lib):
    assert lib.kg_eval(None, None, None, None) == L.KG_ERR_INVALID_ARG
    assert lib.kg_grad(None, None, None, None, None, None, 0, None) == L.KG_ERR_INVALID_ARG
    assert lib.kg_sync(None) == L.KG_ERR_INVALID_ARG
    lib.kg_destroy(None)
    lib.kg_batch_destroy(None)
    assert lib.kg_workspace_bytes(None) == 0


def test_binding_raises_with_message(lib):
    with pytest.raises(L.KGError) as ei:
        L.check(lib.kg_eval(None, None, None, None), "kg_eval")
    assert ei.value.status == L.KG_ERR_INVALID_ARG and "NULL" in str(ei.value)


def test_environment_overrides_of_the_options(lib, monkeypatch):
    for var in ("KG_STRATEGY", "KG_MODE", "KG_ARITH", "KG_CHECK"):
        monkeypatch.delenv(var, raising=False)
    o = L.options()
    L.kg_options_apply_env(o)  # nothing set: unchanged
    assert (o.strategy, o.mode, o.arith, o.check) == (0, 0, 0, 0)
    monkeypatch.setenv("KG_STRATEGY", "csr")
    monkeypatch.setenv("KG_MODE", "tape")
    monkeypatch.setenv("KG_ARITH", "native")
    monkeypatch.setenv("KG_CHECK", "1")
    L.kg_options_apply_env(o)
    assert (o.strategy, o.mode, o.arith, o.check) == (L.KG_STRATEGY_CSR, L.KG_MODE_TAPE,
                                                      L.KG_ARITH_NATIVE, 1)
    monkeypatch.setenv("KG_MODE", "sometimes")
    before = (o.strategy, o.mode, o.arith, o.check)
    with pytest.raises(L.KGError) as ei:
        L.kg_options_apply_env(o)
    assert ei.value.status == L.KG_ERR_INVALID_ARG and "KG_MODE" in str(ei.value)
    assert (o.strategy, o.mode, o.arith, o.check) == before
    # kg_create applies them before it touches the device: a bad value is rejected first
    h = ctypes.c_void_p()
    sz = (ctypes.c_int64 * 1)(8)
    data = (ctypes.c_void_p * 1)(16)
    assert lib.kg_create(ctypes.byref(h), L.KG_QUADFORM, sz, 1, data, 1, None, None) == L.KG_ERR_INVALID_ARG
    assert "KG_MODE" in lib.kg_last_error().decode()


def test_tape_generation_rejects_null(lib):
    g = ctypes.c_uint64(7)
    assert lib.kg_tape_generation(None, ctypes.byref(g)) == L.KG_ERR_INVALID_ARG
