"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/hh.h declares, and rejects bad arguments
before touching the device."""

import ctypes

import pytest

from paper_1811_07624_gb300 import _lib
from paper_1811_07624_gb300.build import build_library


@pytest.fixture(scope="module")
def L():
    build_library()
    return _lib.lib()


def test_exports_every_declared_symbol(L):
    names = _lib.header_symbols()
    assert "hh_create" in names and "hh_apply_sym" in names and "hh_backward" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, f"declared in include/hh.h but not exported: {missing}"


def test_signatures_cover_header(L):
    for name in _lib.header_symbols():
        if name in ("hh_last_error", "hh_version"):
            continue
        assert name in _lib.SIGNATURES, f"no ctypes signature for {name}"


def test_version_and_errors_without_device(L):
    assert L.hh_version().startswith(b"libhh")
    assert L.hh_destroy(None) == 0
    st = L.hh_create(None, 4, 1, None, 4, None, 0)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    assert b"out is NULL" in L.hh_last_error()
    h = ctypes.c_void_p()
    for args in ((0, 1), (4, -1)):
        st = L.hh_create(ctypes.byref(h), args[0], args[1], None, 4, None, 0)
        assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    st = L.hh_create(ctypes.byref(h), 4, 1, None, 4, None, 7)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    st = L.hh_plan_info(None, None, None, None, None)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    st = L.hh_apply(None, None, 4, None, 4, 1, None)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"


def test_python_error_type(L):
    with pytest.raises(_lib.HHError) as ei:
        _lib.call("hh_plan_info", None, None, None, None, None)
    assert ei.value.code == "HH_ERR_INVALID_ARG"
