"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/hh.h declares, and rejects bad arguments
before touching the device."""

import ctypes

import pytest

import paper_1811_07624_gb300 as hh
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
        assert name in _lib.SIGNATURES or name in _lib.VALUE_FUNCTIONS, \
            f"no ctypes signature for {name}"


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


def test_batch_shapes_and_tune_table_without_device(L, tmp_path):
    """The tile-shape table and the autotuner's table I/O are host logic."""
    shapes = hh.batch_shapes()
    assert len(shapes) == L.hh_batch_num_shapes() >= 2
    for s in shapes:
        if s["max_cluster"] == 0:
            assert s["cover"] == s["G"] * s["NG"] * 4 and s["max_h"] == -1
            # every staged shape stages ROWS x COVER floats in at most 128 KB of
            # shared memory: 256 threads holding 64 or 128 floats of vector state each
            assert s["rows_per_tile"] * s["cover"] * 4 in (65536, 131072)
        else:
            # the resident shape: G * NG * 4 columns per CTA, up to max_cluster CTAs,
            # and its CTA's columns of max_h reflectors in 200 KiB of shared memory
            assert s["cover"] == s["G"] * s["NG"] * 4 * s["max_cluster"]
            assert s["max_h"] * s["G"] * s["NG"] * 4 * 4 <= 200 * 1024
    resident = [k for k, s in enumerate(shapes) if s["max_cluster"] > 0]
    assert len(resident) == 1
    covers = sorted({s["cover"] for s in shapes})
    assert covers[-1] >= 4096
    hh.tune_clear()
    # untuned: the fixed rule, the smallest cover with four rows per thread
    for n in (4, 128, 256, 260, 512, 1024, 2048, 4096):
        shape, ms = hh.tune_get(n, 16)
        assert shapes[shape]["cover"] >= n
        assert all(m != m for m in ms)  # NaN: nothing measured
    hh.tune_set(640, 8, 4)
    hh.tune_set(640, 64, 5)
    assert hh.tune_get(640, 8)[0] == 4
    assert hh.tune_get(640, 64)[0] == 5
    assert hh.tune_get(640, 10)[0] == 4   # nearest tuned h
    assert hh.tune_get(640, 50)[0] == 5
    path = tmp_path / "shapes.txt"
    hh.tune_save(str(path))
    lines = [ln for ln in path.read_text().splitlines() if not ln.startswith("#")]
    assert sorted(lines) == ["640 64 5", "640 8 4"]
    hh.tune_clear()
    assert hh.tune_get(640, 8)[0] != 4 or shapes[4]["cover"] < 640
    hh.tune_load(str(path))
    assert hh.tune_get(640, 8)[0] == 4
    # a shape that does not cover n is refused, in both routes
    small = min(range(len(shapes)), key=lambda s: shapes[s]["cover"])
    with pytest.raises(hh.HHError, match="INVALID_ARG"):
        hh.tune_set(4096, 8, small)
    bad = tmp_path / "bad.txt"
    bad.write_text("4096 8 %d\n" % small)
    with pytest.raises(hh.HHError, match="INVALID_ARG"):
        hh.tune_load(str(bad))
    # the resident shape takes h <= max_h and n <= its cover
    r = resident[0]
    hh.tune_set(shapes[r]["cover"], shapes[r]["max_h"], r)
    assert hh.tune_get(shapes[r]["cover"], shapes[r]["max_h"])[0] == r
    for n, h in ((shapes[r]["cover"], shapes[r]["max_h"] + 1), (shapes[r]["cover"] + 4, 8)):
        with pytest.raises(hh.HHError, match="INVALID_ARG"):
            hh.tune_set(n, h, r)
    # a tuned resident entry is not taken for an h above its limit
    hh.tune_set(600, 8, r)
    assert hh.tune_get(600, 8)[0] == r
    assert hh.tune_get(600, shapes[r]["max_h"] + 50)[0] != r
    bad.write_text("600 %d %d\n" % (shapes[r]["max_h"] + 1, r))
    with pytest.raises(hh.HHError, match="INVALID_ARG"):
        hh.tune_load(str(bad))
    bad.write_text("128 x 0\n")
    with pytest.raises(hh.HHError, match="INVALID_ARG"):
        hh.tune_load(str(bad))
    with pytest.raises(hh.HHError, match="INVALID_ARG"):
        hh.tune_load(str(tmp_path / "missing.txt"))
    hh.tune_clear()


def test_batch_errors_without_device(L):
    import ctypes
    assert L.hh_batch_destroy(None) == 0
    st = L.hh_batch_create(None, 0, None, None)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    h = ctypes.c_void_p()
    st = L.hh_batch_create(ctypes.byref(h), -1, None, None)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    st = L.hh_batch_apply(None, 0, None, None, None, None, None)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    assert _lib.STATUS[L.hh_batch_shape(-1, None, None, None, None, None)] == "HH_ERR_INVALID_ARG"
    n = L.hh_batch_num_shapes()
    assert _lib.STATUS[L.hh_batch_shape_limits(n, None, None)] == "HH_ERR_INVALID_ARG"
    st = L.hh_tune(None, 1, None, 1, 16, None)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"


def test_debug_hooks_argument_checks_without_device(L):
    assert _lib.STATUS[L.hh_debug_fail_alloc(-1)] == "HH_ERR_INVALID_ARG"
    assert L.hh_debug_fail_alloc(0) == 0
    assert _lib.STATUS[L.hh_debug_wait_timeout(0, None)] == "HH_ERR_INVALID_ARG"
    assert _lib.STATUS[L.hh_debug_wait_timeout(5_000_000_000, None)] == "HH_ERR_INVALID_ARG"
