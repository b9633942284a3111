"""ctypes binding of libhh.so: signatures, status codes and error messages.

Argument marshalling only; every computation runs in the library's CUDA
kernels.  Importing this module does not load the library; :func:`lib` does,
and raises if ``libhh.so`` has not been built (there is no fallback path).
"""

from __future__ import annotations

import ctypes
import os
import re
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libhh.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "hh.h")

STATUS = {
    0: "HH_OK",
    1: "HH_ERR_INVALID_ARG",
    2: "HH_ERR_UNSUPPORTED",
    3: "HH_ERR_NONFINITE",
    4: "HH_ERR_CUDA",
    5: "HH_ERR_OOM",
    6: "HH_ERR_TIMEOUT",
}
DTYPES = {"f32": 0, "f64": 1, "bf16": 2}
MODES = {"W": 0, "WT": 1, "SYM": 2}
PATHS = {"auto": 0, "fused": 1, "wy": 2}


class HHError(RuntimeError):
    """A libhh call returned a non-zero hh_status."""

    def __init__(self, status: int, func: str, message: str):
        self.status = status
        self.code = STATUS.get(status, str(status))
        super().__init__(f"{func}: {self.code}: {message}")


_lock = threading.Lock()
_lib = None

i64 = ctypes.c_int64
vp = ctypes.c_void_p
ip = ctypes.c_int

SIGNATURES = {
    "hh_create": [ctypes.POINTER(vp), i64, i64, vp, i64, vp, ip],
    "hh_create_ex": [ctypes.POINTER(vp), i64, i64, vp, i64, vp, vp, ip, ip, vp],
    "hh_destroy": [vp],
    "hh_sync": [vp, vp],
    "hh_update": [vp, vp, i64, vp, vp],
    "hh_plan_skip_prefix": [vp, ip, ctypes.POINTER(ip)],
    "hh_plan_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(ip),
                     ctypes.POINTER(ip)],
    "hh_apply": [vp, vp, i64, vp, i64, i64, vp],
    "hh_apply_T": [vp, vp, i64, vp, i64, i64, vp],
    "hh_apply_sym": [vp, vp, i64, vp, i64, i64, vp],
    "hh_backward": [vp, ip, vp, i64, vp, i64, vp, i64, vp, vp, i64, vp],
    "hh_backward_noalloc": [vp, ip, vp, i64, vp, i64, vp, i64, vp, vp, i64, vp],
    "hh_backward_sym_y": [vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, vp, i64, vp],
    "hh_backward_sym_py": [vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, vp, i64, vp],
    "hh_apply_sym_p": [vp, vp, i64, vp, i64, vp, i64, i64, vp],
    "hh_mahalanobis": [vp, vp, i64, i64, vp, vp, i64, vp, vp],
    "hh_mahalanobis_backward": [vp, vp, i64, i64, vp, vp, i64, vp, vp, vp, vp],
    "hh_batch_create": [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(i64)],
    "hh_batch_apply": [vp, ip, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(vp),
                       ctypes.POINTER(i64), vp],
    "hh_batch_sync": [vp, vp],
    "hh_batch_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(ip), ctypes.POINTER(ip)],
    "hh_batch_destroy": [vp],
    "hh_batch_shape": [ip] + [ctypes.POINTER(ip)] * 5,
    "hh_batch_shape_limits": [ip] + [ctypes.POINTER(ip)] * 2,
    "hh_tune": [ctypes.POINTER(i64), ip, ctypes.POINTER(i64), ip, i64, vp],
    "hh_tune_get": [i64, i64, ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_float)],
    "hh_tune_set": [i64, i64, ip],
    "hh_tune_save": [ctypes.c_char_p],
    "hh_tune_load": [ctypes.c_char_p],
    "hh_tune_clear": [],
    "hh_debug_fail_alloc": [ip],
    "hh_debug_wait_timeout": [i64, vp],
}

# Functions that return a plain value, not an hh_status.
VALUE_FUNCTIONS = {"hh_batch_num_shapes": ([], ctypes.c_int)}


def header_symbols() -> list[str]:
    """Names of the functions ``include/hh.h`` declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[A-Za-z0-9_]+)\s*\(", text)))


def lib():
    """Load libhh.so (once) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()'); "
                    "there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            for name, (args, res) in VALUE_FUNCTIONS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            L.hh_last_error.argtypes = []
            L.hh_last_error.restype = ctypes.c_char_p
            L.hh_version.argtypes = []
            L.hh_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def check(status: int, func: str) -> None:
    if status != 0:
        msg = lib().hh_last_error().decode(errors="replace")
        raise HHError(status, func, msg)


def call(name: str, *args) -> None:
    check(getattr(lib(), name)(*args), name)
