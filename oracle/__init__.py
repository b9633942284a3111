"""FP64 CPU oracle for the Householder-chain transforms (arXiv 1811.07624).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg call it; the library path never does.  It shares
no code with the CUDA path: the arithmetic lives in ``hh_oracle.c`` (plain
loops in double, §II-A Eqs. (1)-(2), §III-A Eq. (21), §IV-C) and in
``dense.py`` (explicit n x n matrix products, for tiny n).

Each wrapper takes numpy arrays (converted to float64, C order) and returns
numpy arrays.  The shared object is compiled with gcc on first use (or by
``build_oracle()``) next to this file.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hh_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODES = {"W": 0, "WT": 1, "SYM": 2}


def build_oracle(force: bool = False) -> str:
    """Compile ``hh_oracle.c`` into ``liboracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # HH_ORACLE_LIB points the wrapper at another build of hh_oracle.c
            # (the mutation tests load deliberately broken copies this way).
            path = os.environ.get("HH_ORACLE_LIB") or build_oracle()
            lib = ctypes.CDLL(path)
            i64, dp, vp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
            lib.oracle_tau.argtypes = [i64, i64, dp, i64, dp]
            lib.oracle_apply.argtypes = [ip, i64, i64, dp, i64, vp, dp, i64, dp, i64, dp, i64, ip]
            lib.oracle_backward.argtypes = [ip, i64, i64, dp, i64, vp, dp, i64, dp, i64, dp, i64,
                                            dp, i64, dp, dp, ip]
            lib.oracle_mahalanobis.argtypes = [i64, i64, dp, i64, vp, dp, i64, dp, i64, vp, vp,
                                               dp, ip]
            lib.oracle_max_threads.argtypes = []
            for f in (lib.oracle_tau, lib.oracle_apply, lib.oracle_backward,
                      lib.oracle_mahalanobis, lib.oracle_max_threads):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _sign(sigma, n):
    if sigma is None:
        return None
    s = np.ascontiguousarray(sigma, dtype=np.int8)
    if s.shape != (n,):
        raise ValueError("sign must have shape (n,)")
    return s


def max_threads() -> int:
    """OpenMP threads the oracle uses by default on this host."""
    return int(_load().oracle_max_threads())


def tau(U) -> np.ndarray:
    """tau_k = 2/(v_k^T v_k), 0 for a zero vector (§II-A Eq. (2), §II-B)."""
    U = _f64(np.atleast_2d(U))
    h, n = U.shape
    out = np.zeros(h)
    rc = _load().oracle_tau(n, h, _ptr(U), n, _ptr(out))
    if rc:
        raise ValueError("oracle_tau: invalid argument")
    return out


def apply(mode: str, U, X, sign=None, d=None, threads: int = 0) -> np.ndarray:
    """Per-row transform of X (B x n): mode "W" -> sigma.*(W x), "WT" -> W^T(sigma.*x),
    "SYM" -> sigma.*W(d.*W^T(sigma.*x)), with W = H_1...H_h (Eq. (1), Eq. (21))."""
    X = _f64(np.atleast_2d(X))
    B, n = X.shape
    U = _f64(U).reshape(-1, n)
    h = U.shape[0]
    s = _sign(sign, n)
    dd = None if d is None else _f64(d)
    Y = np.empty_like(X)
    rc = _load().oracle_apply(MODES[mode], n, h, _ptr(U), n, _ptr(s), _ptr(dd), B,
                              _ptr(X), n, _ptr(Y), n, threads)
    if rc:
        raise ValueError("oracle_apply: invalid argument")
    return Y


def backward(mode: str, U, X, gY, sign=None, d=None, threads: int = 0):
    """Gradients of a loss L with dL/dY = gY through ``apply(mode, U, X)``.

    Returns (gX [B x n], gU [h x n], gd [n]); gU and gd are sums over the batch;
    gU is with respect to the reflector vectors exactly as given (unnormalised).
    """
    X = _f64(np.atleast_2d(X))
    B, n = X.shape
    U = _f64(U).reshape(-1, n)
    h = U.shape[0]
    gY = _f64(gY).reshape(B, n)
    s = _sign(sign, n)
    dd = None if d is None else _f64(d)
    gX = np.empty_like(X)
    gU = np.zeros((h, n))
    gd = np.zeros(n)
    rc = _load().oracle_backward(MODES[mode], n, h, _ptr(U), n, _ptr(s), _ptr(dd), B,
                                 _ptr(X), n, _ptr(gY), n, _ptr(gX), n, _ptr(gU), _ptr(gd),
                                 threads)
    if rc:
        raise ValueError("oracle_backward: invalid argument")
    return gX, gU, gd


def mahalanobis(U, X, ia, ib, d, sign=None, threads: int = 0) -> np.ndarray:
    """d_S(x_ia, x_ib) = sum_m d_m [W^T(sigma.*(x_ia - x_ib))]_m^2 per pair (§IV-C)."""
    X = _f64(np.atleast_2d(X))
    N, n = X.shape
    U = _f64(U).reshape(-1, n)
    h = U.shape[0]
    ia = np.ascontiguousarray(ia, dtype=np.int64)
    ib = np.ascontiguousarray(ib, dtype=np.int64)
    if ia.shape != ib.shape or ia.ndim != 1:
        raise ValueError("ia, ib must be equal-length 1-D index arrays")
    if ia.size and (ia.min() < 0 or ib.min() < 0 or ia.max() >= N or ib.max() >= N):
        raise ValueError("pair index out of range")
    s = _sign(sign, n)
    dd = _f64(d)
    out = np.empty(ia.shape[0])
    rc = _load().oracle_mahalanobis(n, h, _ptr(U), n, _ptr(s), _ptr(dd), ia.shape[0],
                                    _ptr(X), n, _ptr(ia), _ptr(ib), _ptr(out), threads)
    if rc:
        raise ValueError("oracle_mahalanobis: invalid argument")
    return out
