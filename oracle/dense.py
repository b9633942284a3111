"""Dense-matrix form of the oracle, for tiny n only.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Builds each reflector
as an explicit n x n matrix I - 2 u u^T (§II-A, Eq. (2), u = v/|v|; the zero
vector gives I), multiplies them in the order W = H_1 H_2 ... H_h, and forms
the sign and symmetric variants of Eq. (1) and Eq. (21) as matrices.  It does
not call the per-vector loops of ``hh_oracle.c``.
"""

from __future__ import annotations

import numpy as np


def reflector(v) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    n = v.shape[0]
    nv = np.sqrt(v @ v)
    if nv == 0.0:
        return np.eye(n)
    u = v / nv
    return np.eye(n) - 2.0 * np.outer(u, u)


def chain(U) -> np.ndarray:
    """W = H_1 H_2 ... H_h as an n x n matrix (rows of U are v_1..v_h)."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    n = U.shape[1]
    W = np.eye(n)
    for v in U:
        W = W @ reflector(v)
    return W


def matrix(mode: str, U, sign=None, d=None) -> np.ndarray:
    """The n x n matrix M with y = M x for ``oracle.apply(mode, ...)``."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    n = U.shape[1]
    W = chain(U)
    D = np.eye(n) if sign is None else np.diag(np.asarray(sign, dtype=np.float64))
    if mode == "W":
        return D @ W
    if mode == "WT":
        return W.T @ D
    if mode == "SYM":
        return D @ W @ np.diag(np.asarray(d, dtype=np.float64)) @ W.T @ D
    raise ValueError(mode)
