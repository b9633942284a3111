"""Closed-form approximations of an orthonormal U by a few reflectors (§II-B,
§II-C, §II-D of arXiv 1811.07624), in plain FP64 numpy with dense matrices.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``); shares no code with
the library's factorization module.

Conventions.  §II writes U_bar = D U_h ... U_1 (Eq. (1)), so U_1 acts first
on a vector.  Reflector matrices are I - 2 u u^T with unit u (zero u: I).

* Result 1 (Eq. (4)-(6)): U_bar_1 = I - 2 sum_k u_k u_k^T with u_k the
  eigenvectors of Z = U + U^T for its most negative eigenvalues (at most n_-
  of them; further reflectors are zero).  Error 2n - 2 tr(U) + 2 sum_k z_k.
* Result 2 (Eq. (8)-(13)): from the eigendecomposition of U, eigenvalues
  taken by ascending z = 2 Re(lambda) while z < 0: a real eigenvalue -1
  gives one reflector, its eigenvector (Case 1); a conjugate pair
  alpha +- i beta gives two, u_1 = sqrt(2) Re(t) and
  u_2 = 2 (gamma Re(t) - delta Im(t)), gamma = -sqrt(1 + alpha)/2,
  delta = -sqrt(1 - alpha)/2 (Case 2).  Reading: t is the unit eigenvector
  of the eigenvalue with positive imaginary part (with the conjugate one the
  printed gamma, delta do not give u_2^T U U_1 u_2 = -1).  With all n_-
  reflectors the error is 2 n_+ - sum_{k > n_-} z_k (Eq. (13)).
* Result 3 (Eq. (14)-(16)): the first h Householder reflectors J_k of the QR
  factorization of U, each mapping the k-th column (after J_1..J_{k-1}) onto
  +e_k, and D = diag(I_h, D_1) with D_1 making the trailing block's diagonal
  positive; U is approximated by J_1 ... J_h D, error 2(n - h) - 2 tr(D_1 U~).
  j_k has k - 1 leading zeros (the sparse reflectors of §II-D's last remark).
"""

from __future__ import annotations

import numpy as np


def reflector(u) -> np.ndarray:
    u = np.asarray(u, dtype=np.float64)
    if not np.any(u):
        return np.eye(u.shape[0])
    return np.eye(u.shape[0]) - 2.0 * np.outer(u, u)


def product_first_acts_first(U) -> np.ndarray:
    """U_h ... U_1 for the rows u_1..u_h of U (Eq. (1) without D)."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    P = np.eye(U.shape[1])
    for u in U:
        P = reflector(u) @ P
    return P


def frob2(A) -> float:
    return float(np.sum(np.asarray(A) ** 2))


# --- Result 1 ----------------------------------------------------------------------


def result1(U, h):
    """Reflector rows (h x n) of U_bar_1 and the error formula of Eq. (6)."""
    U = np.asarray(U, dtype=np.float64)
    n = U.shape[0]
    z, V = np.linalg.eigh(U + U.T)  # ascending
    R = np.zeros((h, n))
    m = min(h, int(np.sum(z < 0)))
    for k in range(m):
        R[k] = V[:, k]
    err = 2 * n - 2 * np.trace(U) + 2 * np.sum(z[:m])
    return R, float(err)


def result1_matrix(R) -> np.ndarray:
    """I - 2 sum_k u_k u_k^T (Eq. (4))."""
    R = np.atleast_2d(np.asarray(R, dtype=np.float64))
    return np.eye(R.shape[1]) - 2.0 * R.T @ R


# --- Result 2 ----------------------------------------------------------------------


def result2(U, h=None):
    """Reflector rows of U_bar_2 = U_h ... U_1 by Cases 1 and 2, at most h of
    them (all n_- when h is None), and the Eq. (13) error for all n_-."""
    U = np.asarray(U, dtype=np.float64)
    n = U.shape[0]
    lam, T = np.linalg.eig(U)
    tol = 1e-9
    groups = []  # (z, kind, vectors)
    minus = [i for i in range(n) if abs(lam[i].imag) <= tol and lam[i].real < 0]
    if minus:
        # eigenvectors of a repeated -1 made orthonormal (footnote of §II-C)
        Q, _ = np.linalg.qr(np.real(T[:, minus]))
        for j in range(len(minus)):
            groups.append((-2.0, "case1", Q[:, j]))
    for i in range(n):
        if lam[i].imag > tol and lam[i].real < 0:
            groups.append((2 * lam[i].real, "case2", (lam[i].real, T[:, i])))
    groups.sort(key=lambda g: g[0])
    rows = []
    for _, kind, data in groups:
        if kind == "case1":
            rows.append(data)
        else:
            a, t = data
            t = t / np.linalg.norm(t)
            rows.append(np.sqrt(2.0) * t.real)
            gamma, delta = -np.sqrt(1.0 + a) / 2.0, -np.sqrt(1.0 - a) / 2.0
            rows.append(2.0 * (gamma * t.real - delta * t.imag))
    z = np.sort(np.linalg.eigvalsh(U + U.T))
    n_minus = int(np.sum(z < 0))
    err_all = 2 * (n - n_minus) - float(np.sum(z[n_minus:]))
    if h is not None:
        rows = rows[:h] + [np.zeros(n)] * max(0, h - len(rows))
    R = np.array(rows).reshape(len(rows), n)
    return R, err_all, n_minus


# --- Result 3 ----------------------------------------------------------------------


def result3(U, h):
    """Reflector rows j_1..j_h of the partial QR of U (Eq. (14)), the sign
    diagonal D, the trailing block D_1 U~ and the error of the proof."""
    U = np.asarray(U, dtype=np.float64)
    n = U.shape[0]
    R = np.zeros((h, n))
    M = U.copy()  # J_k ... J_1 U
    for k in range(h):
        x = M[:, k].copy()
        x[:k] = 0.0
        x /= np.linalg.norm(x)
        v = x.copy()
        v[k] -= 1.0
        nv = np.linalg.norm(v)
        if nv > 1e-14:
            R[k] = v / nv
            M = reflector(R[k]) @ M
    d = np.ones(n)
    tail = np.diag(M)[h:]
    d[h:] = np.where(tail < 0, -1.0, 1.0)
    block = (d[:, None] * M)[h:, h:]
    err = 2 * (n - h) - 2 * float(np.trace(block))
    return R, d, M, err


def result3_matrix(R, d) -> np.ndarray:
    """J_1 ... J_h D (the approximation of Result 3)."""
    R = np.atleast_2d(np.asarray(R, dtype=np.float64))
    P = np.eye(R.shape[1])
    for u in R:
        P = P @ reflector(u)
    return P @ np.diag(np.asarray(d, dtype=np.float64))


def result3_bound(n, h) -> float:
    """Right-hand side of Eq. (14): 2(n - h) - (2 sqrt 2 / sqrt pi) sqrt(n - h)."""
    return 2.0 * (n - h) - 2.0 * np.sqrt(2.0) / np.sqrt(np.pi) * np.sqrt(n - h)


def representation_error(X, Xbar) -> float:
    """Eq. (32): |X - Xbar|_F^2 / (4 |X|_F^2)."""
    return frob2(np.asarray(X) - np.asarray(Xbar)) / (4.0 * frob2(X))
