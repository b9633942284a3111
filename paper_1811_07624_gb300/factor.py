"""Closed-form approximations of an orthonormal matrix U by a few Householder
reflectors (§II-B to §II-D, Results 1-3), producing plans of the library.

The reflectors come from FP64 eigen- and QR-type computations on the host
(torch on the CPU); the approximation is then a plan, and its error
|U - U_bar|_F^2 is measured by applying the plan to the identity on the GPU.
§II writes U_bar = D U_h ... U_1 (U_1 acts first); a plan computes
W = H_1 ... H_h, so each result also says which apply realises its U_bar:

* Result 1: U_bar_1 = I - 2 sum_k u_k u_k^T, u_k the eigenvectors of
  Z = U + U^T with the most negative eigenvalues (at most n_- of them; the
  rest zero).  The u_k are orthonormal, so the factors commute: apply.
  Error 2n - 2 tr(U) + 2 sum_k z_k (Eq. (6)).
* Result 2: eigenvalues of U by ascending z = 2 Re(lambda) while z < 0: a
  real -1 gives its eigenvector (Case 1); a pair alpha +- i beta gives
  u_1 = sqrt(2) Re(t), u_2 = 2 (gamma Re(t) - delta Im(t)),
  gamma = -sqrt(1 + alpha)/2, delta = -sqrt(1 - alpha)/2, t the unit
  eigenvector of the eigenvalue with positive imaginary part (Case 2, the
  reading under which u_2^T U U_1 u_2 = -1).  U_bar_2 = U_h ... U_1 = W^T:
  apply_T.  With all n_- reflectors the error is 2 n_+ - sum_{k>n_-} z_k
  (Eq. (13)).
* Result 3: the first h Householder reflectors of the QR factorization of U,
  J_k mapping column k (after J_1..J_{k-1}) onto +e_k, and
  D = diag(I_h, D_1) with D_1 the signs of the trailing diagonal; U is
  approximated by J_1 ... J_h D, which is apply_T of the plan of the reversed
  reflectors J_h, ..., J_1 with sign D.  Error 2(n - h) - 2 tr(D_1 U~).  J_k
  has k - 1 leading zeros (§II-D's closing remark): a plan created from these
  reflectors skips each zero prefix (4(n - k + 1) operations per reflector).
"""

from __future__ import annotations

import math

import torch

from .api import Plan


def _f64(U) -> torch.Tensor:
    return torch.as_tensor(U).detach().to("cpu", torch.float64)


def result1(U, h: int):
    """(reflector rows h x n, error of Eq. (6)) for U_bar_1."""
    U = _f64(U)
    n = U.shape[0]
    z, V = torch.linalg.eigh(U + U.t())
    m = min(h, int((z < 0).sum()))
    R = torch.zeros(h, n, dtype=torch.float64)
    R[:m] = V[:, :m].t()
    err = 2 * n - 2 * float(torch.trace(U)) + 2 * float(z[:m].sum())
    return R, err


def result2(U, h: int | None = None):
    """(reflector rows, Eq. (13) error with all n_- reflectors, n_-) for U_bar_2.
    With h given, the first h reflectors of the construction (zero rows beyond)."""
    U = _f64(U)
    n = U.shape[0]
    lam, T = torch.linalg.eig(U)
    tol = 1e-9
    items = []  # (z, rows)
    re, im = lam.real, lam.imag
    minus = [i for i in range(n) if abs(float(im[i])) <= tol and float(re[i]) < 0]
    if minus:
        Q, _ = torch.linalg.qr(T[:, minus].real)
        for j in range(len(minus)):
            items.append((-2.0, [Q[:, j]]))
    for i in range(n):
        a = float(re[i])
        if float(im[i]) > tol and a < 0:
            t = T[:, i] / torch.linalg.norm(T[:, i])
            g, dl = -math.sqrt(1.0 + a) / 2.0, -math.sqrt(1.0 - a) / 2.0
            items.append((2.0 * a, [math.sqrt(2.0) * t.real, 2.0 * (g * t.real - dl * t.imag)]))
    items.sort(key=lambda it: it[0])
    rows = [r for _, rs in items for r in rs]
    z = torch.linalg.eigvalsh(U + U.t())
    n_minus = int((z < 0).sum())
    err_all = 2 * (n - n_minus) - float(z[n_minus:].sum())
    if h is not None:
        rows = rows[:h] + [torch.zeros(n, dtype=torch.float64)] * max(0, h - len(rows))
    R = torch.stack(rows) if rows else torch.zeros(0, n, dtype=torch.float64)
    return R, err_all, n_minus


def result3(U, h: int):
    """(reflector rows j_1..j_h, sign diagonal d, error of the proof of Result 3)."""
    U = _f64(U)
    n = U.shape[0]
    M = U.clone()
    R = torch.zeros(h, n, dtype=torch.float64)
    for k in range(h):
        x = M[:, k].clone()
        x[:k] = 0.0
        x = x / torch.linalg.norm(x)
        x[k] -= 1.0
        nv = float(torch.linalg.norm(x))
        if nv > 1e-14:
            v = x / nv
            R[k] = v
            M = M - 2.0 * torch.outer(v, v @ M)
    d = torch.ones(n, dtype=torch.float64)
    d[h:] = torch.where(torch.diagonal(M)[h:] < 0, -1.0, 1.0)
    err = 2 * (n - h) - 2 * float((d[h:] * torch.diagonal(M)[h:]).sum())
    return R, d, err


def plan(kind: str, R, d=None, device="cuda", dtype=torch.float64):
    """(Plan, mode) whose apply_mode(mode, X) computes U_bar x for each row x."""
    R = _f64(R)
    if kind == "result1":
        return Plan(R.to(device, dtype)), "W"
    if kind == "result2":
        return Plan(R.to(device, dtype)), "WT"
    if kind == "result3":
        return Plan(R.flip(0).contiguous().to(device, dtype),
                    sign=_f64(d).to(device)), "WT"
    raise ValueError(kind)


def error_on_gpu(U, kind: str, R, d=None, device="cuda") -> float:
    """|U - U_bar|_F^2 with U_bar applied to the identity by the plan."""
    Ud = _f64(U).to(device)
    n = Ud.shape[0]
    p, mode = plan(kind, R, d, device)
    with p:
        rows = p.apply_mode(mode, torch.eye(n, device=device, dtype=torch.float64))
    E = Ud - rows.t()   # row i of `rows` is (U_bar e_i)^T
    return float((E * E).sum())
