"""Fitting S_bar = D U_1 ... U_h diag(s_bar) U_h ... U_1 D to a symmetric target:
SHF and SHF-SU (Algorithm 1, §III-B/C), with every transform of a matrix by
reflectors run on the library's kernels.

For reflector k of a sweep the symmetric matrices of Eq. (18)-(19),
    A_k = P_k^T (D S D) P_k,        P_k = U_1 ... U_{k-1},
    B_k = Q_k diag(s_bar) Q_k^T,    Q_k = U_{k+1} ... U_h,
are formed by plans of the prefix and suffix reflectors applied to the n
columns of D S D and diag(s_bar) (two batched applies each, W^T then W^T for
A_k and W then W for B_k).  The spectrum update of SHF-SU (Eq. (33)) is the
diagonal of W^T D S D W (the same two applies with all h reflectors), the
sign rule of Eq. (31) reads B_0 = W diag(s_bar) W^T, and the objective of
Eq. (17) applies S_bar to the identity with hh_apply_sym.  What is left per
reflector is dense FP64 work on the same device (torch): the eigensolves that
start Eq. (25), the matrix-vector products of C and of its gradient
(Eq. (21), Eq. (26)), and one-dimensional searches over closed forms of C
along the arcs of Eq. (25) and Eq. (27).

The arcs are parametrised by an angle: with p, q orthonormal,
(1 - g^2/2) p + sqrt(g^2 - g^4/4) q = cos(t) p + sin(t) q for g = 2 sin(t/2),
so g in [0, sqrt 2] is t in [0, pi/2] (and the +- of Eq. (25) is t in
[-pi/2, pi/2]).  Along the arc each quadratic form is
cos^2 t (p'Xp) + 2 sin t cos t (p'Xq) + sin^2 t (q'Xq), so C(t) is a
trigonometric polynomial whose global minimum over the range is found from
nine scalars: a grid of 4097 angles, then golden-section refinement.

Readings where the paper is open (the same as the FP64 reference the tests
compare with): each search takes the global minimiser over its whole range
(the paper's footnote uses a local search from g = 0); D = I while the
reflectors are initialised; u_ddagger parallel to u_dagger gives
u^(1) = u_dagger; Eq. (27) runs at most `inner` steps and stops early when C
falls by less than inner_tol * |C| in a step; the outer loop stops when the
relative error of Eq. (32) falls by less than tol between iterations; the
spectrum update follows the D update; a zero reflector is replaced only by a
start that, descended, gives C < 0; u and -u being the same reflector, every
updated u has its largest-magnitude entry positive.
"""

from __future__ import annotations

import math

import numpy as np
import torch

from .api import Plan

_GRID = 4097
_GOLDEN = 80


def _two_sided_T(U: torch.Tensor, M: torch.Tensor) -> torch.Tensor:
    """P^T M P for symmetric M and P = U_1 ... U_m (rows of U), on the kernels."""
    if U.shape[0] == 0:
        return M.clone()
    with Plan(U) as p:
        R = p.apply_T(M)                       # row j: P^T m_j, i.e. R = M P
        return p.apply_T(R.t().contiguous())   # row i: P^T (M P e_i)


def _two_sided(U: torch.Tensor, M: torch.Tensor) -> torch.Tensor:
    """P M P^T for symmetric M and P = U_1 ... U_m, on the kernels."""
    if U.shape[0] == 0:
        return M.clone()
    with Plan(U) as p:
        R = p.apply(M)                         # row j: P m_j, i.e. R = M P^T
        return p.apply(R.t().contiguous())     # row i: P (M P^T e_i)


def _canonical(u: torch.Tensor) -> torch.Tensor:
    i = int(torch.argmax(u.abs()))
    return -u if float(u[i]) < 0 else u


class _Forms:
    """C along the arc cos(t) p + sin(t) q, from the quadratic forms of
    M = A B + B A, A and B on (p, q)."""

    def __init__(self, A, B, p, q):
        Ap, Aq, Bp, Bq = A @ p, A @ q, B @ p, B @ q
        # p'Mp = 2 (Ap).(Bp); p'Mq = (Ap).(Bq) + (Bp).(Aq); q'Mq = 2 (Aq).(Bq)
        vals = torch.stack([2 * (Ap @ Bp), Ap @ Bq + Bp @ Aq, 2 * (Aq @ Bq),
                            p @ Ap, p @ Aq, q @ Aq, p @ Bp, p @ Bq, q @ Bq]).tolist()
        self.m, self.a, self.b = vals[0:3], vals[3:6], vals[6:9]

    @staticmethod
    def _quad(f, c, s):
        return c * c * f[0] + 2 * s * c * f[1] + s * s * f[2]

    def C(self, t: float) -> float:
        c, s = math.cos(t), math.sin(t)
        return self._quad(self.m, c, s) - 2.0 * self._quad(self.a, c, s) * self._quad(self.b, c, s)

    def argmin(self, lo: float, hi: float) -> float:
        # the grid in one vectorised evaluation on the host, then golden section
        ts = np.linspace(lo, hi, _GRID)
        c, s = np.cos(ts), np.sin(ts)

        def quad(f):
            return c * c * f[0] + 2 * s * c * f[1] + s * s * f[2]
        vals = quad(self.m) - 2.0 * quad(self.a) * quad(self.b)
        i = int(np.argmin(vals))
        best_t, best = float(ts[i]), float(vals[i])
        step = (hi - lo) / (_GRID - 1)
        a, b = max(lo, best_t - step), min(hi, best_t + step)
        r = (math.sqrt(5.0) - 1.0) / 2.0
        c, e = b - r * (b - a), a + r * (b - a)
        fc, fe = self.C(c), self.C(e)
        for _ in range(_GOLDEN):
            if fc < fe:
                b, e, fe = e, c, fc
                c = b - r * (b - a)
                fc = self.C(c)
            else:
                a, c, fc = c, e, fe
                e = a + r * (b - a)
                fe = self.C(e)
        for t, v in ((c, fc), (e, fe)):
            if v < best:
                best_t, best = t, v
        return best_t


def C_value(u, A, B) -> float:
    """C(u) of Eq. (21): u'(AB + BA)u - 2 (u'Au)(u'Bu)."""
    Au, Bu = A @ u, B @ u
    return float(2 * (Au @ Bu) - 2 * (u @ Au) * (u @ Bu))


def C_grad(u, A, B) -> torch.Tensor:
    """Eq. (26): 2 (AB + BA) u - 4 ((u'Au) B + (u'Bu) A) u."""
    Au, Bu = A @ u, B @ u
    return 2 * (A @ Bu + B @ Au) - 4 * ((u @ Au) * Bu + (u @ Bu) * Au)


def start_reflector(A, B) -> torch.Tensor:
    """u^(1) of Eq. (25) from u_dagger (smallest eigenvector of AB + BA) and
    u_ddagger (dominant eigenvector of V + V^T, V = a b^T for the extreme
    eigenvectors a of A and b of B whose eigenvalue product is largest)."""
    M = A @ B + B @ A
    _, E = torch.linalg.eigh(0.5 * (M + M.t()))
    ud = E[:, 0]
    wa, Ea = torch.linalg.eigh(A)
    wb, Eb = torch.linalg.eigh(B)
    best = None
    for ia in (0, -1):
        for ib in (0, -1):
            lam = float(wa[ia] * wb[ib])
            if best is None or lam > best[0]:
                best = (lam, Ea[:, ia], Eb[:, ib])
    a, b = best[1], best[2]
    # V + V^T = a b^T + b a^T has eigenvalues a.b +- 1 on (a +- b) / |a +- b|
    c = float(a @ b)
    udd = a + (1.0 if c >= 0 else -1.0) * b
    udd = udd / torch.linalg.norm(udd)
    udd = udd - (ud @ udd) * ud
    nrm = float(torch.linalg.norm(udd))
    if nrm < 1e-12:
        return _canonical(ud)
    udd = udd / nrm
    f = _Forms(A, B, ud, udd)
    t = f.argmin(-math.pi / 2, math.pi / 2)
    u = math.cos(t) * ud + math.sin(t) * udd
    return _canonical(u / torch.linalg.norm(u))


def descend(u, A, B, inner=20, inner_tol=1e-12):
    """Eq. (27) from u; returns u and the C values (the first at the start)."""
    cs = [C_value(u, A, B)]
    for _ in range(inner):
        g = C_grad(u, A, B)
        g = g - (u @ g) * u
        ng = float(torch.linalg.norm(g))
        if ng < 1e-300:
            break
        q = -g / ng
        f = _Forms(A, B, u, q)
        t = f.argmin(0.0, math.pi / 2)
        if f.C(t) > cs[-1]:
            t = 0.0
        un = math.cos(t) * u + math.sin(t) * q
        un = _canonical(un / torch.linalg.norm(un))
        cn = C_value(un, A, B)
        dec = cs[-1] - cn
        u = un
        cs.append(cn)
        if dec < inner_tol * max(abs(cn), 1e-300):
            break
    return u, cs


class SHF:
    """State of Algorithm 1 on one device: S (n x n, float64, symmetric), the
    reflector rows U (h x n), the spectrum s_bar and the sign diagonal d."""

    def __init__(self, S: torch.Tensor, h: int, U0=None, s_bar0=None, d0=None):
        if S.dim() != 2 or S.shape[0] != S.shape[1]:
            raise ValueError("S must be square")
        if not S.is_cuda:
            raise ValueError("S must be a CUDA tensor")
        self.S = S.to(torch.float64).contiguous()
        self.n, self.h = S.shape[0], int(h)
        dev = self.S.device
        w = torch.linalg.eigvalsh(self.S)
        self.s = w[torch.argsort(-w.abs(), stable=True)]
        self.s_bar = self.s.clone() if s_bar0 is None else s_bar0.to(dev, torch.float64).clone()
        self.d = torch.ones(self.n, device=dev, dtype=torch.float64) if d0 is None else \
            d0.to(dev, torch.float64).clone()
        self.U = torch.zeros(self.h, self.n, device=dev, dtype=torch.float64)
        self.norm_S2 = float((self.S * self.S).sum())
        if U0 is None:
            for k in range(self.h):
                A, B = self.A(k), self.B(k)
                self.U[k] = start_reflector(A, B)
            self.d = self.optimal_sign()
        else:
            self.U.copy_(U0.to(dev, torch.float64))

    # --- the matrices of §III-B, through the kernels ---------------------------------
    def DSD(self):
        return self.d[:, None] * self.S * self.d[None, :]

    def A(self, k):
        """A_k of Eq. (18), k 0-based: reflectors 0..k-1 applied on both sides of D S D."""
        return _two_sided_T(self.U[:k].contiguous(), self.DSD())

    def B(self, k):
        """B_k of Eq. (19), k 0-based: reflectors k+1..h-1 on both sides of diag(s_bar);
        k = -1 gives B_0 = W diag(s_bar) W^T."""
        return _two_sided(self.U[k + 1:].contiguous(), torch.diag(self.s_bar))

    def optimal_sign(self):
        """Eq. (31) against B_0."""
        B0 = self.B(-1)
        off = 1.0 - torch.eye(self.n, device=self.S.device, dtype=torch.float64)
        minus = torch.linalg.norm((self.S - B0) * off, dim=1)
        plus = torch.linalg.norm((self.S + B0) * off, dim=1)
        return torch.where(minus >= plus, 1.0, -1.0).to(torch.float64)

    def spectrum_update(self):
        """Eq. (33): the diagonal of W^T D S D W."""
        return torch.diagonal(_two_sided_T(self.U.contiguous(), self.DSD())).clone()

    def S_bar(self):
        """S_bar of Eq. (16) as a matrix: hh_apply_sym on the identity."""
        eye = torch.eye(self.n, device=self.S.device, dtype=torch.float64)
        with Plan(self.U, d=self.s_bar, sign=self.d) as p:
            return p.apply_sym(eye)

    def objective(self):
        E = self.S - self.S_bar()
        return float((E * E).sum())

    # --- Algorithm 1, step 3 ---------------------------------------------------------
    def iterate(self, spectrum_update=False, inner=20, inner_tol=1e-12, trace=None):
        """One outer iteration: every reflector by Eq. (27), then D by Eq. (31)
        and, for SHF-SU, s_bar by Eq. (33)."""
        for k in range(self.h):
            A, B = self.A(k), self.B(k)
            if bool((self.U[k] != 0).any()):
                u, cs = descend(self.U[k].clone(), A, B, inner, inner_tol)
                self.U[k] = u
            else:
                u, cs = descend(start_reflector(A, B), A, B, inner, inner_tol)
                if cs[-1] < 0.0:
                    self.U[k] = u
            if trace is not None:
                trace.append({"k": k, "C": cs})
        self.d = self.optimal_sign()
        if spectrum_update:
            self.s_bar = self.spectrum_update()


def shf(S: torch.Tensor, h: int, K: int = 10, spectrum_update: bool = False, inner: int = 20,
        inner_tol: float = 1e-12, tol: float = 1e-7, U0=None, s_bar0=None, d0=None):
    """Run Algorithm 1 (SHF, or SHF-SU with spectrum_update=True) on a CUDA
    float64 symmetric S.  Returns a dict: U (h x n rows u_k), s_bar, d, and the
    objective |S - S_bar|_F^2 and relative error (Eq. (32)) after step 2 and
    after each outer iteration."""
    st = SHF(S, h, U0=U0, s_bar0=s_bar0, d0=d0)
    hist = [st.objective()]
    rel = [hist[0] / (4.0 * st.norm_S2)]
    for _ in range(K):
        st.iterate(spectrum_update, inner, inner_tol)
        hist.append(st.objective())
        rel.append(hist[-1] / (4.0 * st.norm_S2))
        if rel[-2] - rel[-1] < tol:
            break
    return {"U": st.U, "s_bar": st.s_bar, "d": st.d, "history": hist, "relative_error": rel,
            "state": st}
