"""Symmetric Householder Factorization (SHF) and SHF with Spectrum Update
(SHF-SU), §III-B/C and Algorithm 1 of arXiv 1811.07624, in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU leg call it; the
library path never does.  It shares no code with the library's fitting
module and builds every matrix densely (explicit n x n products), so it is
meant for n of a few hundred at most.

Notation follows §III.  The target is a symmetric S with eigenvalues s
(Eq. (15)); the approximation is
    S_bar = D U_1 U_2 ... U_h diag(s_bar) U_h ... U_1 D          (Eq. (16))
with Householder reflectors U_k = I - 2 u_k u_k^T (|u_k| = 1, or u_k = 0 for
U_k = I) and D = diag(d), d in {+1, -1}^n.  Products written with a
descending index range in §III (Eq. (18)-(19)) are read left to right, e.g.
prod_{j=k-1}^{1} U_j = U_{k-1} ... U_1; this is the only reading under which
Eq. (17) holds, and the tests check Eq. (17) numerically.

Readings of points the paper leaves open (each is also listed in the design
notes of the repository):
  * the one-dimensional searches of Eq. (25) and Eq. (27) take the global
    minimiser over the whole range of gamma (a dense grid, then a
    golden-section refinement of the best grid cell); the paper's footnote
    uses a local bounded search started at gamma = 0;
  * D = I while the reflectors are initialised (Algorithm 1, step 2 sets D
    after the reflectors);
  * if u_ddagger is parallel to u_dagger after Eq. (24), u_k^(1) = u_dagger;
  * "until convergence" of Eq. (27): at most `inner` steps, stopping early when
    C decreases by less than inner_tol * max(|C|, 1e-300) in one step;
  * the outer stopping rule compares the relative error of Eq. (32) between
    consecutive iterations: stop when it decreased by less than tol
    ("10e-8", read as 1e-7);
  * the spectrum update of SHF-SU runs after the D update of each iteration;
  * a zero reflector row met in step 3 (possible only with a caller's start)
    is replaced by the Eq. (25) start, descended, only when that gives C < 0.
"""

from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------


def reflector(u) -> np.ndarray:
    """U_k = I - 2 u u^T for a unit u (Eq. (2)); u = 0 gives I."""
    u = np.asarray(u, dtype=np.float64)
    if not np.any(u):
        return np.eye(u.shape[0])
    return np.eye(u.shape[0]) - 2.0 * np.outer(u, u)


def product(U, ks) -> np.ndarray:
    """U_{ks[0]} U_{ks[1]} ... as an explicit matrix (rows of U are u_k)."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    P = np.eye(U.shape[1])
    for k in ks:
        P = P @ reflector(U[k])
    return P


def s_bar_matrix(U, s_bar, d) -> np.ndarray:
    """S_bar of Eq. (16)."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    h = U.shape[0]
    D = np.diag(np.asarray(d, dtype=np.float64))
    W = product(U, range(h))
    return D @ W @ np.diag(np.asarray(s_bar, dtype=np.float64)) @ W.T @ D


def objective(S, U, s_bar, d) -> float:
    """|S - S_bar|_F^2, the quantity Algorithm 1 reduces (Eq. (17))."""
    E = np.asarray(S, dtype=np.float64) - s_bar_matrix(U, s_bar, d)
    return float(np.sum(E * E))


def relative_error(S, S_bar) -> float:
    """Normalised representation error of Eq. (32): |S - S_bar|_F^2 / (4 |S|_F^2)."""
    S = np.asarray(S, dtype=np.float64)
    E = S - np.asarray(S_bar, dtype=np.float64)
    return float(np.sum(E * E) / (4.0 * np.sum(S * S)))


def A_mat(S, U, d, k) -> np.ndarray:
    """A_k of Eq. (18), k 0-based: (U_{k-1} ... U_0) D S D (U_0 ... U_{k-1})."""
    D = np.diag(np.asarray(d, dtype=np.float64))
    P = product(U, range(k))  # U_0 ... U_{k-1}
    return P.T @ D @ np.asarray(S, dtype=np.float64) @ D @ P


def B_mat(U, s_bar, k) -> np.ndarray:
    """B_k of Eq. (19), k 0-based: (U_{k+1} ... U_{h-1}) diag(s_bar) (U_{h-1} ... U_{k+1})."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    P = product(U, range(k + 1, U.shape[0]))
    return P @ np.diag(np.asarray(s_bar, dtype=np.float64)) @ P.T


def C_trace(u, A, B) -> float:
    """C(u) of Eq. (21) exactly as printed, with the trace term formed as a matrix."""
    u = np.asarray(u, dtype=np.float64)
    P = np.outer(u, u)
    return float(u @ (A @ B + B @ A) @ u - 2.0 * np.trace(A @ P @ B @ P))


def C(u, A, B) -> float:
    """C(u) of Eq. (21) with the trace term as the product of two quadratic
    forms (the cyclic-trace identity stated before Eq. (26))."""
    u = np.asarray(u, dtype=np.float64)
    return float(u @ (A @ B + B @ A) @ u - 2.0 * (u @ A @ u) * (u @ B @ u))


def _C_with(M, A, B):
    """C as a function of u for fixed A, B, with M = A B + B A formed once."""
    def f(u):
        return float(u @ M @ u - 2.0 * (u @ A @ u) * (u @ B @ u))
    return f


def grad_C(u, A, B) -> np.ndarray:
    """Gradient of C at u, Eq. (26)."""
    u = np.asarray(u, dtype=np.float64)
    return 2.0 * (A @ B + B @ A) @ u - 4.0 * ((u @ A @ u) * (B @ u) + (u @ B @ u) * (A @ u))


def canonical(u) -> np.ndarray:
    """u and -u give the same reflector; return the one whose entry of largest
    magnitude (lowest index on ties) is positive."""
    u = np.asarray(u, dtype=np.float64)
    i = int(np.argmax(np.abs(u)))
    return -u if u[i] < 0 else u.copy()


# ---------------------------------------------------------------------------
# the two starting directions and the one-dimensional searches (§III-B)
# ---------------------------------------------------------------------------


def u_dagger(A, B) -> np.ndarray:
    """Eigenvector of the smallest eigenvalue of A B + B A (first bullet of §III-B)."""
    M = A @ B + B @ A
    w, V = np.linalg.eigh(0.5 * (M + M.T))
    return V[:, 0].copy()


def u_ddagger(A, B) -> np.ndarray:
    """Second bullet of §III-B: the top eigenvector v of B (x) A is the Kronecker
    product of extreme eigenvectors of B and A (the pair with the largest
    product of eigenvalues), V = v reshaped to n x n is rank one, and u_ddagger
    is the best rank-one approximation of V + V^T: its eigenvector of largest
    eigenvalue magnitude (Eq. (22))."""
    wa, Va = np.linalg.eigh(A)
    wb, Vb = np.linalg.eigh(B)
    best = None
    for ia in (0, -1):
        for ib in (0, -1):
            lam = wa[ia] * wb[ib]
            if best is None or lam > best[0]:
                best = (lam, Va[:, ia], Vb[:, ib])
    _, va, vb = best
    # vec(V) = vb (x) va, i.e. V = va vb^T (column-major vec)
    V = np.outer(va, vb)
    w, E = np.linalg.eigh(V + V.T)
    return E[:, int(np.argmax(np.abs(w)))].copy()


def _search(f, lo, hi, grid=257, iters=100):
    """Global minimiser of f on [lo, hi]: best point of a uniform grid, refined
    by golden-section search inside its neighbouring cells."""
    g = np.linspace(lo, hi, grid)
    vals = np.array([f(x) for x in g])
    i = int(np.argmin(vals))
    a, b = g[max(i - 1, 0)], g[min(i + 1, grid - 1)]
    r = (np.sqrt(5.0) - 1.0) / 2.0
    c, e = b - r * (b - a), a + r * (b - a)
    fc, fe = f(c), f(e)
    for _ in range(iters):
        if b - a < 1e-15:
            break
        if fc < fe:
            b, e, fe = e, c, fc
            c = b - r * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, e, fe
            e = a + r * (b - a)
            fe = f(e)
    cand = [(vals[i], g[i]), (fc, c), (fe, e)]
    return min(cand)[1]


def init_reflector(A, B) -> np.ndarray:
    """u_k^(1) of Eq. (25): u_dagger and u_ddagger made orthonormal (Eq. (24)),
    then the point of the arc (1 - g^2/2) u_dagger +- sqrt(g^2 - g^4/4) u_ddagger,
    g in [0, sqrt 2], with the smallest C."""
    ud = u_dagger(A, B)
    udd = u_ddagger(A, B)
    Cf = _C_with(A @ B + B @ A, A, B)
    udd = udd - (ud @ udd) * ud
    nrm = np.sqrt(udd @ udd)
    if nrm < 1e-12:
        return canonical(ud)
    udd = udd / nrm
    best = None
    for sgn in (1.0, -1.0):
        def f(g, sgn=sgn):
            return Cf((1.0 - g * g / 2.0) * ud + sgn * np.sqrt(max(g * g - g ** 4 / 4.0, 0.0)) * udd)
        g = _search(f, 0.0, np.sqrt(2.0))
        val = f(g)
        if best is None or val < best[0]:
            best = (val, (1.0 - g * g / 2.0) * ud + sgn * np.sqrt(max(g * g - g ** 4 / 4.0, 0.0)) * udd)
    u = best[1]
    return canonical(u / np.sqrt(u @ u))


def descend(u, A, B, inner=20, inner_tol=1e-12):
    """Eq. (27) repeated from u: projected, normalised gradient g, then the point
    (1 - g*^2/2) u - sqrt(g*^2 - g*^4/4) g of smallest C.  Returns u and the
    list of C values (the first is C at the starting u)."""
    u = np.asarray(u, dtype=np.float64).copy()
    Cf = _C_with(A @ B + B @ A, A, B)
    cs = [Cf(u)]
    for _ in range(inner):
        gr = grad_C(u, A, B)
        g = gr - (u @ gr) * u
        ng = np.sqrt(g @ g)
        if ng < 1e-300:
            break
        g = g / ng

        def f(gam):
            return Cf((1.0 - gam * gam / 2.0) * u - np.sqrt(max(gam * gam - gam ** 4 / 4.0, 0.0)) * g)
        gam = _search(f, 0.0, np.sqrt(2.0))
        if f(gam) > cs[-1]:  # the range holds the current point (gamma = 0)
            gam = 0.0
        un = (1.0 - gam * gam / 2.0) * u - np.sqrt(max(gam * gam - gam ** 4 / 4.0, 0.0)) * g
        un = canonical(un / np.sqrt(un @ un))
        cn = Cf(un)
        dec = cs[-1] - cn
        u = un
        cs.append(cn)
        if dec < inner_tol * max(abs(cn), 1e-300):
            break
    return u, cs


def optimal_sign(S, B0) -> np.ndarray:
    """Diagonal of D by Eq. (31): row i of S and of B_0 without their diagonal
    entries; d_i = 1 if |s~_i - b~_i| >= |s~_i + b~_i|, else -1."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    d = np.empty(n)
    for i in range(n):
        keep = np.arange(n) != i
        si, bi = S[i, keep], B0[i, keep]
        d[i] = 1.0 if np.linalg.norm(si - bi) >= np.linalg.norm(si + bi) else -1.0
    return d


def spectrum_update(S, U, d) -> np.ndarray:
    """SHF-SU: s_bar = diag(U_bar^T S U_bar) with U_bar = D U_1 ... U_h (Eq. (33))."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    Ub = np.diag(np.asarray(d, dtype=np.float64)) @ product(U, range(U.shape[0]))
    return np.diag(Ub.T @ np.asarray(S, dtype=np.float64) @ Ub).copy()


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------


def eig_desc(S):
    """Eigenvalues of S in descending order of magnitude and their eigenvectors
    (Eq. (15), step 1 of Algorithm 1)."""
    w, Q = np.linalg.eigh(np.asarray(S, dtype=np.float64))
    order = np.argsort(-np.abs(w), kind="stable")
    return w[order], Q[:, order]


def shf(S, h, K=10, spectrum_update_=False, inner=20, inner_tol=1e-12, tol=1e-7, U0=None,
        s_bar0=None, d0=None, trace=False):
    """Algorithm 1 (SHF), or SHF-SU with spectrum_update_=True.

    U0, s_bar0, d0 replace step 2's initial values when given (U0 rows are the
    reflector vectors; the Result-4 start of §III-D passes them).  Returns a
    dict with U (h x n, unit or zero rows), s_bar, d, the objective after each
    outer iteration ("history", index 0 = after step 2) and, with trace=True,
    the per-reflector C values and objective after every reflector update,
    with the state (U before and after, d, s_bar) each update started from.
    """
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    s, _ = eig_desc(S)
    s_bar = s.copy() if s_bar0 is None else np.asarray(s_bar0, dtype=np.float64).copy()
    d = np.ones(n) if d0 is None else np.asarray(d0, dtype=np.float64).copy()
    U = np.zeros((h, n))
    steps = []
    if U0 is None:
        # step 2: reflectors from zero, each by Eq. (25) given those before it
        for k in range(h):
            A = A_mat(S, U, d, k)
            B = B_mat(U, s_bar, k)
            U[k] = init_reflector(A, B)
        d = optimal_sign(S, B_mat(U, s_bar, -1))
    else:
        U[:] = np.asarray(U0, dtype=np.float64)
    history = [objective(S, U, s_bar, d)]
    rel = [history[0] / (4.0 * np.sum(S * S))]
    for _ in range(K):
        for k in range(h):
            A = A_mat(S, U, d, k)
            B = B_mat(U, s_bar, k)
            before = U.copy()
            if np.any(U[k]):
                u, cs = descend(U[k], A, B, inner=inner, inner_tol=inner_tol)
                U[k] = u
            else:
                # a zero reflector (U_k = I, C = 0) is replaced only by a
                # unit vector that lowers C below zero
                u, cs = descend(init_reflector(A, B), A, B, inner=inner, inner_tol=inner_tol)
                if cs[-1] < 0.0:
                    U[k] = u
                cs = [0.0, min(cs[-1], 0.0)]
            if trace:
                steps.append({"k": k, "C": cs, "objective": objective(S, U, s_bar, d),
                              "U_before": before, "U": U.copy(), "d": d.copy(),
                              "s_bar": s_bar.copy()})
        d = optimal_sign(S, B_mat(U, s_bar, -1))
        if spectrum_update_:
            s_bar = spectrum_update(S, U, d)
        history.append(objective(S, U, s_bar, d))
        rel.append(history[-1] / (4.0 * np.sum(S * S)))
        if rel[-2] - rel[-1] < tol:
            break
    out = {"U": U, "s_bar": s_bar, "d": d, "history": history, "relative_error": rel}
    if trace:
        out["steps"] = steps
    return out


def partial_eig_reflectors(S, h):
    """The reflectors of Result 4's proof (Eq. (29)): J_1 ... J_h bring the h
    eigenvectors of largest |eigenvalue| onto e_1 ... e_h, so that
    J_h ... J_1 S J_1 ... J_h = [[Lambda, 0], [0, S~]]; s_bar = [lambda; diag(S~)].
    Returns (U, s_bar) with U's rows the unit vectors of J_1 ... J_h (a zero
    row where a J_k is not needed).  Under the left-to-right reading,
    S_bar = J_1 ... J_h diag(s_bar) J_h ... J_1."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    lam, Q = eig_desc(S)
    U = np.zeros((h, n))
    P = np.eye(n)  # J_h ... J_1 applied so far, as a matrix acting on vectors
    for k in range(h):
        q = P @ Q[:, k]  # the k-th eigenvector after the earlier reflectors
        # q is zero in entries < k (orthogonal to e_0..e_{k-1}); map it to e_k
        v = q.copy()
        v[k] -= 1.0
        nv = np.sqrt(v @ v)
        if nv > 1e-14:
            U[k] = v / nv
            P = reflector(U[k]) @ P
    T = P @ S @ P.T
    s_bar = np.concatenate([lam[:h], np.diag(T)[h:]])
    return U, s_bar
