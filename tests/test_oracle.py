"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: hand-worked closed
forms (tests/golden/), LAPACK's Householder QR, the paper's completeness claim,
determinant and orthonormality facts, a dense-matrix product written
separately, central finite differences, and the paper's own gradient formula.
"""

import numpy as np
import pytest

import oracle
from oracle import dense
import synthetic_inputs as si
from golden_cases import load_closed_forms

RTOL64 = 1e-12


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# --- closed forms (§II-A Eq. (2); swaps and sign flips are exact) -------------

def test_golden_closed_forms_bit_exact():
    cases = load_closed_forms()
    for name, c in cases.items():
        U, x = c["U"], c["x"][None, :]
        assert np.array_equal(oracle.apply("W", U, x)[0], c["W"]), name
        assert np.array_equal(oracle.apply("WT", U, x)[0], c["WT"]), name
        if "sign" in c:
            s = c["sign"].astype(np.int8)
            assert np.array_equal(oracle.apply("W", U, x, sign=s)[0], c["W_sign"]), name
            assert np.array_equal(oracle.apply("WT", U, x, sign=s)[0], c["WT_sign"]), name
        if "d" in c:
            assert np.array_equal(oracle.apply("SYM", U, x, d=c["d"])[0], c["SYM"]), name


def test_single_reflector_closed_form():
    # h = 1: y = x - 2 u (u^T x), u = v/|v|  (Eq. (2))
    n = 17
    v = si.reflectors(n, 1, seed=3, unit=False)[0] * 3.7
    X = si.vectors(5, n, seed=3)
    u = v / np.linalg.norm(v)
    expect = X - 2.0 * np.outer(X @ u, u)
    assert rel(oracle.apply("W", v[None], X), expect) < RTOL64
    assert rel(oracle.apply("WT", v[None], X), expect) < RTOL64


def test_permutation_chain_exact():
    # a chain of transpositions e_i - e_j is the composed permutation, exactly
    rng = np.random.default_rng(7)
    n, h = 12, 9
    pairs = [tuple(rng.choice(n, 2, replace=False)) for _ in range(h)]
    U = np.zeros((h, n))
    for k, (i, j) in enumerate(pairs):
        U[k, i], U[k, j] = 1.0, -1.0
    x = rng.integers(-50, 50, size=(3, n)).astype(np.float64)
    y = x.copy()
    for (i, j) in reversed(pairs):  # H_h first
        y[:, [i, j]] = y[:, [j, i]]
    assert np.array_equal(oracle.apply("W", U, x), y)


def test_zero_reflector_is_identity():
    # u_k = 0 gives U_k = I (Result 1, §II-B)
    n = 9
    U = si.reflectors(n, 3, seed=1)
    U0 = np.vstack([U[:1], np.zeros(n), U[1:]])
    X = si.vectors(4, n, seed=1)
    assert np.array_equal(oracle.tau(np.zeros((1, n))), [0.0])
    for mode in ("W", "WT"):
        assert rel(oracle.apply(mode, U0, X), oracle.apply(mode, U, X)) < RTOL64
    assert np.array_equal(oracle.apply("W", np.zeros((2, n)), X), X)


# --- involution and orthonormality (§II-A: H_k symmetric, orthonormal) ---------

def test_involution():
    n = 33
    v = si.reflectors(n, 1, seed=11, unit=False)
    X = si.vectors(6, n, seed=11)
    twice = np.vstack([v, v])
    assert rel(oracle.apply("W", twice, X), X) < 1e-14


@pytest.mark.parametrize("n,h", [(8, 3), (64, 8), (100, 40)])
def test_orthonormal_norm_and_inverse(n, h):
    U = si.reflectors(n, h, seed=n + h, unit=False)
    X = si.vectors(16, n, seed=n)
    s = si.sign(n, seed=n)
    Y = oracle.apply("W", U, X, sign=s)
    assert np.max(np.abs(np.linalg.norm(Y, axis=1) / np.linalg.norm(X, axis=1) - 1)) < 1e-13
    # W^T(sigma .* (sigma .* W x)) = x
    back = oracle.apply("WT", U, Y, sign=s)
    assert rel(back, X) < 1e-13


def test_determinant():
    # det(H_k) = -1, so det W = (-1)^(#non-zero reflectors)  (§II-A)
    n = 10
    for h in range(0, 6):
        U = si.reflectors(n, h, seed=h)
        if h >= 2:
            U[1] = 0.0  # one identity factor
        nz = int(sum(np.any(U != 0, axis=1))) if h else 0
        M = oracle.apply("W", U, np.eye(n)).T  # columns W e_j
        sgn, logdet = np.linalg.slogdet(M)
        assert sgn == (-1) ** nz and abs(logdet) < 1e-12


# --- LAPACK's Householder QR pins the product order and tau ---------------------

def _lapack_reflectors(A):
    hT, tau_l = np.linalg.qr(A, mode="raw")
    Hm = hT.T
    n = A.shape[0]
    V = np.zeros((n, n))
    for i in range(n):
        if tau_l[i] != 0.0:
            V[i, i] = 1.0
            V[i, i + 1:] = Hm[i + 1:, i]
    return V, tau_l


def test_lapack_qr_product_order():
    # LAPACK stores Q = H(1) H(2) ... H(k), H(i) = I - tau_i v_i v_i^T; the oracle's
    # W = H_1 ... H_h must equal it, and tau_i = 2 / |v_i|^2.
    n = 12
    A = si.vectors(n, n, seed=5)
    V, tau_l = _lapack_reflectors(A)
    nz = tau_l != 0
    assert np.allclose(oracle.tau(V)[nz], tau_l[nz], rtol=1e-13, atol=0)
    Q = np.linalg.qr(A, mode="complete")[0]
    W = oracle.apply("W", V, np.eye(n)).T
    assert np.max(np.abs(W - Q)) < 1e-13
    WT = oracle.apply("WT", V, np.eye(n)).T
    assert np.max(np.abs(WT - Q.T)) < 1e-13


def test_completeness_any_orthonormal():
    # Every orthonormal matrix is n-1 reflectors and a +-1 diagonal (§I, §II-A, Result 3).
    n = 11
    Uo = si.random_orthonormal(n, seed=2)
    V, tau_l = _lapack_reflectors(Uo.T)  # U^T = J_1 ... J_n R, R = diag(+-1)
    R = np.linalg.qr(Uo.T, mode="complete")[1]
    sgn = np.sign(np.diag(R)).astype(np.int8)
    assert np.allclose(np.abs(np.diag(R)), 1.0, atol=1e-12)
    assert int(np.sum(tau_l != 0)) <= n - 1 or np.sum(np.any(V != 0, axis=1)) <= n
    # U = R^T J_n ... J_1 = D (chain over the reversed list)
    M = oracle.apply("W", V[::-1], np.eye(n), sign=sgn).T
    assert np.max(np.abs(M - Uo)) < 1e-13


# --- dense brute force on tiny n ----------------------------------------------

@pytest.mark.parametrize("mode", ["W", "WT", "SYM"])
def test_dense_product(mode):
    n, h = 7, 4
    U = si.reflectors(n, h, seed=21, unit=False)
    s = si.sign(n, seed=21)
    d = si.spectrum(n, seed=21)
    X = si.vectors(9, n, seed=21)
    M = dense.matrix(mode, U, sign=s, d=d)
    assert rel(oracle.apply(mode, U, X, sign=s, d=d), X @ M.T) < RTOL64


def test_orthonormal_reflectors_sum_form():
    # orthonormal u_k: W = I - 2 sum u_k u_k^T, independent of order (Result 1, §II-B)
    n, h = 20, 5
    Q = si.random_orthonormal(n, seed=4)[:, :h].T
    X = si.vectors(4, n, seed=4)
    expect = X - 2.0 * (X @ Q.T) @ Q
    assert rel(oracle.apply("W", Q, X), expect) < RTOL64
    assert rel(oracle.apply("W", Q[::-1], X), expect) < RTOL64


# --- symmetric form (§III-A, Eq. (21)) ------------------------------------------

def test_symmetric_properties():
    n, h = 16, 5
    U = si.reflectors(n, h, seed=8)
    d = si.spectrum(n, seed=8)
    s = si.sign(n, seed=8)
    X = si.vectors(2, n, seed=8)
    S1 = oracle.apply("SYM", U, X, sign=s, d=d)
    # <S x, y> = <x, S y>
    assert abs(S1[0] @ X[1] - X[0] @ S1[1]) < 1e-12 * np.linalg.norm(S1[0]) * np.linalg.norm(X[1])
    # W e_i is an eigenvector with eigenvalue d_i (sign = +1)
    E = oracle.apply("W", U, np.eye(n))  # rows W e_i
    SE = oracle.apply("SYM", U, E, d=d)
    assert rel(SE, d[:, None] * E) < 1e-13
    # W = I gives diag(d) (with the sign squared away)
    assert rel(oracle.apply("SYM", np.zeros((2, n)), X, sign=s, d=d), X * d) < 1e-15
    # positive spectrum -> positive definite
    q = np.einsum("bi,bi->b", X, oracle.apply("SYM", U, X, d=d))
    assert np.all(q > 0)


# --- gradients --------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["W", "WT", "SYM"])
def test_backward_central_differences(mode):
    n, h, B = 6, 3, 2
    U = si.reflectors(n, h, seed=31, unit=False)
    s = si.sign(n, seed=31)
    d = si.spectrum(n, seed=31)
    X = si.vectors(B, n, seed=31)
    G = si.vectors(B, n, seed=32)
    gX, gU, gd = oracle.backward(mode, U, X, G, sign=s, d=d)

    def f(U_, X_, d_):
        return float(np.sum(G * oracle.apply(mode, U_, X_, sign=s, d=d_)))

    eps = 1e-6
    num_U = np.zeros_like(U)
    for idx in np.ndindex(U.shape):
        Up, Um = U.copy(), U.copy()
        Up[idx] += eps
        Um[idx] -= eps
        num_U[idx] = (f(Up, X, d) - f(Um, X, d)) / (2 * eps)
    num_X = np.zeros_like(X)
    for idx in np.ndindex(X.shape):
        Xp, Xm = X.copy(), X.copy()
        Xp[idx] += eps
        Xm[idx] -= eps
        num_X[idx] = (f(U, Xp, d) - f(U, Xm, d)) / (2 * eps)
    assert rel(gU, num_U) < 1e-7
    assert rel(gX, num_X) < 1e-7
    if mode == "SYM":
        num_d = np.zeros_like(d)
        for i in range(n):
            dp, dm = d.copy(), d.copy()
            dp[i] += eps
            dm[i] -= eps
            num_d[i] = (f(U, X, dp) - f(U, X, dm)) / (2 * eps)
        assert rel(gd, num_d) < 1e-7
    else:
        assert np.all(gd == 0)


def test_backward_matches_paper_gradient():
    # §III-B: with A_k, B_k of Eqs. (23)-(24), |S - Sbar|_F^2 = const + 4 C(u_k) on the
    # unit sphere (Eq. (25)), with grad C of Eq. (33).  So the tangential gradient of
    # the Frobenius objective w.r.t. u_k is 4 (I - u u^T) grad C(u_k).
    n, h = 6, 3
    U = si.reflectors(n, h, seed=41)  # unit rows
    sbar = si.spectrum(n, seed=41)
    Xs = si.vectors(n, n, seed=42)
    S = 0.5 * (Xs + Xs.T)
    I = np.eye(n)
    Sbar = oracle.apply("SYM", U, I, d=sbar)  # rows S e_i = columns (symmetric)
    gY = 2.0 * (Sbar - S)
    _, gU, _ = oracle.backward("SYM", U, I, gY, d=sbar)
    H = [dense.reflector(v) for v in U]
    for k in range(h):
        Ak = S.copy()
        for j in range(k):  # A_k = U_{k-1}...U_1 S U_1...U_{k-1}
            Ak = H[j] @ Ak @ H[j]
        Bk = np.diag(sbar)
        for j in range(h - 1, k, -1):  # B_k = U_{k+1}...U_h diag U_h...U_{k+1}
            Bk = H[j] @ Bk @ H[j]
        u = U[k]
        gradC = 2 * (Ak @ Bk + Bk @ Ak) @ u - 4 * ((u @ Ak @ u) * Bk + (u @ Bk @ u) * Ak) @ u
        paper = 4 * (np.eye(n) - np.outer(u, u)) @ gradC
        assert np.max(np.abs(gU[k] - paper)) < 1e-11 * max(1.0, np.max(np.abs(paper)))


# --- fast Mahalanobis distance (§IV-C) ------------------------------------------

def test_mahalanobis_matches_quadratic_form():
    n, h, N = 10, 4, 7
    U = si.reflectors(n, h, seed=51)
    d = si.spectrum(n, seed=51)
    s = si.sign(n, seed=51)
    X = si.vectors(N, n, seed=51)
    ia = np.array([0, 1, 2, 6, 3, 3])
    ib = np.array([1, 2, 0, 5, 4, 3])
    out = oracle.mahalanobis(U, X, ia, ib, d, sign=s)
    M = dense.matrix("SYM", U, sign=s, d=d)
    delta = X[ia] - X[ib]
    expect = np.einsum("pi,ij,pj->p", delta, M, delta)
    assert rel(out, expect) < RTOL64
    assert out[-1] == 0.0
    # W = I: sum d_i delta_i^2
    out0 = oracle.mahalanobis(np.zeros((h, n)), X, ia, ib, d)
    assert rel(out0, (delta ** 2) @ d) < 1e-15


def test_mahalanobis_gradient_composition_central_differences():
    # The gradient reference of the GPU tests for the distance of §IV-C: with
    # z_p = W^T(sigma .* delta_p) and L = sum_p g_p sum_m d_m z_pm^2,
    # dL/dd = sum_p g_p z_p .* z_p and dL/dU is the W^T adjoint seeded with
    # 2 g_p d .* z_p.  Pinned here against central differences of the distance.
    n, h = 6, 3
    U = si.reflectors(n, h, seed=61, unit=False)
    d = si.spectrum(n, seed=61)
    s = si.sign(n, seed=61)
    X = si.vectors(5, n, seed=61)
    ia, ib = np.array([0, 1, 2, 4]), np.array([1, 3, 0, 2])
    g = np.random.default_rng(61).standard_normal(ia.shape[0])
    delta = X[ia] - X[ib]
    z = oracle.apply("WT", U, delta, sign=s)
    gd_ref = (g[:, None] * z * z).sum(axis=0)
    _, gU_ref, _ = oracle.backward("WT", U, delta, 2.0 * g[:, None] * d[None, :] * z, sign=s)

    def f(U_, d_):
        return float(g @ oracle.mahalanobis(U_, X, ia, ib, d_, sign=s))

    eps = 1e-6
    num_U = np.zeros_like(U)
    for idx in np.ndindex(U.shape):
        Up, Um = U.copy(), U.copy()
        Up[idx] += eps
        Um[idx] -= eps
        num_U[idx] = (f(Up, d) - f(Um, d)) / (2 * eps)
    num_d = np.zeros_like(d)
    for i in range(n):
        dp, dm = d.copy(), d.copy()
        dp[i] += eps
        dm[i] -= eps
        num_d[i] = (f(U, dp) - f(U, dm)) / (2 * eps)
    assert rel(gU_ref, num_U) < 1e-7
    assert rel(gd_ref, num_d) < 1e-7


def test_invalid_arguments():
    with pytest.raises(ValueError):
        oracle.apply("SYM", np.ones((1, 4)), np.ones((1, 4)))  # SYM without d
    with pytest.raises(ValueError):
        oracle.mahalanobis(np.ones((1, 4)), np.ones((2, 4)), [0], [2], np.ones(4))
