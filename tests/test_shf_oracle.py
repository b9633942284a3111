"""Pins of the SHF / SHF-SU oracle (§III, Algorithm 1) against what the paper
and the mathematics fix, independently of the oracle's own code paths:

* Eq. (20): the objective of Eq. (17), formed densely, equals
  |s|^2 + |s_bar|^2 - 2 tr(A_k B_k) + 4 C(u_k) for every k (pins the product
  order of A_k, B_k, S_bar and the formula of C);
* C as printed (a trace) equals its product-of-quadratic-forms form;
* Eq. (26) against central differences of C;
* u_dagger attains the smallest eigenvalue of A B + B A, and no random unit
  vector goes below it;
* u_ddagger against the closed form of the dominant eigenvector of
  a b^T + b a^T for chosen extreme eigenvectors a, b;
* the arcs of Eq. (25) and Eq. (27) stay on the unit sphere, and the
  one-dimensional search matches a brute-force grid of 200,001 points;
* monotone decrease of the objective over reflector updates (the paper's
  claim after Eq. (27)) and over the spectrum update;
* Eq. (33): the spectrum update is optimal (closed form of the residual, and
  no coordinate perturbation improves it);
* Eq. (31) recovers a known sign diagonal up to the global sign;
* Result 4's construction (Eq. (29)) gives the block structure and the error
  |S~|_F^2 - |diag S~|^2, and SHF-SU started from it never does worse; the
  averaged error sits below the bound of Eq. (28).
"""

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import shf as O


def rand_sym(n, seed):
    return si.random_symmetric(n, seed)


def rand_unit_rows(h, n, seed):
    return si.reflectors(n, h, seed=seed, unit=True)


# --- Eq. (20) / Eq. (21) -------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_objective_expansion_eq20(seed):
    n, h = 9, 3
    S = rand_sym(n, seed)
    U = rand_unit_rows(h, n, seed + 10)
    d = si.sign(n, seed).astype(np.float64)
    s_bar = si.spectrum(n, seed) - 5.0
    s, _ = O.eig_desc(S)
    f = O.objective(S, U, s_bar, d)
    for k in range(h):
        A = O.A_mat(S, U, d, k)
        B = O.B_mat(U, s_bar, k)
        rhs = s @ s + s_bar @ s_bar - 2.0 * np.trace(A @ B) + 4.0 * O.C(U[k], A, B)
        assert abs(f - rhs) <= 1e-10 * f, (k, f, rhs)


def test_objective_expansion_fails_for_reversed_products():
    # the other reading of the descending products breaks Eq. (20)
    n, h = 8, 3
    S = rand_sym(n, 4)
    U = rand_unit_rows(h, n, 5)
    d = np.ones(n)
    s_bar = np.linspace(-2, 3, n)
    s, _ = O.eig_desc(S)
    f = O.objective(S, U, s_bar, d)
    k = 2  # A_k holds two reflectors, so their order matters
    P = O.product(U, range(k))
    A_rev = P @ S @ P.T  # (U_0 ... U_{k-1}) S (U_{k-1} ... U_0)
    B = O.B_mat(U, s_bar, k)
    rhs = s @ s + s_bar @ s_bar - 2.0 * np.trace(A_rev @ B) + 4.0 * O.C(U[k], A_rev, B)
    assert abs(f - rhs) > 1e-6 * f


def test_C_trace_equals_product_form():
    g = np.random.default_rng(3)
    for _ in range(5):
        A = rand_sym(7, int(g.integers(1000)))
        B = rand_sym(7, int(g.integers(1000)))
        u = g.standard_normal(7)
        u /= np.linalg.norm(u)
        assert abs(O.C_trace(u, A, B) - O.C(u, A, B)) <= 1e-12 * (1 + abs(O.C(u, A, B)))


def test_gradient_eq26_central_differences():
    g = np.random.default_rng(7)
    A, B = rand_sym(6, 1), rand_sym(6, 2)
    u = g.standard_normal(6)
    gr = O.grad_C(u, A, B)
    eps = 1e-6
    fd = np.array([(O.C(u + eps * e, A, B) - O.C(u - eps * e, A, B)) / (2 * eps)
                   for e in np.eye(6)])
    assert np.max(np.abs(gr - fd)) <= 1e-7 * (1 + np.max(np.abs(gr)))


# --- the two starting directions -------------------------------------------------

def test_u_dagger_is_the_minimiser_of_the_first_term():
    A, B = rand_sym(8, 11), rand_sym(8, 12)
    M = A @ B + B @ A
    lam = np.linalg.eigvalsh(M)[0]
    ud = O.u_dagger(A, B)
    assert abs(np.linalg.norm(ud) - 1) < 1e-12
    assert abs(ud @ M @ ud - lam) < 1e-10 * max(1, abs(lam))
    g = np.random.default_rng(0)
    for _ in range(200):
        v = g.standard_normal(8)
        v /= np.linalg.norm(v)
        assert v @ M @ v >= lam - 1e-12


@pytest.mark.parametrize("case", ["max_max", "min_min", "min_max"])
def test_u_ddagger_closed_form(case):
    n = 7
    Qa = si.random_orthonormal(n, 1)
    Qb = si.random_orthonormal(n, 2)
    wa = np.linspace(-1.0, 2.0, n)
    wb = np.linspace(-1.5, 1.0, n)
    if case == "min_min":      # largest product from the two smallest eigenvalues
        wa = np.linspace(-5.0, 1.0, n)
        wb = np.linspace(-4.0, 0.5, n)
    if case == "min_max":      # from A's smallest and B's largest (both products < 0 else)
        wa = np.linspace(-5.0, -1.0, n)
        wb = np.linspace(0.5, 3.0, n)
    A = (Qa * wa) @ Qa.T
    B = (Qb * wb) @ Qb.T
    prods = {(ia, ib): wa[ia] * wb[ib] for ia in (0, n - 1) for ib in (0, n - 1)}
    ia, ib = max(prods, key=prods.get)
    a, b = Qa[:, ia], Qb[:, ib]
    c = a @ b
    want = a + (1.0 if c >= 0 else -1.0) * b
    want /= np.linalg.norm(want)
    got = O.u_ddagger(A, B)
    assert min(np.linalg.norm(got - want), np.linalg.norm(got + want)) < 1e-10


# --- the arcs and the one-dimensional search ---------------------------------------

def test_arcs_stay_on_the_unit_sphere():
    g = np.random.default_rng(5)
    a = g.standard_normal(9)
    a /= np.linalg.norm(a)
    b = g.standard_normal(9)
    b -= (a @ b) * a
    b /= np.linalg.norm(b)
    for gam in np.linspace(0.0, np.sqrt(2.0), 41):
        for sgn in (1.0, -1.0):
            u = (1 - gam ** 2 / 2) * a + sgn * np.sqrt(max(gam ** 2 - gam ** 4 / 4, 0.0)) * b
            assert abs(np.linalg.norm(u) - 1.0) < 1e-13


def test_search_matches_brute_force():
    A, B = rand_sym(10, 21), rand_sym(10, 22)
    ud = O.u_dagger(A, B)
    g = np.random.default_rng(1).standard_normal(10)
    g -= (ud @ g) * ud
    g /= np.linalg.norm(g)

    def f(gam):
        return O.C((1 - gam ** 2 / 2) * ud - np.sqrt(max(gam ** 2 - gam ** 4 / 4, 0.0)) * g, A, B)
    best = O._search(f, 0.0, np.sqrt(2.0))
    grid = np.linspace(0.0, np.sqrt(2.0), 200001)
    M = A @ B + B @ A
    us = (1 - grid ** 2 / 2)[:, None] * ud - np.sqrt(np.maximum(grid ** 2 - grid ** 4 / 4, 0))[:, None] * g
    vals = np.einsum("ij,jk,ik->i", us, M, us) - 2 * np.einsum("ij,jk,ik->i", us, A, us) * \
        np.einsum("ij,jk,ik->i", us, B, us)
    assert f(best) <= vals.min() + 1e-9 * (1 + abs(vals.min()))


def test_descend_is_monotone_and_reaches_a_stationary_point():
    A, B = rand_sym(8, 31), rand_sym(8, 32)
    u0 = O.init_reflector(A, B)
    u, cs = O.descend(u0, A, B, inner=400, inner_tol=0.0)
    assert all(b <= a + 1e-12 * (1 + abs(a)) for a, b in zip(cs, cs[1:]))
    gr = O.grad_C(u, A, B)
    tang = gr - (u @ gr) * u  # Riemannian gradient on the sphere
    assert np.linalg.norm(tang) < 1e-4 * (1 + np.linalg.norm(gr))


# --- Algorithm 1 -------------------------------------------------------------------

@pytest.mark.parametrize("su", [False, True])
def test_shf_monotone_over_reflector_and_spectrum_updates(su):
    n, h = 16, 3
    S = rand_sym(n, 40)
    r = O.shf(S, h, K=3, spectrum_update_=su, inner=6, tol=0.0, trace=True)
    steps = r["steps"]
    # within each outer iteration the objective never rises over reflector updates
    for it in range(3):
        objs = [s["objective"] for s in steps[it * h:(it + 1) * h]]
        assert all(b <= a * (1 + 1e-12) for a, b in zip(objs, objs[1:])), objs
        for s in steps[it * h:(it + 1) * h]:
            assert all(b <= a + 1e-12 * (1 + abs(a)) for a, b in zip(s["C"], s["C"][1:]))
    # unit reflectors
    assert np.allclose(np.linalg.norm(r["U"], axis=1), 1.0)
    assert set(np.unique(r["d"])) <= {-1.0, 1.0}


def test_spectrum_update_eq33_is_optimal():
    n, h = 12, 3
    S = rand_sym(n, 50)
    U = rand_unit_rows(h, n, 51)
    d = si.sign(n, 52).astype(np.float64)
    sb = O.spectrum_update(S, U, d)
    f = O.objective(S, U, sb, d)
    # residual of the best diagonal: |U^T S U|^2 - |diag|^2 = |S|^2 - |s_bar|^2
    assert abs(f - (np.sum(S * S) - sb @ sb)) <= 1e-10 * f
    for i in range(n):
        for eps in (1e-3, -1e-3):
            sp = sb.copy()
            sp[i] += eps
            assert O.objective(S, U, sp, d) > f


def test_optimal_sign_eq31_recovers_a_planted_diagonal():
    n = 10
    Q = si.random_orthonormal(n, 60)
    B0 = (Q * np.linspace(1.0, 4.0, n)) @ Q.T
    dp = si.sign(n, 61).astype(np.float64)
    S = np.diag(dp) @ B0 @ np.diag(dp)
    d = O.optimal_sign(S, B0)
    assert np.array_equal(d, dp) or np.array_equal(d, -dp)


# --- Result 4 -----------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1])
def test_result4_construction_eq29(seed):
    n, h = 14, 4
    S = rand_sym(n, 70 + seed)
    U, sb = O.partial_eig_reflectors(S, h)
    P = O.product(U, range(h))  # J_1 ... J_h
    T = P.T @ S @ P             # J_h ... J_1 S J_1 ... J_h
    lam, _ = O.eig_desc(S)
    assert np.max(np.abs(T[:h, h:])) < 1e-10
    assert np.allclose(np.diag(T)[:h], lam[:h], atol=1e-10)
    St = T[h:, h:]
    f = O.objective(S, U, sb, np.ones(n))
    want = np.sum(St * St) - np.sum(np.diag(St) ** 2)
    assert abs(f - want) <= 1e-9 * f
    # |S~|_F^2 is the sum of the n - h smallest squared singular values
    sig = np.sort(np.abs(lam))[::-1]
    assert abs(np.sum(St * St) - np.sum(sig[h:] ** 2)) <= 1e-9 * np.sum(St * St)


def test_shf_su_from_result4_start_never_worse():
    n, h = 16, 3
    S = rand_sym(n, 80)
    U, sb = O.partial_eig_reflectors(S, h)
    start = O.objective(S, U, sb, np.ones(n))
    r = O.shf(S, h, K=3, spectrum_update_=True, inner=5, tol=0.0, U0=U, s_bar0=sb,
              trace=True)
    objs = [s["objective"] for s in r["steps"][:h]]
    assert objs[-1] <= start * (1 + 1e-12)
    assert r["history"][-1] <= start * (1 + 1e-12) or np.min(r["history"]) <= start


def test_result4_bound_on_average():
    n, h, trials = 16, 3, 6
    errs, bounds = [], []
    for t in range(trials):
        S = rand_sym(n, 90 + t)
        U, sb = O.partial_eig_reflectors(S, h)
        r = O.shf(S, h, K=3, spectrum_update_=True, inner=5, tol=0.0, U0=U, s_bar0=sb)
        errs.append(min(r["history"]))
        lam, _ = O.eig_desc(S)
        sig = np.sort(np.abs(lam))[::-1]
        bounds.append(np.sum(sig[h:] ** 2) - (n - h) / 2.0)
    assert np.mean(errs) <= np.mean(bounds)
