"""Pins of the closed-form factorizations of §II (Results 1-3) in the oracle:
each construction, multiplied out densely, has exactly the error the paper
prints for it, plus the structural facts the paper states (orthonormal
reflectors for Result 1, u_2^T U U_1 u_2 = -1 in Case 2, Result 2 never worse
than Result 1, the block structure and sparse reflectors of the partial QR,
exact reconstruction with n - 1 reflectors, exactness on a symmetric
Hadamard matrix, and the average of Result 3's error against Eq. (14))."""

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import factor as F


def sylvester_hadamard(n):
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H / np.sqrt(n)


@pytest.mark.parametrize("seed", range(4))
def test_result1_error_formula_and_structure(seed):
    n = 10 + seed
    U = si.random_orthonormal(n, seed)
    z = np.linalg.eigvalsh(U + U.T)
    n_minus = int(np.sum(z < 0))
    for h in range(1, n_minus + 3):
        R, err = F.result1(U, h)
        Ub = F.result1_matrix(R)
        assert abs(F.frob2(U - Ub) - err) <= 1e-10 * max(1.0, err)
        live = R[np.any(R != 0, axis=1)]
        assert live.shape[0] == min(h, n_minus)
        assert np.allclose(live @ live.T, np.eye(live.shape[0]), atol=1e-12)
    # with all n_- reflectors: 2n - sum |z|  (Eq. (6))
    _, err = F.result1(U, n_minus)
    assert abs(err - (2 * n - np.sum(np.abs(z)))) <= 1e-10 * err


def test_result1_exact_on_hadamard():
    # a symmetric orthonormal matrix with eigenvalues +-1: z in {+-2}, so
    # h = n_- reflectors reproduce it exactly (remark after Eq. (6), and §IV's
    # note on the Hadamard matrix: half the eigenvalues of H + H^T are -2)
    H = sylvester_hadamard(16)
    z = np.linalg.eigvalsh(H + H.T)
    assert np.sum(np.isclose(z, -2)) == 8 and np.sum(np.isclose(z, 2)) == 8
    R, err = F.result1(H, 8)
    assert abs(err) < 1e-10
    assert F.frob2(H - F.result1_matrix(R)) < 1e-20


@pytest.mark.parametrize("seed", range(4))
def test_result2_error_formula_and_monotone(seed):
    n = 9 + seed
    U = si.random_orthonormal(n, 10 + seed)
    R, err, n_minus = F.result2(U)
    assert R.shape[0] == n_minus
    assert abs(F.frob2(U - F.product_first_acts_first(R)) - err) <= 1e-9 * max(1.0, err)
    errs = [F.frob2(U - F.product_first_acts_first(R[:h])) for h in range(n_minus + 1)]
    assert all(b <= a + 1e-12 for a, b in zip(errs, errs[1:]))
    # the unconstrained construction is never worse than the constrained one
    _, err1 = F.result1(U, n_minus)
    assert err <= err1 + 1e-10


def test_result2_case2_second_reflector():
    U = si.random_orthonormal(11, 3)
    lam, T = np.linalg.eig(U)
    for i in np.flatnonzero((lam.imag > 1e-9) & (lam.real < 0)):
        a, t = lam[i].real, T[:, i] / np.linalg.norm(T[:, i])
        u1 = np.sqrt(2) * t.real
        u2 = 2 * (-np.sqrt(1 + a) / 2 * t.real + np.sqrt(1 - a) / 2 * t.imag)
        assert abs(np.linalg.norm(u1) - 1) < 1e-12 and abs(np.linalg.norm(u2) - 1) < 1e-12
        assert abs(u1 @ (U + U.T) @ u1 - 2 * a) < 1e-12
        assert abs(u2 @ U @ F.reflector(u1) @ u2 + 1.0) < 1e-12


@pytest.mark.parametrize("h", [1, 3, 7])
def test_result3_structure_and_error(h):
    n = 12
    U = si.random_orthonormal(n, 40 + h)
    R, d, M, err = F.result3(U, h)
    # D J_h ... J_1 U = [[I, 0], [0, D_1 U~]] with D_1 U~ having a positive diagonal
    DM = d[:, None] * M
    assert np.allclose(DM[:h, :h], np.eye(h), atol=1e-12)
    assert np.max(np.abs(DM[:h, h:])) < 1e-12 and np.max(np.abs(DM[h:, :h])) < 1e-12
    assert np.all(np.diag(DM)[h:] > 0)
    # reflector k has k leading zeros (0-based), i.e. costs 4 (n - k) per apply
    for k in range(h):
        assert np.all(R[k, :k] == 0)
    assert abs(F.frob2(U - F.result3_matrix(R, d)) - err) <= 1e-10 * max(1.0, err)


def test_result3_complete_with_n_minus_1():
    n = 10
    U = si.random_orthonormal(n, 5)
    R, d, _, err = F.result3(U, n - 1)
    assert abs(err) < 1e-12
    assert F.frob2(U - F.result3_matrix(R, d)) < 1e-24


def test_result3_average_error_near_eq14():
    n, h, trials = 64, 8, 40
    errs = [F.result3(si.random_orthonormal(n, 100 + t), h)[3] for t in range(trials)]
    bound = F.result3_bound(n, h)
    assert abs(np.mean(errs) - bound) <= 0.02 * bound
