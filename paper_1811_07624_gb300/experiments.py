"""The synthetic experiments of §IV (Figs. 1-9), run through the library.

Every approximation is built by the library's factorization and fitting
modules (`factor`, `shf`), and every error is measured by applying the
approximation with the library's kernels.  The paper's figures print no
readable values, so the curves are compared with what the text says about
them (the tests and the design notes list those statements), not with
numbers.  Errors are the normalised representation error of Eq. (32),
|X - X_bar|_F^2 / (4 |X|_F^2), averaged over `reps` random instances.

    fig1  n = 32: U_bar_1 (Result 1) and U_bar_2 (Result 2) against h
    fig2  U_bar_2 and the partial QR (Result 3) against h, n in {32, 64, 128}
    fig3  n = 128: U_bar_2, the partial QR and the average bound of Eq. (14)
    fig4  SHF and SHF-SU against h, n in {32, 64, 128}, S = (X + X^T)/2
    fig5  the same with S = X X^T
    fig6  n = 128: SHF-SU, Result 4's partial eigendecomposition, Eq. (28)
    fig7  h = 16: SHF-SU against n, indefinite and positive definite
    fig8  n = 64, h in {18, 24, 30}: SHF-SU's error per iteration, indefinite
    fig9  the same, positive definite

    python -m paper_1811_07624_gb300.experiments --fig 1 [--reps R] [--out F.json]

Reflector counts beyond n_- (Results 1 and 2) add zero reflectors, as the
paper prescribes after Eq. (6); U_bar_2's curve for h > n_- therefore stays
flat, while the partial QR reaches zero error at h = n - 1.
"""

from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import factor, shf


def _rng_gauss(n, seed):
    return np.random.default_rng(seed).standard_normal((n, n))


def random_orthonormal(n, seed):
    q, _ = np.linalg.qr(_rng_gauss(n, seed))
    return q


def random_symmetric(n, seed, psd=False):
    x = _rng_gauss(n, seed)
    return x @ x.T if psd else 0.5 * (x + x.T)


def rel_error_orth(U, kind, R, d=None, device="cuda"):
    """Eq. (32) for an orthonormal U (|U|_F^2 = n)."""
    return factor.error_on_gpu(U, kind, R, d, device=device) / (4.0 * U.shape[0])


# --- §IV-A: orthonormal matrices ------------------------------------------------------


def fig1(n=32, hs=None, reps=10, seed=0, device="cuda"):
    hs = hs or list(range(1, n // 2 + 1))
    e1, e2 = np.zeros(len(hs)), np.zeros(len(hs))
    for r in range(reps):
        U = random_orthonormal(n, seed + r)
        R2, _, _ = factor.result2(U)
        for i, h in enumerate(hs):
            R1, _ = factor.result1(U, h)
            e1[i] += rel_error_orth(U, "result1", R1, device=device)
            Rh = torch.zeros(h, n, dtype=torch.float64)
            m = min(h, R2.shape[0])
            Rh[:m] = R2[:m]
            e2[i] += rel_error_orth(U, "result2", Rh, device=device)
    return {"n": n, "h": hs, "U_bar_1": list(e1 / reps), "U_bar_2": list(e2 / reps)}


def fig2(ns=(32, 64, 128), reps=5, seed=0, device="cuda", hstep=None):
    out = {}
    for n in ns:
        hs = list(range(1, n, hstep or max(1, n // 16)))
        e2, eq = np.zeros(len(hs)), np.zeros(len(hs))
        for r in range(reps):
            U = random_orthonormal(n, seed + r)
            R2, _, _ = factor.result2(U)
            for i, h in enumerate(hs):
                Rh = torch.zeros(h, n, dtype=torch.float64)
                m = min(h, R2.shape[0])
                Rh[:m] = R2[:m]
                e2[i] += rel_error_orth(U, "result2", Rh, device=device)
                R3, d3, _ = factor.result3(U, h)
                eq[i] += rel_error_orth(U, "result3", R3, d3, device=device)
        out[str(n)] = {"h": hs, "U_bar_2": list(e2 / reps), "partial_QR": list(eq / reps)}
    return out


def fig3(n=128, reps=5, seed=0, device="cuda", hstep=8):
    hs = list(range(1, n, hstep))
    r = fig2((n,), reps, seed, device, hstep)[str(n)]
    bound = [(2.0 * (n - h) - 2.0 * math.sqrt(2.0 / math.pi) * math.sqrt(n - h)) / (4.0 * n)
             for h in hs]
    return {"n": n, "h": hs, "U_bar_2": r["U_bar_2"], "partial_QR": r["partial_QR"],
            "result3_bound": bound}


# --- §IV-B: symmetric matrices --------------------------------------------------------


def _shf_error(S, h, su, K, inner, device, U0=None, s_bar0=None):
    St = torch.tensor(S, device=device)
    r = shf.shf(St, h, K=K, spectrum_update=su, inner=inner, tol=0.0,
                U0=None if U0 is None else torch.as_tensor(U0, device=device),
                s_bar0=None if s_bar0 is None else torch.as_tensor(s_bar0, device=device))
    return r["relative_error"]


def fig4(ns=(32, 64, 128), hs=None, reps=3, seed=0, K=10, inner=10, psd=False, device="cuda"):
    out = {}
    for n in ns:
        hh = hs or sorted({1, 2, 4, max(1, n // 8), max(1, n // 4)})
        e_shf, e_su = np.zeros(len(hh)), np.zeros(len(hh))
        for r in range(reps):
            S = random_symmetric(n, seed + r, psd)
            for i, h in enumerate(hh):
                e_shf[i] += _shf_error(S, h, False, K, inner, device)[-1]
                e_su[i] += _shf_error(S, h, True, K, inner, device)[-1]
        out[str(n)] = {"h": hh, "SHF": list(e_shf / reps), "SHF_SU": list(e_su / reps)}
    return out


def fig5(**kw):
    kw["psd"] = True
    return fig4(**kw)


def _partial_eig(S, h):
    """Result 4's construction (Eq. (29)): J_1..J_h bring the h eigenvectors of
    largest |eigenvalue| onto e_1..e_h; s_bar = [lambda; diag(S~)]."""
    w, Q = np.linalg.eigh(S)
    order = np.argsort(-np.abs(w), kind="stable")
    w, Q = w[order], Q[:, order]
    n = S.shape[0]
    R = np.zeros((h, n))
    P = np.eye(n)
    for k in range(h):
        v = P @ Q[:, k]
        v[k] -= 1.0
        nv = np.linalg.norm(v)
        if nv > 1e-14:
            R[k] = v / nv
            P = P - 2.0 * np.outer(R[k], R[k] @ P)
    T = P @ S @ P.T
    return R, np.concatenate([w[:h], np.diag(T)[h:]])


def fig6(n=128, hs=None, reps=3, seed=0, K=10, inner=10, device="cuda"):
    hs = hs or [2, 4, 8, 16, 24, 32]
    e_su, e_eig, bound = np.zeros(len(hs)), np.zeros(len(hs)), np.zeros(len(hs))
    for r in range(reps):
        S = random_symmetric(n, seed + r)
        s2 = float(np.sum(S * S))
        sig = np.sort(np.abs(np.linalg.eigvalsh(S)))[::-1]
        for i, h in enumerate(hs):
            R, sb = _partial_eig(S, h)
            rel = _shf_error(S, h, True, K, inner, device, U0=R, s_bar0=sb)
            e_eig[i] += rel[0]
            e_su[i] += rel[-1]
            bound[i] += (np.sum(sig[h:] ** 2) - (n - h) / 2.0) / (4.0 * s2)
    return {"n": n, "h": hs, "SHF_SU": list(e_su / reps), "partial_eig": list(e_eig / reps),
            "result4_bound": list(bound / reps)}


def fig7(ns=(32, 48, 64, 96, 128), h=16, reps=3, seed=0, K=10, inner=10, device="cuda"):
    ind, pd = [], []
    for n in ns:
        a = b = 0.0
        for r in range(reps):
            a += _shf_error(random_symmetric(n, seed + r), h, True, K, inner, device)[-1]
            b += _shf_error(random_symmetric(n, seed + r, True), h, True, K, inner, device)[-1]
        ind.append(a / reps)
        pd.append(b / reps)
    return {"h": h, "n": list(ns), "indefinite": ind, "positive_definite": pd}


def fig8(n=64, hs=(18, 24, 30), reps=3, seed=0, K=30, inner=10, psd=False, device="cuda"):
    out = {}
    for h in hs:
        acc = np.zeros(K + 1)
        for r in range(reps):
            rel = _shf_error(random_symmetric(n, seed + r, psd), h, True, K, inner, device)
            rel = rel + [rel[-1]] * (K + 1 - len(rel))
            acc += np.array(rel)
        out[str(h)] = list(acc / reps)
    return {"n": n, "iterations": list(range(K + 1)), "h": out}


def fig9(**kw):
    kw["psd"] = True
    return fig8(**kw)


FIGS = {1: fig1, 2: fig2, 3: fig3, 4: fig4, 5: fig5, 6: fig6, 7: fig7, 8: fig8, 9: fig9}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--fig", type=int, required=True, choices=sorted(FIGS))
    ap.add_argument("--reps", type=int, default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    kw = {} if a.reps is None else {"reps": a.reps}
    res = FIGS[a.fig](**kw)
    text = json.dumps({"fig": a.fig, "result": res}, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    else:
        print(text)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
