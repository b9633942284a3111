"""Seeded synthetic inputs for the Householder-chain transforms.

This module only draws random numbers and shapes them into the workloads the
paper experiments with; it holds none of the method's arithmetic, so both the
FP64 oracle (``oracle/``) and the CUDA path may be fed from it.

Recipes (each a numpy ``default_rng(seed)``, PCG64):

* reflector vectors ``U``: ``h x n``, row k is v_k, i.i.d. N(0, 1) entries,
  optionally scaled to unit length (the paper's reflectors have unit norm,
  §II-A, Eq. (2); the library normalises internally anyway);
* spectrum ``d``: ``n`` entries i.i.d. U[0.1, 10] (the symmetric form S̄ of
  §III-A, Eq. (21), with a positive spectrum, as a learned metric has);
* sign ``sigma``: ``n`` entries drawn uniformly from {-1, +1} (the diagonal D
  of Eq. (1));
* vectors ``X``: ``B x n``, i.i.d. N(0, 1);
* random orthonormal matrix: Gaussian matrix, then QR, keep Q (the recipe the
  paper states in §II-D);
* random symmetric targets for the factorization of §III: indefinite
  (X + X^T)/2 and positive semidefinite X X^T, X i.i.d. N(0, 1);
* a symmetric target with decaying spectrum and a Gaussian-mixture metric
  learning set (the differentiation workloads).

Large batches for the GPU are drawn on the device with a seeded
``torch.Generator`` by the callers; :func:`vectors` is the host-side draw used
for the sizes the oracle handles.
"""

from __future__ import annotations

import numpy as np

# Named workloads.  Sizes follow the paper's regime (h much smaller than n,
# §II-A) at the scales the benchmark and parity tests use.
CONFIGS = {
    # small FP64 case, oracle over the whole batch
    "c1_small_fp64": dict(n=64, h=8, batch=1024, dtype="f64", seed=0),
    # FP32 chain at scale
    "c2_n1024_h10": dict(n=1024, h=10, batch=1_048_576, dtype="f32", seed=0),
    "c2_n1024_h32": dict(n=1024, h=32, batch=1_048_576, dtype="f32", seed=0),
    "c2_n4096_h12": dict(n=4096, h=12, batch=262_144, dtype="f32", seed=0),
    "c2_n4096_h16": dict(n=4096, h=16, batch=262_144, dtype="f32", seed=0),
    "c2_n4096_h64": dict(n=4096, h=64, batch=262_144, dtype="f32", seed=0),
    # BF16 storage, compact-WY path
    "c3_n4096_h64_bf16": dict(n=4096, h=64, batch=262_144, dtype="bf16", seed=0),
    "c3_n4096_h256_bf16": dict(n=4096, h=256, batch=262_144, dtype="bf16", seed=0),
    "c3_n4096_h1024_bf16": dict(n=4096, h=1024, batch=262_144, dtype="bf16", seed=0),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def reflectors(n: int, h: int, seed: int = 0, unit: bool = True) -> np.ndarray:
    """``h x n`` float64 array; row k holds reflector vector v_k."""
    g = rng(seed)
    U = g.standard_normal((h, n))
    if unit and h > 0:
        U /= np.linalg.norm(U, axis=1, keepdims=True)
    return U


def spectrum(n: int, seed: int = 0, lo: float = 0.1, hi: float = 10.0) -> np.ndarray:
    """Length-n float64 spectrum, i.i.d. uniform on [lo, hi]."""
    g = rng(seed + 1)
    return g.uniform(lo, hi, size=n)


def sign(n: int, seed: int = 0) -> np.ndarray:
    """Length-n int8 vector of +-1."""
    g = rng(seed + 2)
    return np.where(g.random(n) < 0.5, -1, 1).astype(np.int8)


def vectors(batch: int, n: int, seed: int = 0) -> np.ndarray:
    """``batch x n`` float64 Gaussian vectors (row-major, one vector per row)."""
    g = rng(seed + 3)
    return g.standard_normal((batch, n))


def random_orthonormal(n: int, seed: int = 0) -> np.ndarray:
    """Gaussian n x n matrix orthogonalised by QR (the Q factor)."""
    g = rng(seed + 4)
    q, _ = np.linalg.qr(g.standard_normal((n, n)))
    return q


def decaying_symmetric(n: int, seed: int = 0, power: float = 1.5):
    """Symmetric target S = Q diag(k^-power) Q^T with a random orthonormal Q.

    Returns (S, Q, lam) with lam[k-1] = k^-power, k = 1..n.
    """
    q = random_orthonormal(n, seed)
    lam = np.arange(1, n + 1, dtype=np.float64) ** (-power)
    return (q * lam) @ q.T, q, lam


def random_symmetric(n: int, seed: int = 0) -> np.ndarray:
    """Indefinite symmetric S = (X + X^T) / 2 with X i.i.d. N(0, 1) (§III-D,
    the random symmetric matrices of Result 4 and of the §IV experiments)."""
    x = rng(seed + 5).standard_normal((n, n))
    return 0.5 * (x + x.T)


def random_wishart(n: int, seed: int = 0) -> np.ndarray:
    """Positive semidefinite S = X X^T with X i.i.d. N(0, 1) (the Wishart
    matrices of the remark after Result 4)."""
    x = rng(seed + 6).standard_normal((n, n))
    return x @ x.T


def gaussian_mixture(n_points: int, n: int = 256, classes: int = 10, seed: int = 0,
                     n_wide: int = 64, wide: float = 4.0, narrow: float = 0.25,
                     mean_scale: float = 3.0):
    """Labelled points from a ``classes``-component Gaussian mixture in R^n.

    Class means lie in a random (classes-1)-dimensional subspace; the shared
    noise covariance has ``n_wide`` random directions of variance ``wide`` and
    the rest of variance ``narrow``, so the Euclidean metric is a poor one.
    Returns (X float64 [n_points, n], labels int64 [n_points]).
    """
    g = rng(seed + 5)
    basis, _ = np.linalg.qr(g.standard_normal((n, classes - 1)))
    means = mean_scale * (g.standard_normal((classes, classes - 1)) @ basis.T)
    qn, _ = np.linalg.qr(g.standard_normal((n, n)))
    var = np.full(n, narrow)
    var[g.choice(n, size=n_wide, replace=False)] = wide
    labels = g.integers(0, classes, size=n_points)
    z = g.standard_normal((n_points, n)) * np.sqrt(var)
    X = means[labels] + z @ qn.T
    return X, labels


def labelled_pairs(labels: np.ndarray, n_pairs: int, seed: int = 0, same_frac: float = 0.5):
    """Index pairs (ia, ib) into a labelled set, ``same_frac`` of them same-class.

    Returns (ia int64, ib int64, same bool).
    """
    g = rng(seed + 6)
    labels = np.asarray(labels)
    n_pts = labels.shape[0]
    by_class = [np.flatnonzero(labels == c) for c in range(int(labels.max()) + 1)]
    ia = g.integers(0, n_pts, size=n_pairs)
    same = g.random(n_pairs) < same_frac
    ib = g.integers(0, n_pts, size=n_pairs)
    for p in np.flatnonzero(same):
        members = by_class[labels[ia[p]]]
        ib[p] = members[g.integers(0, members.shape[0])]
    same = labels[ia] == labels[ib]
    return ia.astype(np.int64), ib.astype(np.int64), same


def ragged_transforms(count: int = 512, seed: int = 1000):
    """Shapes of ``count`` independent transforms for the batched launch.

    n uniform on {128, 192, ..., 2048}, h uniform on {4, ..., 64}, batch
    uniform on {1024, ..., 16384}; transform i uses seed ``seed + i``.
    """
    out = []
    for i in range(count):
        g = rng(seed + i)
        n = int(g.integers(2, 33)) * 64
        h = int(g.integers(4, 65))
        b = int(g.integers(1024, 16385))
        out.append(dict(n=n, h=h, batch=b, seed=seed + i))
    return out
