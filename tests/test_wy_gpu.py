"""GPU parity of the compact-WY BF16 path (tcgen05 GEMMs) against the FP64 oracle.

Two errors are checked for every result (relative L2 over the output):
  * kernel arithmetic: the oracle on the BF16-rounded X and reflectors;
  * end to end: the oracle on the unrounded values.
Both must be <= 1e-2, the BF16 bound.  The kernel stores Z = X V and
V' = V T^T in BF16 and accumulates in FP32; T and the normalisation are FP64.
Integer swap chains are exact (every intermediate is a small integer).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic_inputs as si  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
BF16_TOL = 1e-2


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _wy_case(mode, n, h, B, seed=0, with_sign=True, inplace=False):
    from paper_1811_07624_gb300 import Plan

    U = si.reflectors(n, h, seed=seed)
    s = si.sign(n, seed=seed) if with_sign else None
    X = si.vectors(B, n, seed=seed)
    Ub = torch.as_tensor(U, dtype=torch.bfloat16, device=DEV)
    plan = Plan(Ub, sign=None if s is None else torch.as_tensor(s, device=DEV))
    assert plan.path == "wy"
    Xb = torch.as_tensor(X, dtype=torch.bfloat16, device=DEV)
    if inplace:
        Y = Xb.clone()
        plan.apply_mode(mode, Y, out=Y)
    else:
        Y = plan.apply_mode(mode, Xb)
    plan.sync()
    got = Y.double().cpu().numpy()
    ref_rounded = oracle.apply(mode, Ub.double().cpu().numpy(), Xb.double().cpu().numpy(), sign=s)
    ref_exact = oracle.apply(mode, U, X, sign=s)
    e_kernel, e_total = _rel(got, ref_rounded), _rel(got, ref_exact)
    assert e_kernel <= BF16_TOL, f"{mode} n={n} h={h} B={B}: kernel err {e_kernel:.2e}"
    assert e_total <= BF16_TOL, f"{mode} n={n} h={h} B={B}: end-to-end err {e_total:.2e}"
    return e_kernel, e_total


@pytest.mark.parametrize("mode", ["W", "WT"])
@pytest.mark.parametrize("n,h,B", [(64, 1, 5), (256, 16, 130), (512, 64, 256), (1000, 100, 129),
                                   (4096, 64, 300), (4096, 256, 200), (2048, 300, 127),
                                   (4096, 1024, 64)])
def test_wy_parity(mode, n, h, B):
    _wy_case(mode, n, h, B, seed=n + h)


@pytest.mark.parametrize("mode", ["W", "WT"])
@pytest.mark.parametrize("n,h,B", [(256, 128, 20000), (520, 192, 19500), (128, 64, 40001)])
def test_wy_parity_many_tiles(mode, n, h, B):
    """More 128-row tiles than SMs: each persistent CTA walks several tiles, so
    the next tile's GEMM 1 overlaps the previous tile's epilogue."""
    _wy_case(mode, n, h, B, seed=n + h + 1)


def test_wy_no_sign_and_in_place():
    for mode in ("W", "WT"):
        _wy_case(mode, 1024, 128, 200, with_sign=False)
        _wy_case(mode, 1024, 128, 200, inplace=True)


def test_wy_swap_chain_exact():
    from paper_1811_07624_gb300 import Plan

    rng = np.random.default_rng(4)
    n, h, B = 4096, 24, 300
    pairs = [tuple(rng.choice(n, 2, replace=False)) for _ in range(h)]
    U = np.zeros((h, n))
    for k, (i, j) in enumerate(pairs):
        U[k, i], U[k, j] = 1.0, -1.0
    x = rng.integers(-100, 100, size=(B, n)).astype(np.float64)
    y = x.copy()
    for (i, j) in reversed(pairs):
        y[:, [i, j]] = y[:, [j, i]]
    plan = Plan(torch.as_tensor(U, dtype=torch.bfloat16, device=DEV))
    got = plan.apply(torch.as_tensor(x, dtype=torch.bfloat16, device=DEV)).double().cpu().numpy()
    assert np.array_equal(got, y)


def test_wy_orthonormal():
    from paper_1811_07624_gb300 import Plan

    n, h, B = 4096, 256, 1024
    plan = Plan(torch.as_tensor(si.reflectors(n, h, seed=3), dtype=torch.bfloat16, device=DEV))
    g = torch.Generator(device=DEV).manual_seed(3)
    X = torch.randn(B, n, device=DEV, generator=g).bfloat16()
    Y = plan.apply(X)
    Z = plan.apply_T(Y)
    ratio = Y.double().norm(dim=1) / X.double().norm(dim=1)
    assert float((ratio - 1).abs().max()) < 1e-2
    assert float((Z.double() - X.double()).norm() / X.double().norm()) < 2e-2


def test_wy_errors():
    from paper_1811_07624_gb300 import HHError, Plan

    with pytest.raises(HHError) as ei:
        Plan(torch.randn(4, 100, device=DEV).bfloat16())  # n not a multiple of 8
    assert ei.value.code == "HH_ERR_UNSUPPORTED"
    plan = Plan(torch.randn(4, 128, device=DEV).bfloat16(), d=torch.rand(128, device=DEV).bfloat16())
    with pytest.raises(HHError) as ei:
        plan.apply_sym(torch.randn(3, 128, device=DEV).bfloat16())
    assert ei.value.code == "HH_ERR_UNSUPPORTED"
    with pytest.raises(HHError) as ei:
        Plan(torch.full((2, 128), float("nan"), device=DEV).bfloat16())
    assert ei.value.code == "HH_ERR_NONFINITE"
