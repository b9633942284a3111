"""GPU parity of the fused apply kernels against the FP64 oracle.

Every case runs the CUDA path through the C ABI (via the Plan binding) and the
oracle on the same seeded inputs (the GPU's F32/F64 values upcast to FP64),
and compares element by element.  Tolerances: relative L2 <= 1e-5 for F32 with
h <= 64 and <= 1e-12 for F64; swap and sign-flip chains are exact.
Outputs are pre-filled with NaN so an unwritten element fails the check.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic_inputs as si  # noqa: E402
from golden_cases import load_closed_forms  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}
DEV = "cuda"


def _plan(U, d=None, sign=None, dtype=torch.float32):
    from paper_1811_07624_gb300 import Plan

    Ut = torch.as_tensor(U, dtype=dtype, device=DEV)
    dt = None if d is None else torch.as_tensor(d, dtype=dtype, device=DEV)
    st = None if sign is None else torch.as_tensor(sign, device=DEV)
    return Plan(Ut, d=dt, sign=st)


def _as64(t):
    return t.detach().double().cpu().numpy()


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _check(mode, n, h, batch, dtype, seed=0, with_sign=True, ld_extra=0, offset=0, inplace=False):
    U = si.reflectors(n, h, seed=seed, unit=False)
    d = si.spectrum(n, seed=seed)
    s = si.sign(n, seed=seed) if with_sign else None
    X = si.vectors(batch, n, seed=seed)
    plan = _plan(U, d=d, sign=s, dtype=dtype)
    ld = n + ld_extra
    base = torch.full((batch * ld + offset + 8,), float("nan"), dtype=dtype, device=DEV)
    Xg = base[offset:offset + batch * ld].view(batch, ld)[:, :n] if batch else base[:0].view(0, n)
    Xg.copy_(torch.as_tensor(X, dtype=dtype))
    Xin = _as64(Xg)
    if inplace:
        Y = plan.apply_mode(mode, Xg, out=Xg)
    else:
        out = torch.full((batch, n), float("nan"), dtype=dtype, device=DEV)
        Y = plan.apply_mode(mode, Xg, out=out)
    plan.sync()  # raises if a kernel gave up a bounded wait
    torch.cuda.synchronize()
    ref = oracle.apply(mode, _as64(torch.as_tensor(U, dtype=dtype)), Xin, sign=s,
                       d=_as64(torch.as_tensor(d, dtype=dtype)))
    got = _as64(Y)
    assert np.all(np.isfinite(got)), "unwritten or non-finite output"
    err = _rel(got, ref)
    assert err <= TOL[dtype], f"{mode} n={n} h={h} B={batch} {dtype}: rel err {err:.3e}"
    plan.close()
    return err


# --- the small FP64 workload: n=64, h=8, 1024 vectors, whole batch -----------------

@pytest.mark.parametrize("mode", ["W", "WT", "SYM"])
def test_small_fp64_full_batch(mode):
    n, h, B = 64, 8, 1024
    U = si.reflectors(n, h, seed=0)  # unit length, as the workload states
    d = si.spectrum(n, seed=0)
    X = si.vectors(B, n, seed=0)
    plan = _plan(U, d=d, dtype=torch.float64)
    Y = _as64(plan.apply_mode(mode, torch.as_tensor(X, device=DEV)))
    ref = oracle.apply(mode, U, X, d=d)
    assert _rel(Y, ref) <= 1e-12


# --- shapes: every kernel configuration, ragged tails, tiny and odd n -------------

F32_N = [1, 3, 5, 64, 100, 128, 129, 256, 300, 512, 700, 1024, 1500, 2048, 3000, 4096, 5000,
         8192, 12000, 16384, 17000]
F64_N = [1, 2, 7, 64, 65, 128, 200, 256, 511, 1024, 1025, 2048, 4000, 4096, 8192, 9000]


@pytest.mark.parametrize("n", F32_N)
def test_f32_shapes(n):
    for mode in ("W", "WT", "SYM"):
        _check(mode, n, 7, 37, torch.float32, seed=n)


@pytest.mark.parametrize("n", F64_N)
def test_f64_shapes(n):
    for mode in ("W", "WT", "SYM"):
        _check(mode, n, 5, 19, torch.float64, seed=n)


@pytest.mark.parametrize("h", [0, 1, 2, 16, 33, 64])
def test_f32_reflector_counts(h):
    for mode in ("W", "WT", "SYM"):
        _check(mode, 1024, h, 70, torch.float32, seed=h)
        _check(mode, 4096, h, 9, torch.float32, seed=h)


@pytest.mark.parametrize("n,h", [(2052, 26), (3000, 40), (4096, 100), (4096, 101)])
def test_f32_eight_cta_clusters(n, h):
    # 2048 < n <= 4096 beyond the CTA pair's h: clusters of eight CTAs with 512
    # columns each (the last ones partly past n) up to h = 100, staged above
    for mode in ("W", "WT", "SYM"):
        _check(mode, n, h, 21, torch.float32, seed=n + h)


@pytest.mark.parametrize("inplace", [False, True])
def test_f32_eight_cta_clusters_with_idle_sm_fill(inplace):
    # A batch large enough that the SMs eight-CTA clusters leave idle run the
    # staged kernel on a share of the rows beside them: every row is written
    # (no NaN left) and the rows sampled everywhere, densely around the
    # possible split points, match the oracle.
    n, h, B = 4096, 40, 12000
    U = si.reflectors(n, h, seed=11, unit=False)
    d = si.spectrum(n, seed=11)
    s = si.sign(n, seed=11)
    plan = _plan(U, d=d, sign=s, dtype=torch.float32)
    X = torch.as_tensor(si.vectors(B, n, seed=11), dtype=torch.float32, device=DEV)
    idx = np.unique(np.concatenate([np.linspace(0, B - 1, 97).astype(np.int64),
                                    np.arange(8960, 10560, 8), np.arange(B - 70, B)]))
    Xs = _as64(X[torch.as_tensor(idx, device=DEV)])
    for mode in ("W", "WT", "SYM"):
        if inplace:
            Xg = X.clone()
            Y = plan.apply_mode(mode, Xg, out=Xg)
        else:
            Y = plan.apply_mode(mode, X, out=torch.full((B, n), float("nan"), device=DEV))
        plan.sync()
        assert bool(torch.isfinite(Y).all()), f"{mode}: unwritten rows"
        ref = oracle.apply(mode, _as64(torch.as_tensor(U, dtype=torch.float32)), Xs, sign=s,
                           d=_as64(torch.as_tensor(d, dtype=torch.float32)))
        got = _as64(Y[torch.as_tensor(idx, device=DEV)])
        assert _rel(got, ref) <= TOL[torch.float32], f"{mode}: rel err {_rel(got, ref):.3e}"
    plan.close()


def test_idle_sm_fill_in_cuda_graph():
    # the cluster kernel and the staged kernel on the idle SMs fork to a second
    # stream and join back: the pair captures into a CUDA graph and replays to
    # the eager result
    n, h, B = 4096, 40, 12000
    U = si.reflectors(n, h, seed=21, unit=False)
    plan = _plan(U, dtype=torch.float32)
    X = torch.as_tensor(si.vectors(B, n, seed=21), dtype=torch.float32, device=DEV)
    Y_eager = plan.apply(X)  # the first call creates the second stream, outside capture
    Yg = torch.empty_like(X)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.apply(X, out=Yg)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.apply(X, out=Yg)
    Yg.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    plan.sync()
    assert torch.equal(Yg, Y_eager)
    plan.close()


@pytest.mark.parametrize("batch", [0, 1, 2, 7, 8, 9, 31, 33, 513])
def test_batch_tails(batch):
    for n in (256, 1000, 4096):
        for mode in ("W", "SYM"):
            _check(mode, n, 6, batch, torch.float32, seed=batch)


def test_strided_and_unaligned_rows():
    for dtype in (torch.float32, torch.float64):
        _check("W", 1000, 8, 21, dtype, ld_extra=24)     # ld > n, still aligned
        _check("WT", 1000, 8, 21, dtype, ld_extra=3)     # odd ld: scalar loads
        _check("SYM", 1024, 8, 21, dtype, offset=1)      # misaligned base pointer
        _check("W", 4096, 8, 5, dtype, ld_extra=1, offset=3)


def test_in_place():
    for n in (64, 4096):
        for mode in ("W", "WT", "SYM"):
            _check(mode, n, 10, 33, torch.float32, inplace=True)


def test_no_sign():
    for mode in ("W", "WT", "SYM"):
        _check(mode, 512, 9, 40, torch.float32, with_sign=False)


# --- exact cases ---------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_golden_closed_forms_exact(dtype):
    for name, c in load_closed_forms().items():
        plan = _plan(c["U"], d=c.get("d"), sign=None, dtype=dtype)
        x = torch.as_tensor(c["x"][None], dtype=dtype, device=DEV)
        assert np.array_equal(_as64(plan.apply(x))[0], c["W"]), name
        assert np.array_equal(_as64(plan.apply_T(x))[0], c["WT"]), name
        if "d" in c:
            assert np.array_equal(_as64(plan.apply_sym(x))[0], c["SYM"]), name
        if "sign" in c:
            ps = _plan(c["U"], sign=c["sign"].astype(np.int8), dtype=dtype)
            assert np.array_equal(_as64(ps.apply(x))[0], c["W_sign"]), name
            assert np.array_equal(_as64(ps.apply_T(x))[0], c["WT_sign"]), name


def test_permutation_chain_exact_large():
    # transpositions e_i - e_j compose to a permutation: exact in F32 on integers
    rng = np.random.default_rng(3)
    n, h, B = 4096, 24, 50
    pairs = [tuple(rng.choice(n, 2, replace=False)) for _ in range(h)]
    U = np.zeros((h, n))
    for k, (i, j) in enumerate(pairs):
        U[k, i], U[k, j] = 1.0, -1.0
    x = rng.integers(-1000, 1000, size=(B, n)).astype(np.float64)
    y = x.copy()
    for (i, j) in reversed(pairs):
        y[:, [i, j]] = y[:, [j, i]]
    plan = _plan(U, dtype=torch.float32)
    got = _as64(plan.apply(torch.as_tensor(x, dtype=torch.float32, device=DEV)))
    assert np.array_equal(got, y)


@pytest.mark.parametrize("n", [516, 768, 1020, 1024])
@pytest.mark.parametrize("h", [1, 15, 16, 50, 51])
def test_resident_reflectors_single_cta(n, h):
    """512 < n <= 1024, h <= 50: all reflectors resident in one CTA (two or four
    reflectors per round either side of h = 16); h = 51 takes the staged kernel."""
    for mode in ("W", "WT", "SYM"):
        _check(mode, n, h, 37, torch.float32, seed=n + h)


def test_permutation_chain_exact_resident():
    # the same exactness through the single-CTA resident-reflector kernel (n = 1024)
    rng = np.random.default_rng(4)
    n, h, B = 1024, 20, 40
    pairs = [tuple(rng.choice(n, 2, replace=False)) for _ in range(h)]
    U = np.zeros((h, n))
    for k, (i, j) in enumerate(pairs):
        U[k, i], U[k, j] = 1.0, -1.0
    x = rng.integers(-1000, 1000, size=(B, n)).astype(np.float64)
    y = x.copy()
    for (i, j) in reversed(pairs):
        y[:, [i, j]] = y[:, [j, i]]
    plan = _plan(U, dtype=torch.float32)
    got = _as64(plan.apply(torch.as_tensor(x, dtype=torch.float32, device=DEV)))
    assert np.array_equal(got, y)


# --- properties -------------------------------------------------------------------

def test_orthonormality_on_gpu():
    n, h, B = 4096, 16, 4096
    plan = _plan(si.reflectors(n, h, seed=9), sign=si.sign(n, seed=9), dtype=torch.float32)
    g = torch.Generator(device=DEV).manual_seed(9)
    X = torch.randn(B, n, device=DEV, generator=g)
    Y = plan.apply(X)
    Z = plan.apply_T(Y)
    nx, ny = X.double().norm(dim=1), Y.double().norm(dim=1)
    assert float(((ny / nx) - 1).abs().max()) < 1e-5
    assert float((Z - X).double().norm() / X.double().norm()) < 1e-5


# --- argument errors ------------------------------------------------------------------

def test_errors():
    from paper_1811_07624_gb300 import HHError, Plan

    U = torch.randn(3, 16, device=DEV)
    with pytest.raises(HHError) as ei:
        Plan(torch.full((3, 16), float("nan"), device=DEV))
    assert ei.value.code == "HH_ERR_NONFINITE"
    with pytest.raises(HHError) as ei:
        Plan(U, d=torch.full((16,), float("inf"), device=DEV))
    assert ei.value.code == "HH_ERR_NONFINITE"
    with pytest.raises(HHError) as ei:
        Plan(U, sign=torch.zeros(16, dtype=torch.int8, device=DEV))
    assert ei.value.code == "HH_ERR_INVALID_ARG"
    plan = Plan(U)
    X = torch.randn(4, 16, device=DEV)
    with pytest.raises(HHError) as ei:
        plan.apply_sym(X)  # no spectrum
    assert ei.value.code == "HH_ERR_INVALID_ARG"
    # a host pointer is rejected by the C ABI itself
    from paper_1811_07624_gb300 import _lib

    Xh = torch.randn(4, 16).pin_memory()
    Yd = torch.empty(4, 16, device=DEV)
    st = _lib.lib().hh_apply(plan.handle, Xh.data_ptr(), 16, Yd.data_ptr(), 16, 4, None)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    Xp = np.zeros((4, 16), dtype=np.float32)
    st = _lib.lib().hh_apply(plan.handle, Xp.ctypes.data, 16, Yd.data_ptr(), 16, 4, None)
    assert _lib.STATUS[st] == "HH_ERR_INVALID_ARG"
    with pytest.raises(ValueError):
        plan.apply(X, out=torch.empty(3, 16, device=DEV))  # row count differs
    with pytest.raises(ValueError):
        plan.apply(X.double())  # dtype differs from the plan's
