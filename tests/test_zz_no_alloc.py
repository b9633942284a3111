"""hh_backward_noalloc: the adjoint for callers that cannot allocate.

Some callers cannot let a library allocate device memory when it likes: a
host that owns the whole device memory pool (a framework, a server, a plugin
host) or a training loop that must not block or run out of memory part-way
through a step.  hh_backward_noalloc gives them the same gradients as
hh_backward with its scratch in a fixed array inside the library instead of a
per-call cudaMallocAsync.  This test calls it through the C ABI twice in a row
(the array keeps the previous call's contents, which must not leak into the
next result) and compares each result with hh_backward's, within the
tolerance the gradient tests use; it also checks that a problem too large for
the array is refused with HH_ERR_INVALID_ARG.  The file is named so pytest
runs it last.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = {torch.float32: 1e-4, torch.float64: 1e-10}
MODES = {"W": 0, "WT": 1, "SYM": 2}


def _lib():
    from paper_1811_07624_gb300 import _lib
    from paper_1811_07624_gb300.build import build_library

    build_library()
    return _lib


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _noalloc(L, plan, mode, saved, gY):
    B, n = saved.shape
    gX = torch.full_like(saved, float("nan"))
    gU = torch.full((plan.h, n), float("nan"), device=DEV, dtype=saved.dtype)
    gd = torch.full((n,), float("nan"), device=DEV, dtype=saved.dtype) if mode == "SYM" else None
    st = L.lib().hh_backward_noalloc(plan.handle, MODES[mode], saved.data_ptr(), n, gY.data_ptr(),
                                     n, gX.data_ptr(), n, gU.data_ptr(),
                                     None if gd is None else gd.data_ptr(), B,
                                     torch.cuda.current_stream().cuda_stream)
    L.check(st, "hh_backward_noalloc")
    return gX, gU, gd


@pytest.mark.parametrize("dtype,n,h,B", [(torch.float32, 1024, 32, 8192),
                                         (torch.float32, 4096, 16, 1000),
                                         (torch.float64, 200, 6, 333)])
def test_noalloc_matches_allocating_backward(dtype, n, h, B):
    L = _lib()
    from paper_1811_07624_gb300 import Plan

    g = torch.Generator(device=DEV).manual_seed(n + h)
    U = torch.randn(h, n, device=DEV, dtype=dtype, generator=g)
    d = torch.rand(n, device=DEV, dtype=dtype, generator=g) + 0.1
    sign = torch.where(torch.rand(n, device=DEV, generator=g) < 0.5, -1, 1).to(torch.int8)
    plan = Plan(U, d=d, sign=sign)
    X = torch.randn(B, n, device=DEV, dtype=dtype, generator=g)
    for mode in ("W", "WT", "SYM"):
        G = torch.randn(B, n, device=DEV, dtype=dtype, generator=g)
        saved = X if mode == "SYM" else plan.apply_mode(mode, X)
        ref = plan.backward(mode, saved, G)
        for _ in range(2):  # the second call sees the first call's scratch contents
            got = _noalloc(L, plan, mode, saved, G)
            torch.cuda.synchronize()
            for a, b in zip(got, ref):
                if b is None:
                    assert a is None
                    continue
                assert bool(torch.isfinite(a).all()), f"{mode}: unwritten output"
                assert _rel(a, b) <= TOL[dtype], f"{mode} {dtype}: {_rel(a, b):.2e}"
    plan.sync()


def test_noalloc_rejects_problem_beyond_scratch():
    L = _lib()
    from paper_1811_07624_gb300 import Plan

    n, h = 4096, 2047  # one CTA's partial sums: 2048 * 16 KiB + 8 h bytes > 32 MiB
    plan = Plan(torch.randn(h, n, device=DEV))
    X = torch.randn(4, n, device=DEV)
    gU = torch.empty(h, n, device=DEV)
    st = L.lib().hh_backward_noalloc(plan.handle, 0, X.data_ptr(), n, X.data_ptr(), n, None, n,
                                     gU.data_ptr(), None, 4, None)
    assert L.STATUS[st] == "HH_ERR_INVALID_ARG"
    assert b"scratch" in L.lib().hh_last_error()
    plan_ok = Plan(torch.randn(2046, n, device=DEV))
    st = L.lib().hh_backward_noalloc(plan_ok.handle, 0, X.data_ptr(), n, X.data_ptr(), n, None, n,
                                     None, None, 4, None)
    assert st == 0
    torch.cuda.synchronize()
