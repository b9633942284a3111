"""Failure handling on the GPU without a GPU fault.

* The bounded mbarrier wait every pipelined kernel uses gives up on a barrier
  nothing arrives on; the host reads HH_ERR_TIMEOUT and the context stays
  usable (a following apply matches the oracle).
* An injected device-allocation failure (the library's allocation hook) makes
  plan creation, the compact-WY preparation, the backward scratch and the
  batched launch return HH_ERR_OOM; the next call succeeds.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic_inputs as si  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _hh():
    import paper_1811_07624_gb300 as hh

    return hh


def _apply_ok(hh, n=256, h=12, B=300):
    U = si.reflectors(n, h, seed=3)
    X = si.vectors(B, n, seed=4)
    with hh.Plan(torch.tensor(U, dtype=torch.float32, device=DEV)) as p:
        Y = p.apply(torch.tensor(X, dtype=torch.float32, device=DEV))
        p.sync()
    ref = oracle.apply("W", torch.tensor(U, dtype=torch.float32).double().numpy(),
                       torch.tensor(X, dtype=torch.float32).double().numpy())
    err = np.linalg.norm(Y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-5


def test_bounded_wait_gives_up_and_context_survives():
    import ctypes

    hh = _hh()
    from paper_1811_07624_gb300 import _lib

    stream = torch.cuda.current_stream().cuda_stream
    st = _lib.lib().hh_debug_wait_timeout(ctypes.c_int64(20_000_000), ctypes.c_void_p(stream))
    assert _lib.STATUS[st] == "HH_ERR_TIMEOUT"
    assert b"gave up" in _lib.lib().hh_last_error()
    torch.cuda.synchronize()
    _apply_ok(hh)


@pytest.mark.parametrize("k", [1, 3, 9])
def test_injected_allocation_failure_in_create(k):
    hh = _hh()
    from paper_1811_07624_gb300 import _lib

    U = torch.tensor(si.reflectors(128, 5, seed=1), dtype=torch.float32, device=DEV)
    d = torch.tensor(si.spectrum(128, seed=1), dtype=torch.float32, device=DEV)
    s = torch.tensor(si.sign(128, seed=1), device=DEV)
    _lib.call("hh_debug_fail_alloc", k)
    try:
        with pytest.raises(hh.HHError, match="OOM"):
            hh.Plan(U, d=d, sign=s)
    finally:
        _lib.call("hh_debug_fail_alloc", 0)
    _apply_ok(hh)


def test_injected_allocation_failure_wy_backward_batch():
    hh = _hh()
    from paper_1811_07624_gb300 import _lib

    try:
        # compact-WY preparation (BF16 plan): its allocations follow the plan's own
        Ub = torch.tensor(si.reflectors(256, 64, seed=2), dtype=torch.float32, device=DEV).bfloat16()
        _lib.call("hh_debug_fail_alloc", 11)
        with pytest.raises(hh.HHError, match="OOM"):
            hh.Plan(Ub)
        _lib.call("hh_debug_fail_alloc", 0)
        with hh.Plan(Ub) as pw:
            Yw = pw.apply(torch.randn(130, 256, device=DEV).bfloat16())
            pw.sync()
            assert bool(torch.isfinite(Yw.float()).all())

        # backward scratch (stream-ordered allocation)
        U = torch.tensor(si.reflectors(512, 8, seed=5), dtype=torch.float32, device=DEV)
        d = torch.tensor(si.spectrum(512, seed=5), dtype=torch.float32, device=DEV)
        with hh.Plan(U, d=d) as p:
            X = torch.randn(64, 512, device=DEV)
            G = torch.randn(64, 512, device=DEV)
            _lib.call("hh_debug_fail_alloc", 1)
            with pytest.raises(hh.HHError, match="OOM"):
                p.backward("SYM", X, G)
            _lib.call("hh_debug_fail_alloc", 0)
            gX, gU, gd = p.backward("SYM", X, G)
            p.sync()
            assert bool(torch.isfinite(gU).all())

            # batched launch
            _lib.call("hh_debug_fail_alloc", 2)
            with pytest.raises(hh.HHError, match="OOM"):
                hh.Batch([p], [64])
            _lib.call("hh_debug_fail_alloc", 0)
            with hh.Batch([p], [64]) as b:
                b.apply([X])
                b.sync()
    finally:
        _lib.call("hh_debug_fail_alloc", 0)
    _apply_ok(hh)
