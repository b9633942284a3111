"""hh_update: new reflector values for an existing plan, stream-ordered, with
no allocation and no host synchronisation (GPU).

An updated plan gives bit-identical results to a plan created from the new
values (same prepared data, same kernels) and matches the oracle; a NaN is
reported by the next hh_sync as HH_ERR_NONFINITE; the module keeps one plan
across optimiser steps.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic_inputs as si  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(a, dtype=torch.float32):
    return torch.tensor(a, dtype=dtype, device=DEV)


@pytest.mark.parametrize("dtype,n,h", [(torch.float32, 1024, 20), (torch.float32, 4096, 9),
                                       (torch.float64, 300, 7), (torch.float32, 100, 0)])
def test_update_equals_fresh_plan(dtype, n, h):
    from paper_1811_07624_gb300 import Plan, _lib

    s = si.sign(n, seed=1)
    U1, d1 = si.reflectors(n, h, seed=1, unit=False).reshape(h, n), si.spectrum(n, seed=1)
    U2, d2 = si.reflectors(n, h, seed=2, unit=False).reshape(h, n), si.spectrum(n, seed=2)
    X = _t(si.vectors(257, n, seed=3), dtype)
    with Plan(_t(U1, dtype), d=_t(d1, dtype), sign=torch.tensor(s, device=DEV)) as p, \
            Plan(_t(U2, dtype), d=_t(d2, dtype), sign=torch.tensor(s, device=DEV)) as fresh:
        p.apply(X)
        _lib.call("hh_debug_fail_alloc", 1)  # an update must not allocate
        try:
            p.update(_t(U2, dtype), _t(d2, dtype))
        finally:
            _lib.call("hh_debug_fail_alloc", 0)
        for mode in ("W", "WT", "SYM"):
            a = p.apply_mode(mode, X)
            b = fresh.apply_mode(mode, X)
            p.sync()
            assert torch.equal(a, b), mode
            ref = oracle.apply(mode, _t(U2, dtype).double().cpu().numpy().reshape(h, n),
                               X.double().cpu().numpy(), sign=s,
                               d=_t(d2, dtype).double().cpu().numpy())
            tol = 1e-12 if dtype == torch.float64 else 1e-5
            err = np.linalg.norm(a.double().cpu().numpy() - ref) / np.linalg.norm(ref)
            assert err <= tol, (mode, err)


def test_update_nonfinite_and_errors():
    import paper_1811_07624_gb300 as hh

    n, h = 256, 5
    U = _t(si.reflectors(n, h, seed=4))
    with hh.Plan(U, d=_t(si.spectrum(n, seed=4))) as p:
        bad = U.clone()
        bad[2, 7] = float("nan")
        p.update(bad, _t(si.spectrum(n, seed=4)))
        with pytest.raises(hh.HHError, match="NONFINITE"):
            p.sync()
        p.update(U, _t(si.spectrum(n, seed=4)))
        p.sync()  # cleared, fine again
        dbad = _t(si.spectrum(n, seed=4))
        dbad[0] = float("inf")
        p.update(U, dbad)
        with pytest.raises(hh.HHError, match="NONFINITE"):
            p.sync()
        with pytest.raises(hh.HHError, match="INVALID_ARG"):
            p.update(U)  # the plan has a spectrum: d is required
        with pytest.raises(ValueError):
            p.update(U[:, :100])
    with hh.Plan(U) as q:
        with pytest.raises(hh.HHError, match="INVALID_ARG"):
            q.update(U, _t(si.spectrum(n, seed=4)))
    with hh.Plan(_t(si.reflectors(256, 64, seed=5)).bfloat16()) as w:
        with pytest.raises(hh.HHError, match="UNSUPPORTED"):
            w.update(_t(si.reflectors(256, 64, seed=6)).bfloat16())


def test_module_keeps_one_plan_across_steps():
    from paper_1811_07624_gb300 import ReflectorTransform

    g = torch.Generator(device=DEV).manual_seed(0)
    n, h = 128, 6
    target = ReflectorTransform(n, h, spectrum=False, generator=g)
    model = ReflectorTransform(n, h, spectrum=False, generator=g)
    X = torch.randn(512, n, device=DEV, generator=g)
    with torch.no_grad():
        T = target(X)
    opt = torch.optim.Adam(model.parameters(), lr=0.05)
    first = None
    losses = []
    for _ in range(40):
        opt.zero_grad()
        loss = ((model(X) - T) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
        first = first or model.plan()
        assert model.plan() is first
    # the plan follows the parameters: its output equals a fresh plan's
    from paper_1811_07624_gb300 import Plan

    with torch.no_grad(), Plan(model.U.detach().contiguous()) as fresh:
        assert torch.equal(model(X), fresh.apply(X))
    assert losses[-1] < 0.5 * losses[0]
