"""GPU parity of the batched persistent launch (hh_batch_*) against the FP64 oracle.

Many transforms of uneven n, h and batch run in one graph-replayed kernel
launch; every transform's output is compared element by element with the
oracle on the same seeded inputs (relative L2 <= 1e-5, F32, h <= 64).  Cases
cover every tile shape, ragged n (not a multiple of the shape's 128-column
granule), n at each shape's full cover, empty transforms, strided rows,
in-place apply, graph replay with new buffers, and the autotuner.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic_inputs as si  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"
TOL = 1e-5


def _hh():
    import paper_1811_07624_gb300 as hh

    return hh


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _make(specs, with_sign=True):
    """Plans and host data for a list of (n, h, batch, seed)."""
    hh = _hh()
    plans, data = [], []
    for n, h, b, seed in specs:
        U = si.reflectors(n, h, seed=seed, unit=False) if h > 0 else np.zeros((0, n))
        d = si.spectrum(n, seed=seed)
        s = si.sign(n, seed=seed) if with_sign else None
        X = si.vectors(b, n, seed=seed + 7) if b > 0 else np.zeros((0, n))
        Ut = torch.as_tensor(U, dtype=torch.float32, device=DEV).reshape(h, n)
        plans.append(hh.Plan(Ut, d=torch.as_tensor(d, dtype=torch.float32, device=DEV),
                             sign=None if s is None else torch.as_tensor(s, device=DEV)))
        data.append((U, d, s, X))
    return plans, data


def _inputs(data, ld_extra=0):
    Xs = []
    for U, d, s, X in data:
        b, n = X.shape
        base = torch.full((b, n + ld_extra), float("nan"), dtype=torch.float32, device=DEV)
        Xg = base[:, :n]
        Xg.copy_(torch.as_tensor(X, dtype=torch.float32))
        Xs.append(Xg)
    return Xs


def _check(data, Xs, Ys, mode, tol=TOL):
    worst = 0.0
    for i, ((U, d, s, _), Xg, Yg) in enumerate(zip(data, Xs, Ys)):
        if Xg.shape[0] == 0:
            continue
        X64 = Xg.double().cpu().numpy()
        ref = oracle.apply(mode, U, X64, sign=s, d=d)
        got = Yg.double().cpu().numpy()
        assert np.isfinite(got).all(), f"transform {i}: unwritten or non-finite output"
        err = _rel(got, ref)
        worst = max(worst, err)
        assert err <= tol, f"transform {i} (n={U.shape[1]}, h={U.shape[0]}, mode {mode}): {err:.3e}"
    return worst


RAGGED = [
    # (n, h, batch, seed): every n range, ragged n, h = 0 and 1, empty and tiny batches
    (64, 8, 300, 1), (100, 5, 77, 2), (128, 4, 1024, 3), (192, 17, 500, 4), (256, 64, 129, 5),
    (260, 9, 65, 6), (320, 33, 400, 7), (512, 1, 256, 8), (640, 12, 0, 9), (704, 40, 333, 10),
    (1000, 7, 31, 11), (1024, 64, 200, 12), (1088, 23, 257, 13), (1536, 0, 90, 14),
    (2048, 16, 129, 15), (2052, 10, 40, 16), (3000, 6, 17, 17), (4096, 12, 33, 18),
]


@pytest.mark.parametrize("mode", ["W", "WT", "SYM"])
def test_batched_ragged_matches_oracle(mode):
    hh = _hh()
    hh.tune_clear()
    plans, data = _make(RAGGED)
    batch = hh.Batch(plans, [x.shape[0] for (_, _, _, x) in data])
    Xs = _inputs(data)
    Ys = [torch.full_like(X, float("nan")) for X in Xs]
    batch.apply(Xs, Ys, mode=mode)
    batch.sync()
    torch.cuda.synchronize()
    _check(data, Xs, Ys, mode)
    info = batch.info()
    assert info["items"] > 0 and info["grid"] > 0
    batch.close()


@pytest.mark.parametrize("shape", range(11))
def test_every_tile_shape(shape):
    """Each compiled shape, at its full cover, one granule short, and ragged."""
    hh = _hh()
    shapes = hh.batch_shapes()
    assert len(shapes) == 11
    cover = shapes[shape]["cover"]
    ns = sorted({cover, max(4, cover - 64), max(4, cover // 2 + 4), max(4, cover - 124)})
    specs = [(n, h, b, 100 + 10 * shape + j)
             for j, (n, h, b) in enumerate(zip(ns, (16, 3, 33, 64), (97, 64, 130, 9)))]
    hh.tune_clear()
    for n, h, _, _ in specs:
        hh.tune_set(n, h, shape)
    try:
        plans, data = _make(specs)
        batch = hh.Batch(plans, [x.shape[0] for (_, _, _, x) in data])
        assert batch.info()["shapes"] == [shape] * len(specs)
        Xs = _inputs(data)
        for mode in ("W", "WT", "SYM"):
            Ys = [torch.full_like(X, float("nan")) for X in Xs]
            batch.apply(Xs, Ys, mode=mode)
            batch.sync()
            _check(data, Xs, Ys, mode)
        batch.close()
    finally:
        hh.tune_clear()


def _resident_shape():
    shapes = _hh().batch_shapes()
    return next(k for k, s in enumerate(shapes) if s["max_cluster"] > 0)


RESIDENT = [
    # (n, h, batch, seed): clusters of one to four CTAs (512 columns each), n
    # ragged inside a CTA's columns, h = 0, 1 and the largest, empty and
    # one-row batches, batches that are not a multiple of the 64-row unit
    (4, 3, 70, 31), (68, 16, 129, 32), (128, 1, 64, 33), (500, 100, 65, 34),
    (512, 0, 40, 35), (516, 9, 300, 36), (700, 33, 1, 37), (1024, 64, 257, 38),
    (1028, 5, 128, 39), (1300, 17, 0, 40), (1536, 100, 63, 41), (1540, 2, 191, 42),
    (1996, 40, 77, 43), (2048, 64, 130, 44),
]


@pytest.mark.parametrize("mode", ["W", "WT", "SYM"])
@pytest.mark.parametrize("ld_extra", [0, 12])
def test_resident_shape_matches_oracle(mode, ld_extra):
    """The resident-reflector shape on every cluster size, against the oracle;
    strided rows padded with NaN (nothing past n is read), then in place."""
    hh = _hh()
    r = _resident_shape()
    hh.tune_clear()
    for n, h, _, _ in RESIDENT:
        hh.tune_set(n, h, r)
    try:
        plans, data = _make(RESIDENT)
        with hh.Batch(plans, [x.shape[0] for (_, _, _, x) in data]) as batch:
            assert batch.info()["shapes"] == [r] * len(RESIDENT)
            Xs = _inputs(data, ld_extra)
            Ys = [torch.full_like(X, float("nan")) for X in Xs]
            batch.apply(Xs, Ys, mode=mode)
            batch.sync()
            _check(data, Xs, Ys, mode)
            X0 = [X.clone() for X in Xs]
            batch.apply(Xs, Xs, mode=mode)  # in place
            batch.sync()
            _check(data, X0, Xs, mode)
    finally:
        hh.tune_clear()


def test_resident_shape_many_transforms_per_cluster():
    """Far more transforms than clusters of each size, so that a cluster walks
    several tasks and reloads reflectors between them; mixed with staged-shape
    transforms in the same batch (both kinds of launch in one graph), replayed."""
    hh = _hh()
    r = _resident_shape()
    rng = np.random.default_rng(5)
    specs = []
    for j in range(160):
        n = int(rng.integers(1, 33)) * 64
        h = int(rng.integers(0, 25))
        specs.append((n, h, int(rng.integers(0, 400)), 500 + j))
    hh.tune_clear()
    for j, (n, h, _, _) in enumerate(specs):
        hh.tune_set(n, h, r if j % 5 else 3 if n <= 1024 else 6)
    try:
        plans, data = _make(specs)
        with hh.Batch(plans, [x.shape[0] for (_, _, _, x) in data]) as batch:
            got = batch.info()["shapes"]
            assert got.count(r) > 100 and got.count(r) < len(specs)
            Xs = _inputs(data)
            for mode in ("W", "SYM"):
                Ys = [torch.full_like(X, float("nan")) for X in Xs]
                batch.apply(Xs, Ys, mode=mode)
                batch.sync()
                _check(data, Xs, Ys, mode)
                Y2 = [torch.full_like(X, float("nan")) for X in Xs]
                batch.apply(Xs, Y2, mode=mode)  # the captured graph, replayed on new buffers
                batch.sync()
                assert all(torch.equal(a, b) for a, b in zip(Ys, Y2))
    finally:
        hh.tune_clear()


def test_batched_equals_separate_launches_and_replays():
    """The same transforms through 1 batched launch and through one hh_apply each."""
    hh = _hh()
    hh.tune_clear()
    specs = [(t["n"], t["h"], min(t["batch"], 600), t["seed"]) for t in si.ragged_transforms(24)]
    plans, data = _make(specs)
    batch = hh.Batch(plans, [x.shape[0] for (_, _, _, x) in data])
    Xs = _inputs(data)
    Ys = batch.apply(Xs, mode="W")
    batch.sync()
    first = [Y.clone() for Y in Ys]
    _check(data, Xs, Ys, "W")
    sep = [p.apply(X) for p, X in zip(plans, Xs)]
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(first, sep)):
        n = a.shape[1]
        assert _rel(a.double().cpu().numpy(), b.double().cpu().numpy()) <= 2 * TOL, i
        assert a.shape == (data[i][3].shape[0], n)
    # replay into the same buffers: bit-identical (each tile is computed in a fixed order)
    batch.apply(Xs, Ys, mode="W")
    batch.sync()
    for a, b in zip(first, Ys):
        assert torch.equal(a, b)
    # new buffers (the task table is re-uploaded), then in place
    Xs2 = [X * 2.0 for X in Xs]
    Ys2 = batch.apply(Xs2, mode="W")
    batch.sync()
    for a, b in zip(first, Ys2):
        torch.testing.assert_close(b, 2.0 * a, rtol=1e-5, atol=1e-5)
    batch.apply(Xs2, Xs2, mode="W")
    batch.sync()
    for a, b in zip(Ys2, Xs2):
        assert torch.equal(a, b)
    batch.close()


def test_batched_strided_rows():
    hh = _hh()
    hh.tune_clear()
    specs = [(256, 8, 100, 1), (1088, 20, 50, 2), (4096, 4, 9, 3)]
    plans, data = _make(specs)
    batch = hh.Batch(plans, [x.shape[0] for (_, _, _, x) in data])
    Xs = _inputs(data, ld_extra=12)
    Ys = [torch.full((X.shape[0], X.shape[1] + 4), float("nan"), device=DEV)[:, :X.shape[1]]
          for X in Xs]
    batch.apply(Xs, Ys, mode="SYM")
    batch.sync()
    _check(data, Xs, Ys, "SYM")
    batch.close()


def test_batched_empty_and_errors():
    hh = _hh()
    hh.tune_clear()
    with hh.Batch([], []) as b:
        assert b.apply([], []) == []
        assert b.info()["items"] == 0
    plans, data = _make([(128, 4, 0, 1), (256, 4, 0, 2)])
    with hh.Batch(plans, [0, 0]) as b:
        Xs = _inputs(data)
        b.apply(Xs, mode="SYM")
        b.sync()
        assert b.info()["items"] == 0
    # unsupported plans at the C ABI: F64, BF16 (compact-WY); and n % 4 != 0, n > 4096
    import ctypes

    from paper_1811_07624_gb300 import _lib

    def raw_create(plan):
        h = ctypes.c_void_p()
        st = _lib.lib().hh_batch_create(ctypes.byref(h), 1, (ctypes.c_void_p * 1)(plan.handle.value),
                                        (ctypes.c_int64 * 1)(4))
        assert not h.value
        return _lib.STATUS[st]

    p64 = hh.Plan(torch.randn(3, 64, device=DEV, dtype=torch.float64))
    assert raw_create(p64) == "HH_ERR_UNSUPPORTED"
    with pytest.raises(ValueError):
        hh.Batch([p64], [4])
    pbf = hh.Plan(torch.randn(64, 256, device=DEV).bfloat16())
    assert raw_create(pbf) == "HH_ERR_UNSUPPORTED"
    p6 = hh.Plan(torch.randn(2, 6, device=DEV))
    with pytest.raises(hh.HHError, match="UNSUPPORTED"):
        hh.Batch([p6], [4])
    p8k = hh.Plan(torch.randn(2, 8192, device=DEV))
    with pytest.raises(hh.HHError, match="UNSUPPORTED"):
        hh.Batch([p8k], [4])
    p8 = hh.Plan(torch.randn(2, 8, device=DEV))
    with pytest.raises(hh.HHError, match="INVALID_ARG"):
        hh.Batch([p8], [-1])
    # SYM without a spectrum
    Uh = si.reflectors(128, 3, seed=5)
    pnod = hh.Plan(torch.as_tensor(Uh, dtype=torch.float32, device=DEV))
    with hh.Batch([pnod], [8]) as b:
        X = torch.randn(8, 128, device=DEV)
        with pytest.raises(hh.HHError, match="INVALID_ARG"):
            b.apply([X], mode="SYM")
        # unaligned rows
        base = torch.randn(8 * 128 + 1, device=DEV)
        Xu = base[1:].view(8, 128)
        with pytest.raises(hh.HHError, match="INVALID_ARG"):
            b.apply([Xu], mode="W")
        with pytest.raises(ValueError):
            b.apply([torch.randn(7, 128, device=DEV)])
        # still usable after the errors
        Y = b.apply([X], mode="WT")[0]
        b.sync()
        ref = oracle.apply("WT", Uh, X.double().cpu().numpy())
        assert _rel(Y.double().cpu().numpy(), ref) <= TOL


def test_autotuner_picks_fastest_measured():
    hh = _hh()
    hh.tune_clear()
    ns, hs = [192, 1088], [8, 40]
    hh.tune(ns, hs, rows=8192)
    shapes = hh.batch_shapes()
    for n in ns:
        for h in hs:
            s, ms = hh.tune_get(n, h)
            for k, m in enumerate(ms):
                if shapes[k]["cover"] >= n:
                    assert math.isfinite(m) and m > 0, (n, h, k, ms)
                else:
                    assert math.isnan(m)
            finite = [(m, k) for k, m in enumerate(ms) if math.isfinite(m)]
            assert s == min(finite)[1]
    # a batch created now uses the tuned shapes, and a nearby h takes the nearest entry
    plans, data = _make([(192, 8, 64, 1), (1088, 40, 64, 2), (1088, 36, 64, 3)])
    with hh.Batch(plans, [64, 64, 64]) as b:
        got = b.info()["shapes"]
        assert got == [hh.tune_get(192, 8)[0], hh.tune_get(1088, 40)[0], hh.tune_get(1088, 40)[0]]
        Xs = _inputs(data)
        Ys = b.apply(Xs, mode="W")
        b.sync()
        _check(data, Xs, Ys, "W")
    hh.tune_clear()
