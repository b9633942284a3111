"""Reflectors with zero prefixes (§II-D, the remark after Result 3): F32 plans
skip the column blocks before each round's first non-zero.  The skipped terms
are exact zeros, so results equal those of the same plan without skipping,
and match the FP64 oracle; the recorded prefixes follow hh_update."""

import numpy as np
import pytest

import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__

    __graft_entry__.build()
    return torch.device("cuda:0")


def prefixed(n, h, seed, lengths):
    U = si.reflectors(n, h, seed=seed)
    for k, L in enumerate(lengths):
        U[k, :L] = 0.0
    return U


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# shapes where the unskipped apply runs the staged kernel too (the column-split
# kernels take h <= 50 at n <= 1024 and h <= 100 at 2048 < n <= 4096), so that
# skipping the exact zeros must give bit-identical results
@pytest.mark.parametrize("n,h,B", [(1024, 256, 1000), (1000, 96, 777), (2048, 128, 513),
                                   (4096, 128, 130)])
def test_partial_qr_reflectors_skip_and_match(dev, n, h, B):
    import oracle
    from paper_1811_07624_gb300 import Plan

    lengths = [min(n - 1, k * (n // h)) for k in range(h)]  # growing zero prefixes
    U = prefixed(n, h, seed=n + h, lengths=lengths)
    d = si.spectrum(n, seed=1)
    s = si.sign(n, seed=2)
    X = si.vectors(B, n, seed=3)
    Xg = torch.tensor(X, device=dev, dtype=torch.float32)
    with Plan(torch.tensor(U, device=dev, dtype=torch.float32),
              d=torch.tensor(d, device=dev, dtype=torch.float32),
              sign=torch.tensor(s, device=dev)) as p:
        assert p.skip_prefix() is True          # chosen at create: prefixes >= 1/16 of U
        U32 = torch.tensor(U, dtype=torch.float32).double().numpy()
        d32 = torch.tensor(d, dtype=torch.float32).double().numpy()
        X64 = Xg.double().cpu().numpy()
        for mode in ("W", "WT", "SYM"):
            on = p.apply_mode(mode, Xg)
            assert p.skip_prefix(0) is False
            off = p.apply_mode(mode, Xg)
            assert p.skip_prefix(-1) is True
            assert torch.equal(on, off), mode   # the skipped terms are exact zeros
            ref = oracle.apply(mode, U32, X64, sign=s, d=d32)
            assert rel(on.double().cpu().numpy(), ref) <= 1e-5, mode


def test_irregular_prefixes_forced_on(dev):
    """Prefixes in no particular order (the round's smallest decides)."""
    import oracle
    from paper_1811_07624_gb300 import Plan

    n, h, B = 1536, 40, 300
    g = np.random.default_rng(5)
    lengths = list(g.integers(0, n, size=h))
    U = prefixed(n, h, seed=9, lengths=lengths)
    X = si.vectors(B, n, seed=4)
    Xg = torch.tensor(X, device=dev, dtype=torch.float32)
    with Plan(torch.tensor(U, device=dev, dtype=torch.float32)) as p:
        p.skip_prefix(1)
        for mode in ("W", "WT"):
            Y = p.apply_mode(mode, Xg).double().cpu().numpy()
            ref = oracle.apply(mode, torch.tensor(U, dtype=torch.float32).double().numpy(),
                               Xg.double().cpu().numpy())
            assert rel(Y, ref) <= 1e-5


def test_prefixes_follow_update(dev):
    import oracle
    from paper_1811_07624_gb300 import Plan

    n, h, B = 1024, 64, 256
    U1 = prefixed(n, h, 11, [k * 16 for k in range(h)])
    U2 = prefixed(n, h, 12, [(h - 1 - k) * 16 for k in range(h)])  # other prefixes
    X = torch.tensor(si.vectors(B, n, seed=6), device=dev, dtype=torch.float32)
    with Plan(torch.tensor(U1, device=dev, dtype=torch.float32)) as p:
        p.skip_prefix(1)
        p.update(torch.tensor(U2, device=dev, dtype=torch.float32))
        Y = p.apply(X).double().cpu().numpy()
        ref = oracle.apply("W", torch.tensor(U2, dtype=torch.float32).double().numpy(),
                           X.double().cpu().numpy())
        assert rel(Y, ref) <= 1e-5


def test_dense_reflectors_do_not_skip(dev):
    from paper_1811_07624_gb300 import Plan

    U = si.reflectors(512, 16, seed=1)
    with Plan(torch.tensor(U, device=dev, dtype=torch.float32)) as p:
        assert p.skip_prefix() is False
    with Plan(torch.tensor(U, device=dev, dtype=torch.float64)) as p:
        assert p.skip_prefix(1) is False      # F64 plans never skip
