"""GPU parity of the fast Mahalanobis distance (§IV-C) and its gradient.

Forward: hh_mahalanobis against oracle.mahalanobis on gathered pairs.
Gradient: against the oracle composed from its own pieces, for
L = sum_p g_p d_p with d_p = sum_m d_m z_m^2, z = W^T(sigma .* (x_a - x_b)):
dL/dd = sum_p g_p z_p^2 and dL/dU = backward of W^T with seed 2 g_p d .* z_p.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic_inputs as si  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = {torch.float32: 1e-5, torch.float64: 1e-12}
GTOL = {torch.float32: 1e-4, torch.float64: 1e-10}


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _setup(n, h, N, P, dtype, seed):
    from paper_1811_07624_gb300 import Plan

    U = si.reflectors(n, h, seed=seed, unit=False)
    d = si.spectrum(n, seed=seed)
    s = si.sign(n, seed=seed)
    X, labels = si.gaussian_mixture(N, n=n, seed=seed)
    ia, ib, _ = si.labelled_pairs(labels, P, seed=seed)
    ia[:3] = ib[:3]  # identical rows: distance 0
    Ut = torch.as_tensor(U, dtype=dtype, device=DEV)
    dt = torch.as_tensor(d, dtype=dtype, device=DEV)
    plan = Plan(Ut, d=dt, sign=torch.as_tensor(s, device=DEV))
    Xg = torch.as_tensor(X, dtype=dtype, device=DEV)
    as64 = lambda t: t.double().cpu().numpy()  # noqa: E731
    return plan, Xg, torch.as_tensor(ia, device=DEV), torch.as_tensor(ib, device=DEV), \
        as64(Ut), as64(dt), s, as64(Xg), ia, ib


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,h", [(256, 16), (100, 7), (1024, 8), (4096, 4)])
def test_mahalanobis_forward(dtype, n, h):
    plan, Xg, iag, ibg, U, d, s, X, ia, ib = _setup(n, h, 300, 1001, dtype, seed=n + h)
    out = plan.mahalanobis(Xg, iag, ibg)
    plan.sync()
    ref = oracle.mahalanobis(U, X, ia, ib, d, sign=s)
    got = out.double().cpu().numpy()
    assert _rel(got, ref) <= TOL[dtype]
    assert np.all(got[:3] == 0.0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,h", [(256, 16), (100, 7), (1024, 8), (512, 12), (256, 5)])
def test_mahalanobis_gradient(dtype, n, h):
    plan, Xg, iag, ibg, U, d, s, X, ia, ib = _setup(n, h, 200, 777, dtype, seed=3 * n + h)
    g = np.random.default_rng(n).standard_normal(ia.shape[0])
    gU, gd = plan.mahalanobis_backward(Xg, iag, ibg, torch.as_tensor(g, dtype=dtype, device=DEV))
    plan.sync()
    delta = X[ia] - X[ib]
    z = oracle.apply("WT", U, delta, sign=s)
    gd_ref = (g[:, None] * z * z).sum(axis=0)
    _, gU_ref, _ = oracle.backward("WT", U, delta, 2.0 * g[:, None] * d[None, :] * z, sign=s)
    assert _rel(gd.double().cpu().numpy(), gd_ref) <= GTOL[dtype]
    assert _rel(gU.double().cpu().numpy(), gU_ref) <= GTOL[dtype]


def test_mahalanobis_bad_index_reported():
    from paper_1811_07624_gb300 import HHError, Plan

    plan = Plan(torch.randn(3, 64, device=DEV), d=torch.rand(64, device=DEV))
    X = torch.randn(10, 64, device=DEV)
    ia = torch.tensor([0, 1, 10], device=DEV)
    ib = torch.tensor([1, -1, 2], device=DEV)
    out = plan.mahalanobis(X, ia, ib)
    with pytest.raises(HHError) as ei:
        plan.sync()
    assert ei.value.code == "HH_ERR_INVALID_ARG"
    o = out.cpu()
    assert torch.isfinite(o[0]) and torch.isnan(o[1]) and torch.isnan(o[2])
    plan.sync()  # the status word was cleared


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("h", [5, 8])
def test_mahalanobis_gradient_bad_index_reported(dtype, h):
    """An out-of-range index in the gradient call is reported, and its pair
    contributes nothing: the gradients equal those of the valid pairs alone."""
    from paper_1811_07624_gb300 import HHError

    plan, Xg, iag, ibg, U, d, s, X, ia, ib = _setup(64, h, 40, 30, dtype, seed=9)
    g = torch.ones(ia.shape[0], dtype=dtype, device=DEV)
    bad_a, bad_b = iag.clone(), ibg.clone()
    bad_a[3], bad_b[7] = 40, -1
    gU, gd = plan.mahalanobis_backward(Xg, bad_a, bad_b, g)
    with pytest.raises(HHError) as ei:
        plan.sync()
    assert ei.value.code == "HH_ERR_INVALID_ARG"
    keep = torch.ones(ia.shape[0], dtype=torch.bool, device=DEV)
    keep[3] = keep[7] = False
    gU_ref, gd_ref = plan.mahalanobis_backward(Xg, iag[keep], ibg[keep], g[keep])
    plan.sync()
    tol = 1e-5 if dtype == torch.float32 else 1e-12
    assert _rel(gU.double().cpu().numpy(), gU_ref.double().cpu().numpy()) <= tol
    assert _rel(gd.double().cpu().numpy(), gd_ref.double().cpu().numpy()) <= tol


def test_mahalanobis_gradcheck_f64():
    from paper_1811_07624_gb300 import autograd

    g = torch.Generator(device=DEV).manual_seed(2)
    n, h, N = 8, 3, 6
    X = torch.randn(N, n, device=DEV, dtype=torch.float64, generator=g)
    U = torch.randn(h, n, device=DEV, dtype=torch.float64, generator=g, requires_grad=True)
    d = (torch.rand(n, device=DEV, dtype=torch.float64, generator=g) + 0.5).requires_grad_(True)
    ia = torch.tensor([0, 1, 2, 5], device=DEV)
    ib = torch.tensor([3, 4, 2, 0], device=DEV)
    fn = lambda U, d: autograd.mahalanobis(X, ia, ib, U, d)  # noqa: E731
    assert torch.autograd.gradcheck(fn, (U, d), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_metric_learning_hinge_improves_separation():
    # the differentiation workload in small: learn U, d on a Gaussian mixture
    # with a hinge loss over same/different pairs; the loss must go down
    from paper_1811_07624_gb300 import autograd

    n, h = 256, 16
    X, labels = si.gaussian_mixture(2000, n=n, seed=11)
    ia, ib, same = si.labelled_pairs(labels, 20000, seed=11)
    Xg = torch.as_tensor(X, dtype=torch.float32, device=DEV)
    iag, ibg = torch.as_tensor(ia, device=DEV), torch.as_tensor(ib, device=DEV)
    sameg = torch.as_tensor(same, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(0)
    U = torch.nn.Parameter(torch.randn(h, n, device=DEV, generator=g))
    theta = torch.nn.Parameter(torch.zeros(n, device=DEV))
    opt = torch.optim.Adam([U, theta], lr=0.05)
    scale = float(((Xg[iag] - Xg[ibg]) ** 2).sum(1).mean())

    def loss_fn():
        dist = autograd.mahalanobis(Xg, iag, ibg, U, torch.nn.functional.softplus(theta)) / scale
        return dist[sameg].mean() + torch.relu(1.0 - dist[~sameg]).mean()

    first = float(loss_fn().detach())
    for _ in range(40):
        opt.zero_grad()
        loss = loss_fn()
        loss.backward()
        opt.step()
    assert float(loss_fn().detach()) < 0.8 * first
