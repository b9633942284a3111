"""Fitting through the differentiable path at the paper's workload shapes (GPU).

* Symmetric form (§III-A, the objective of §IV): fit S_bar = W diag(d) W^T with
  h = 32 reflectors to S = Q diag(k^-1.5) Q^T (n = 1024) from Gaussian probe
  batches; E_x |S x - S_bar x|^2 = |S - S_bar|_F^2 for x ~ N(0, I), so the
  probe loss estimates the paper's objective.  The fitted S_bar is compared
  with S densely at the end.
* Fast Mahalanobis metric (§IV-C): fit U (h = 16) and d = softplus(theta) with
  a hinge loss on labelled pairs of a 10-class mixture in n = 256 whose noise
  has wide directions; the loss falls and 1-NN accuracy with the learned metric
  is no worse than Euclidean on held-out points.
* Checkpoint and resume: a fit interrupted after N steps, saved (module and
  optimiser state dicts, the probe generator's state, the step), restored into
  fresh objects and continued for M steps retraces the uninterrupted N + M
  steps (the kernels reduce in a fixed order, so the losses agree to rounding).
All run every forward and backward through the library's kernels (autograd).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic_inputs as si  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def test_fit_symmetric_form_to_decaying_spectrum():
    from paper_1811_07624_gb300 import ReflectorTransform

    n, h, probes, steps = 1024, 32, 8192, 200
    S, _, _ = si.decaying_symmetric(n, seed=0)
    St = torch.tensor(S, dtype=torch.float32, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(0)
    model = ReflectorTransform(n, h, spectrum=True, generator=g)
    opt = torch.optim.Adam(model.parameters(), lr=0.02)
    losses = []
    for _ in range(steps):
        x = torch.randn(probes, n, device=DEV, generator=g)
        opt.zero_grad()
        loss = ((x @ St - model(x, "SYM")) ** 2).sum(1).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert all(np.isfinite(losses))
    with torch.no_grad():
        Sb = model(torch.eye(n, device=DEV), "SYM")  # row i = S_bar e_i
        rel = float(((St - Sb) ** 2).sum() / (St ** 2).sum())
    print(f"probe loss {losses[0]:.3g} -> {losses[-1]:.3g}; |S - S_bar|^2 / |S|^2 = {rel:.3f}")
    assert losses[-1] < 0.01 * losses[0]
    assert rel < 0.6


def test_fit_mahalanobis_metric_hinge_loss():
    from paper_1811_07624_gb300 import Plan
    from paper_1811_07624_gb300.autograd import mahalanobis

    n, h, steps, n_ref = 256, 16, 60, 3000
    X, labels = si.gaussian_mixture(4000, n=n, seed=0)
    ia, ib, same = si.labelled_pairs(labels[:n_ref], 65536, seed=0)
    Xg = torch.tensor(X, dtype=torch.float32, device=DEV)
    iat, ibt = torch.tensor(ia, device=DEV), torch.tensor(ib, device=DEV)
    samet = torch.tensor(same, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(1)
    U = torch.nn.Parameter(torch.randn(h, n, device=DEV, generator=g))
    theta = torch.nn.Parameter(torch.zeros(n, device=DEV))
    opt = torch.optim.Adam([U, theta], lr=0.02)
    with torch.no_grad():
        m0 = mahalanobis(Xg, iat, ibt, U, torch.nn.functional.softplus(theta)).mean()
    losses = []
    for _ in range(steps):
        opt.zero_grad()
        ds = mahalanobis(Xg, iat, ibt, U, torch.nn.functional.softplus(theta)) / m0
        loss = ds[samet].mean() + torch.relu(1 - ds[~samet]).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.85 * losses[0]

    def knn(Z):
        D = torch.cdist(Z[n_ref:], Z[:n_ref])
        lab = torch.tensor(labels, device=DEV)
        return float((lab[:n_ref][D.argmin(1)] == lab[n_ref:]).float().mean())

    with torch.no_grad():
        d = torch.nn.functional.softplus(theta)
        with Plan(U.detach()) as p:
            Z = p.apply_T(Xg) * d.sqrt()
        acc_learned, acc_euclid = knn(Z), knn(Xg)
    print(f"hinge loss {losses[0]:.3f} -> {losses[-1]:.3f}; 1-NN accuracy "
          f"Euclidean {acc_euclid:.3f}, learned {acc_learned:.3f}")
    assert acc_learned >= acc_euclid - 0.01


def test_checkpoint_resume_matches_uninterrupted(tmp_path):
    from paper_1811_07624_gb300 import ReflectorTransform

    n, h, probes, N, M = 256, 8, 2048, 6, 5
    S, _, _ = si.decaying_symmetric(n, seed=1)
    St = torch.tensor(S, dtype=torch.float32, device=DEV)

    def make():
        g = torch.Generator(device=DEV).manual_seed(3)
        model = ReflectorTransform(n, h, spectrum=True, generator=g)
        return model, torch.optim.Adam(model.parameters(), lr=0.02)

    def run(model, opt, gen, steps):
        out = []
        for _ in range(steps):
            x = torch.randn(probes, n, device=DEV, generator=gen)
            opt.zero_grad()
            loss = ((x @ St - model(x, "SYM")) ** 2).sum(1).mean()
            loss.backward()
            opt.step()
            out.append(float(loss.detach()))
        return out

    model, opt = make()
    ref = run(model, opt, torch.Generator(device=DEV).manual_seed(11), N + M)

    model1, opt1 = make()
    gen1 = torch.Generator(device=DEV).manual_seed(11)
    first = run(model1, opt1, gen1, N)
    path = tmp_path / "fit.pt"
    torch.save({"model": model1.state_dict(), "opt": opt1.state_dict(),
                "rng": gen1.get_state(), "step": N}, path)
    del model1, opt1, gen1

    ck = torch.load(path)
    model2, opt2 = make()
    model2.load_state_dict(ck["model"])
    opt2.load_state_dict(ck["opt"])
    gen2 = torch.Generator(device=DEV)
    gen2.set_state(ck["rng"])
    assert ck["step"] == N
    second = run(model2, opt2, gen2, M)
    np.testing.assert_allclose(first + second, ref, rtol=1e-6)
    with torch.no_grad():
        for a, b in zip(model.parameters(), model2.parameters()):
            torch.testing.assert_close(a, b, rtol=1e-5, atol=1e-6)
