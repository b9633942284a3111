"""The closed-form factorizations of §II (Results 1-3) as library plans: the
approximation applied on the GPU (to the identity) has the error the FP64
oracle's dense product gives and the paper prints; Result 3's reflectors are
unique and match the oracle's."""

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


@pytest.mark.parametrize("n", [16, 64, 200])
def test_results_1_2_3_errors_on_gpu(dev, n):
    from oracle import factor as F
    from paper_1811_07624_gb300 import factor as G

    U = si.random_orthonormal(n, n)
    z = np.linalg.eigvalsh(U + U.T)
    n_minus = int(np.sum(z < 0))
    # Result 1, a few reflector counts up to n_-
    for h in sorted({1, n_minus // 2, n_minus}):
        R, err = G.result1(U, h)
        Ro, erro = F.result1(U, h)
        dense = F.frob2(U - F.result1_matrix(Ro))
        assert abs(err - erro) <= 1e-9 * max(1, erro)
        assert abs(G.error_on_gpu(U, "result1", R) - dense) <= 1e-9 * max(1, dense)
    # Result 2 with all n_- reflectors: Eq. (13)
    R, err, nm = G.result2(U)
    Ro, erro, nmo = F.result2(U)
    assert nm == nmo and abs(err - erro) <= 1e-9 * max(1, erro)
    assert abs(G.error_on_gpu(U, "result2", R) - erro) <= 1e-8 * max(1, erro)
    # Result 3: unique reflectors and sign, error of the proof
    for h in (1, n // 4, n - 1):
        R, d, err = G.result3(U, h)
        Ro, do, _, erro = F.result3(U, h)
        np.testing.assert_allclose(R.numpy(), Ro, atol=1e-10)
        assert np.array_equal(d.numpy(), do)
        assert abs(err - erro) <= 1e-9 * max(1, abs(erro))
        dense = F.frob2(U - F.result3_matrix(Ro, do))
        assert abs(G.error_on_gpu(U, "result3", R, d) - dense) <= 1e-9 * max(1, dense) + 1e-20


def test_result3_plan_in_fp32_against_oracle(dev):
    """The partial-QR reflectors (zero prefixes of growing length) in an F32
    plan applied to a batch: parity with the oracle's chain."""
    import oracle
    from oracle import factor as F
    from paper_1811_07624_gb300 import factor as G

    n, h, B = 1024, 256, 4096
    U = si.random_orthonormal(n, 7)
    R, d, _ = G.result3(U, h)
    X = si.vectors(B, n, seed=8)
    p, mode = G.plan("result3", R, d, device=dev, dtype=torch.float32)
    with p:
        Y = p.apply_mode(mode, torch.tensor(X, device=dev, dtype=torch.float32))
    R32 = R.float().double().numpy()
    # U_bar x = J_1 ... J_h D x = (W^T with the reversed reflectors and sign D)
    ref = oracle.apply("WT", R32[::-1].copy(), torch.tensor(X).float().double().numpy(),
                       sign=d.numpy().astype(np.int8))
    err = np.linalg.norm(Y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-5
    # the same through the dense matrix of the approximation
    ref2 = torch.tensor(X).float().double().numpy() @ F.result3_matrix(R32, d.numpy()).T
    assert np.linalg.norm(Y.double().cpu().numpy() - ref2) / np.linalg.norm(ref2) <= 1e-5
