"""GPU parity of the community membership (otm_membership, Lemma 4 community
case) and of the p-value validation (otm_pvalue_match) against the FP64
oracle, on the same float32 inputs.

Tolerances:
  * membership: FP32 dot products of length k, then an FP64 scale; each entry
    is within 2 k 2^-24 scale_i sum_j |v_ij y_xj| of the exact value (the
    standard bound for a recursively summed dot product, doubled for the
    rounding of the inputs' product).  Where thresholding decides an entry
    within that bound of tau, either outcome is correct.
  * validation: FP64 throughout; the p-values within 1e-9 relative (+1e-14
    absolute: the log-gamma terms of the incomplete beta lose about 1e-12 at
    n = 5,000), l1 within 1e-12 relative; the significant pairs, the recovery
    ratio and the number of pairs identical (no p-value of these inputs lies
    within 1e-6 of the threshold, checked).
"""
import numpy as np
import pytest

from oracle import community as oc
from oracle import stgd as ostgd
from oracle import whiten as ow
from tests._util import to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def otm():
    from paper_1309_0787_gb300 import otm as _otm
    return _otm


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _bound(Y, V, theta):
    """Per-entry error bound of the FP32 membership (see the module doc)."""
    k = V.shape[0]
    norms = np.linalg.norm(V, axis=0)
    lam = ostgd.kappa(theta) * norms ** 3
    g13 = np.sum(lam ** -2.0) ** (-1.0 / 6.0)
    scale = g13 / (lam * norms)
    return 2.0 * k * 2.0 ** -24 * scale[:, None] * (np.abs(V).T @ np.abs(Y).T) + 1e-30


def _check_membership(otm, Y, V, theta, tau=-np.inf):
    Y = Y.astype(np.float32)
    V = V.astype(np.float32)
    got = to_np(otm.membership(_dev(Y), _dev(V.T.copy()), theta, tau)).astype(np.float64)
    torch.cuda.synchronize()
    raw = oc.membership(Y.astype(np.float64), V.astype(np.float64), theta)
    want = np.where(raw >= tau, raw, 0.0)
    bound = _bound(Y.astype(np.float64), V.astype(np.float64), theta)
    # float32 rounding of the output adds 2^-24 relative
    tol = bound + np.abs(want) * 2.0 ** -24
    near = np.abs(raw - tau) <= bound
    ok = (np.abs(got - want) <= tol) | (near & ((got == 0.0) | (np.abs(got - raw) <= tol)))
    assert ok.all(), (np.abs(got - want) / tol).max()
    return got


@pytest.mark.parametrize("n,k", [(1, 3), (63, 10), (64, 16), (1000, 64), (5000, 100),
                                 (777, 130), (300, 256)])
def test_membership_random(otm, n, k):
    g = np.random.default_rng(n * 1000 + k)
    V = g.standard_normal((k, k)) + 2.0 * np.eye(k)
    Y = g.standard_normal((n, k))
    _check_membership(otm, Y, V, 1.0)
    _check_membership(otm, Y, V, 0.5, tau=0.05)


def test_membership_population_recovers_pi(otm):
    """Exact components of population MMSB moments: the estimate is the true
    membership, to FP32 rounding."""
    g = np.random.default_rng(7)
    k, n_a, n_x, theta = 12, 300, 2000, 1.0
    alpha = g.uniform(0.2, 1.0, k)
    ahat = alpha / alpha.sum()
    Pi_A = g.dirichlet(alpha, size=n_a)
    Pi_X = g.dirichlet(alpha, size=n_x)
    P = 0.01 + 0.2 * np.eye(k)
    F = Pi_A @ P.T
    W = ow.whiten_exact((F * ahat) @ F.T, k)["W"]
    R = W.T @ F * np.sqrt(ahat)
    V = R * (ahat ** -0.5 / ostgd.kappa(theta)) ** (1.0 / 3.0)
    Y = (Pi_X @ F.T) @ W
    got = _check_membership(otm, Y, V, theta)
    assert np.abs(got - Pi_X.T).max() < 1e-4


def test_membership_empty_and_invalid(otm):
    V = _dev(np.eye(4, dtype=np.float32))
    out = otm.membership(torch.empty(0, 4, dtype=torch.float32, device="cuda"), V, 1.0)
    assert tuple(out.shape) == (4, 0)
    with pytest.raises(otm.OtmError):
        otm.membership(torch.zeros(8, 1025, dtype=torch.float32, device="cuda"),
                       torch.zeros(1025, 1025, dtype=torch.float32, device="cuda"), 1.0)


def _estimates(seed, k_hat, k, n):
    """Ground truth Pi (k x n, Dirichlet columns) and an estimate mixing
    permuted noisy copies, anti-correlated rows and one constant row."""
    g = np.random.default_rng(seed)
    Pi = g.dirichlet(np.full(k, 0.1), size=n).T
    est = np.empty((k_hat, n))
    src = g.integers(0, k, k_hat)
    noise = np.geomspace(1e-3, 3.0, k_hat)
    for i in range(k_hat):
        sign = -1.0 if i % 7 == 3 else 1.0
        est[i] = sign * Pi[src[i]] + noise[i] * g.standard_normal(n) * Pi[src[i]].std()
    est[k_hat // 2] = 0.25
    return est.astype(np.float32), Pi.astype(np.float32)


@pytest.mark.parametrize("k_hat,k,n", [(2, 2, 3), (5, 4, 4), (17, 33, 130), (40, 40, 1000),
                                       (100, 100, 5000)])
def test_pvalue_match(otm, k_hat, k, n):
    est, Pi = _estimates(k_hat * 7 + n, k_hat, k, n)
    out = otm.pvalue_match(_dev(est), _dev(Pi), 0.01)
    torch.cuda.synchronize()
    ref = oc.match_scores(est.astype(np.float64), Pi.astype(np.float64), 0.01)
    p = to_np(out["pvalues"])
    np.testing.assert_allclose(p, ref["pvalues"], rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(to_np(out["l1"]), ref["l1"], rtol=1e-12, atol=0)
    assert not (np.abs(ref["pvalues"] - 0.01) < 1e-6).any()
    np.testing.assert_array_equal(p <= 0.01, ref["edges"])
    s = to_np(out["scores"])
    assert s[0] == ref["recovery"]
    assert abs(s[1] - ref["error"]) <= 1e-12 * max(ref["error"], 1e-300)
    # the constant row: p = 1/2 against every ground-truth row
    np.testing.assert_array_equal(p[k_hat // 2], 0.5)


def test_pvalue_match_closed_forms(otm):
    """n = 3 and n = 4 (t with 1 and 2 degrees of freedom, closed-form tails),
    exact copies (p = 0) and negated copies (p = 1)."""
    g = np.random.default_rng(11)
    for n, tail in ((3, lambda T: 0.5 - np.arctan(T) / np.pi),
                    (4, lambda T: 0.5 - T / (2.0 * np.sqrt(T * T + 2.0)))):
        Pi = g.random((3, n)).astype(np.float32)
        est = g.random((5, n)).astype(np.float32)
        est[3] = Pi[1]
        est[4] = -Pi[2]
        p = to_np(otm.pvalue_match(_dev(est), _dev(Pi))["pvalues"])
        for i in range(3):
            for j in range(3):
                rho = oc.pearson(est[i], Pi[j])
                T = rho * np.sqrt(n - 2.0) / np.sqrt(1.0 - rho * rho)
                assert abs(p[i, j] - tail(T)) < 1e-12
        assert p[3, 1] == 0.0 and p[4, 2] == 1.0


def test_pvalue_match_invalid(otm):
    z = torch.zeros(2, 2, dtype=torch.float32, device="cuda")
    with pytest.raises(otm.OtmError):
        otm.pvalue_match(z, z)  # n = 2 < 3
