"""CPU pins of the oracle's community membership (Section 3.3 Lemma 4,
community case) and of its validation (p-value graph, recovery ratio, average
error), each against something other than the oracle's own formulas: exact
recovery from population moments, closed-form Student-t tails, the library
correlation, and hand-computed scores."""
import numpy as np
import pytest

from oracle import community as oc
from oracle import stgd as ost
from oracle import whiten as ow


def _population(seed, n_x, n_a, k, theta, perm=None):
    """Population MMSB quantities for view A: F_A = Pi_A P^T, M2 = F_A
    diag(alpha_hat) F_A^T, the exact whitening W, whitened expected rows
    Y_A = E[G_{X,A}] W, and the stationary STGD components V."""
    g = np.random.default_rng(seed)
    alpha = g.uniform(0.2, 1.0, k)
    ahat = alpha / alpha.sum()
    Pi_A = g.dirichlet(alpha, size=n_a)                 # n_a x k
    Pi_X = g.dirichlet(alpha, size=n_x)                 # n_x x k
    P = 0.01 + 0.2 * np.eye(k) + 0.01 * g.random((k, k))
    F_A = Pi_A @ P.T                                    # n_a x k
    M2 = (F_A * ahat) @ F_A.T
    W = ow.whiten_exact(M2, k)["W"]
    R = W.T @ F_A * np.sqrt(ahat)                       # orthogonal k x k
    lam = ahat ** -0.5                                  # whitened tensor sum lam_i r_i^(x)3
    V = R * (lam / ost.kappa(theta)) ** (1.0 / 3.0)     # stationary points, ||v||^3 = lam / kappa
    if perm is not None:
        V = V[:, perm]
    YA = (Pi_X @ F_A.T) @ W                             # n_x x k
    return {"YA": YA, "V": V, "R": R, "Pi_X": Pi_X, "ahat": ahat}


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_membership_recovers_population_pi(theta):
    pop = _population(3, 40, 60, 5, theta)
    np.testing.assert_allclose(pop["R"].T @ pop["R"], np.eye(5), atol=1e-10)
    Pi_hat = oc.membership(pop["YA"], pop["V"], theta)
    np.testing.assert_allclose(Pi_hat, pop["Pi_X"].T, atol=1e-9)
    # every column of the estimate is a membership vector (sums to 1)
    np.testing.assert_allclose(Pi_hat.sum(axis=0), 1.0, atol=1e-9)


def test_membership_permuted_components_permute_rows():
    perm = np.array([2, 0, 4, 1, 3])
    pop = _population(4, 30, 50, 5, 1.0, perm=perm)
    Pi_hat = oc.membership(pop["YA"], pop["V"], 1.0)
    np.testing.assert_allclose(Pi_hat, pop["Pi_X"].T[perm], atol=1e-9)


def test_membership_threshold_zeroes_small_entries():
    pop = _population(5, 50, 60, 4, 1.0)
    tau = 0.2
    Pi_hat = oc.membership(pop["YA"], pop["V"], 1.0, tau=tau)
    truth = pop["Pi_X"].T
    assert np.count_nonzero(truth < tau) > 0
    np.testing.assert_allclose(Pi_hat, np.where(truth >= tau, truth, 0.0), atol=1e-9)


def test_pearson_against_library_and_constant_rows():
    g = np.random.default_rng(0)
    a, b = g.standard_normal((2, 50))
    b += 0.3 * a
    assert abs(oc.pearson(a, b) - np.corrcoef(a, b)[0, 1]) < 1e-14
    assert oc.pearson(np.zeros(7), g.standard_normal(7)) == 0.0


@pytest.mark.parametrize("T", [-7.5, -1.0, -0.2, 0.0, 0.3, 1.0, 2.5, 40.0])
def test_right_pvalue_closed_forms(T):
    # nu = 1 (Cauchy): P(t > T) = 1/2 - atan(T)/pi
    assert abs(oc.right_pvalue(T, 1) - (0.5 - np.arctan(T) / np.pi)) < 1e-14
    # nu = 2: P(t > T) = 1/2 - T / (2 sqrt(T^2 + 2))
    assert abs(oc.right_pvalue(T, 2) - (0.5 - T / (2.0 * np.sqrt(T * T + 2.0)))) < 1e-14
    # nu = 4, with s = T / sqrt(T^2 + 4): P(t > T) = 1/2 - (3 s - s^3) / 4
    s = T / np.sqrt(T * T + 4.0)
    assert abs(oc.right_pvalue(T, 4) - (0.5 - (3.0 * s - s ** 3) / 4.0)) < 1e-14


def test_right_pvalue_limits():
    assert oc.right_pvalue(np.inf, 10) == 0.0
    assert oc.right_pvalue(-np.inf, 10) == 1.0
    # large degrees of freedom: the normal tail, to O(1/nu)
    from math import erfc, sqrt
    for T in (0.5, 1.5, 3.0):
        assert abs(oc.right_pvalue(T, 1e7) - 0.5 * erfc(T / sqrt(2.0))) < 1e-6


@pytest.mark.parametrize("rho", [-0.9, -0.1, 0.0, 0.05, 0.4, 0.99])
def test_pvalue_matrix_constructed_correlation(rho):
    # a = z, b = rho z + sqrt(1 - rho^2) w with z, w centred and orthonormal
    n = 12
    g = np.random.default_rng(1)
    Z = g.standard_normal((n, 2))
    Z -= Z.mean(axis=0)
    Q = np.linalg.qr(Z)[0]
    z, w = Q[:, 0], Q[:, 1]
    a = z
    b = rho * z + np.sqrt(1.0 - rho * rho) * w
    T = rho * np.sqrt(n - 2.0) / np.sqrt(1.0 - rho * rho)
    P = oc.pvalue_matrix(a[None, :], b[None, :])
    assert abs(oc.pearson(a, b) - rho) < 1e-13
    # nu = 10 closed form through the regularised incomplete beta:
    # P(t > T) = I_x(5, 1/2) / 2 for T >= 0, x = nu / (nu + T^2)
    from scipy.special import betainc
    x = 10.0 / (10.0 + T * T)
    tail = 0.5 * betainc(5.0, 0.5, x)
    want = tail if T >= 0 else 1.0 - tail
    assert abs(P[0, 0] - want) < 1e-12


def test_match_scores_hand_examples():
    Pi = np.array([[1, 1, 1, 0, 0, 0], [0, 0, 0, 1, 1, 1]], dtype=float)
    # exact copy: rho = 1 on the diagonal (p = 0), -1 off it (p = 1)
    s = oc.match_scores(Pi, Pi)
    assert s["recovery"] == 1.0 and s["error"] == 0.0
    np.testing.assert_array_equal(s["pvalues"], [[0.0, 1.0], [1.0, 0.0]])
    # swapped rows: still a perfect matching
    s = oc.match_scores(Pi[::-1], Pi)
    assert s["recovery"] == 1.0 and s["error"] == 0.0
    # second estimated row empty: community 1 is not recovered
    est = Pi.copy()
    est[1] = 0.0
    s = oc.match_scores(est, Pi)
    assert s["recovery"] == 0.5 and s["error"] == 0.0
    assert s["pvalues"][1, 0] == 0.5 and s["pvalues"][1, 1] == 0.5
    # noisy copy: l1 distances 0.2 / 6 and 0.4 / 6 on the two matched pairs
    est = np.array([[0.9, 1.0, 1.0, 0.1, 0.0, 0.0], [0.0, 0.2, 0.0, 1.0, 0.8, 1.0]])
    s = oc.match_scores(est, Pi)
    np.testing.assert_array_equal(s["edges"], [[True, False], [False, True]])
    assert s["recovery"] == 1.0
    assert abs(s["error"] - (0.2 / 6 + 0.4 / 6) / 2) < 1e-15


def test_match_scores_false_pairing_counts_in_error():
    # one estimated row correlated with both of two ground-truth rows
    Pi = np.array([[1, 1, 0, 0, 0, 0, 0, 0], [0, 0, 1, 1, 0, 0, 0, 0]], dtype=float)
    est = np.array([[1, 1, 1, 1, 0, 0, 0, 0]], dtype=float)
    s = oc.match_scores(est, Pi)
    # rho = 1 / sqrt(3) for both pairs, n = 8: T = rho sqrt(6) / sqrt(2/3) = sqrt(3),
    # P(t_6 > sqrt 3) = I_{6/9}(3, 1/2) / 2 = 0.067: no edge at 0.01, both at 0.1
    from scipy.special import betainc
    p = 0.5 * betainc(3.0, 0.5, 6.0 / 9.0)
    np.testing.assert_allclose(s["pvalues"], [[p, p]], rtol=1e-12)
    assert 0.05 < p < 0.1
    assert not s["edges"].any() and s["recovery"] == 0.0 and s["error"] == 0.0
    s = oc.match_scores(est, Pi, threshold=0.1)
    assert s["edges"].all() and s["recovery"] == 1.0
    # each pair: |est - Pi_j| = 2 ones on the other community's nodes -> l1 / n = 2 / 8
    assert abs(s["error"] - (2 / 8 + 2 / 8) / 2) < 1e-15


def test_pvalue_matrix_needs_three_nodes():
    with pytest.raises(ValueError):
        oc.pvalue_matrix(np.ones((1, 2)), np.ones((1, 2)))


def test_pvalue_graph_of_the_papers_figure():
    """The paper's example graph (golden fixture, 1-based indices as printed):
    estimated rows 2, 3, 6 pair with ground truth 1; 1 with 2; 4, 5 with 4;
    ground truth 3 has no partner, so R = 3/4.  Memberships realising it:
    disjoint blocks of nodes for the ground truth, each estimated row an affine
    copy 0.9 Pi_j + 0.05 of its partner (rho = 1, p = 0; against the other
    blocks rho < 0, p > 1/2), so every pair's l1 / n is 0.05 and E = 6 x 0.05 / 4."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden",
                           "pvalue_graph_figure.json")) as f:
        fig = json.load(f)
    k, k_hat, blk = fig["ground_truth_communities"], fig["estimated_communities"], 50
    n = k * blk
    Pi = np.zeros((k, n))
    for j in range(k):
        Pi[j, j * blk:(j + 1) * blk] = 1.0
    est = np.zeros((k_hat, n))
    for i, j in fig["edges_estimated_to_truth"]:
        est[i - 1] = 0.9 * Pi[j - 1] + 0.05
    s = oc.match_scores(est, Pi, 0.01)
    edges = {(int(i) + 1, int(j) + 1) for i, j in zip(*np.nonzero(s["edges"]))}
    assert edges == {tuple(e) for e in fig["edges_estimated_to_truth"]}
    np.testing.assert_array_equal(s["degree"], fig["degrees_of_truth"])
    assert s["recovery"] == fig["recovery_ratio"]
    assert abs(s["error"] - 6 * 0.05 / 4) < 1e-12
