"""CPU pins of the oracle's moment estimators (Section 2, Eqs. (1)-(3), (7)-(11)).

Each test checks the oracle against something other than its own formula:
brute-force enumeration of word positions, Lemma 1's closed form under exact
Dirichlet expectations, and Lemma 2's factorised form on expected graphs.
"""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import moments as om


def _docs_to_csr(docs, d):
    dense = np.zeros((len(docs), d))
    for t, doc in enumerate(docs):
        for w in doc:
            dense[t, w] += 1.0
    return synth.csr_from_dense(dense)


def _bruteforce(docs, d):
    """Moments by enumerating ordered distinct word positions in each document."""
    n = len(docs)
    M1 = np.zeros(d)
    P2 = np.zeros((d, d))
    E3 = np.zeros((d, d, d))
    for doc in docs:
        l = len(doc)
        for p in range(l):
            M1[doc[p]] += 1.0 / l / n
        if l >= 2:
            for p, q in itertools.permutations(range(l), 2):
                P2[doc[p], doc[q]] += 1.0 / (l * (l - 1)) / n
        if l >= 3:
            for p, q, r in itertools.permutations(range(l), 3):
                E3[doc[p], doc[q], doc[r]] += 1.0 / (l * (l - 1) * (l - 2)) / n
    return M1, P2, E3


def test_topic_moments_match_position_enumeration():
    docs = [[0, 1, 1, 3], [2, 2, 2], [4, 0, 3, 3, 1, 0], [1], [], [3, 4]]
    d = 5
    X = _docs_to_csr(docs, d)
    M1, P2, E3 = _bruteforce(docs, d)
    np.testing.assert_allclose(om.topic_first_moment(X), M1, atol=1e-14)
    np.testing.assert_allclose(om.topic_pair_moment(X), P2, atol=1e-14)
    np.testing.assert_allclose(om.topic_triple_moment(X), E3, atol=1e-14)


def _rising(x, n):
    out = 1.0
    for i in range(n):
        out *= x + i
    return out


def _dirichlet_moment(alpha, counts):
    """E[prod_i h_i^{n_i}] for h ~ Dir(alpha): prod_i alpha_i^(n_i) / alpha0^(N)."""
    num = 1.0
    for a, c in zip(alpha, counts):
        num *= _rising(a, c)
    return num / _rising(sum(alpha), sum(counts))


def _population_corpus(mu, alpha, lengths):
    """Every word sequence of the given lengths, weighted by its exact LDA probability."""
    d, k = mu.shape
    docs, weights = [], []
    for L, share in lengths:
        for seq in itertools.product(range(d), repeat=L):
            p = 0.0
            for z in itertools.product(range(k), repeat=L):
                counts = np.bincount(np.array(z), minlength=k)
                p += np.prod([mu[seq[i], z[i]] for i in range(L)]) * _dirichlet_moment(alpha, counts)
            docs.append(list(seq))
            weights.append(share * p)
    return docs, np.array(weights)


@pytest.mark.parametrize("alpha", [[0.3, 0.5], [1.2, 0.4]])
def test_topic_lemma1_exact_population(alpha):
    """Lemma 1: under exact expectation, M1 = sum a_i mu_i, M2 = sum a_i mu_i mu_i^T,
    M3 = sum a_i mu_i^(x)3 with a_i = alpha_i/alpha0 (mixed document lengths)."""
    g = np.random.default_rng(7)
    d, k = 3, 2
    mu = g.dirichlet(np.ones(d), size=k).T
    alpha = np.array(alpha)
    a0 = alpha.sum()
    ah = alpha / a0
    docs, w = _population_corpus(mu, alpha, [(3, 0.6), (4, 0.4)])
    assert abs(w.sum() - 1.0) < 1e-12
    X = _docs_to_csr(docs, d)
    np.testing.assert_allclose(om.topic_first_moment(X, w), mu @ ah, atol=1e-13)
    np.testing.assert_allclose(om.topic_second_moment(X, a0, w), (mu * ah) @ mu.T, atol=1e-13)
    M3 = np.einsum("i,ai,bi,ci->abc", ah, mu, mu, mu)
    np.testing.assert_allclose(om.topic_third_moment(X, a0, w), M3, atol=1e-13)


def test_topic_second_moment_apply_matches_dense():
    c = synth.lda_corpus(3, 60, 12, 3, 0.2, 0.5, 9, poisson_len=True)
    S = np.random.default_rng(0).standard_normal((12, 5))
    dense = om.topic_second_moment(c["X"], 0.7) @ S
    np.testing.assert_allclose(om.topic_second_moment_apply(c["X"], S, 0.7), dense, atol=1e-13)


def _expected_graph(seed, n, k, alpha):
    """Edges replaced by their expectation given memberships: G_{x,Y}^T = F_Y pi_x."""
    g = np.random.default_rng(seed)
    Pi = {p: g.dirichlet(alpha, size=n) for p in "XABC"}
    P = g.uniform(0.1, 0.9, size=(k, k))
    G = {p: Pi["X"] @ P @ Pi[p].T for p in "ABC"}
    F = {p: Pi[p] @ P.T for p in "ABC"}
    return Pi, P, G, F


def test_community_moments_lemma2_factorisation():
    """Eqs. (7)-(11) on expected graphs reduce to the factorised form of Lemma 2:
    with F_A = Pi_A P^T, H = E_x[pi pi^T], pbar = E_x[pi]:
    M2 = (a0+1) F_A H F_A^T - a0 F_A pbar pbar^T F_A^T, and
    M3 = c1 E_x[(F_A pi)^(x)3] - c2 E_x[(F_A pi)(x)(F_A pi)(x)M1 + perms] + c3 M1^(x)3."""
    k, n, a0 = 3, 10, 0.9
    alpha = np.full(k, a0 / k)
    Pi, P, G, F = _expected_graph(11, n, k, alpha)
    Y = Pi["X"] @ F["A"].T                    # rows: (F_A pi_x)^T
    H = Pi["X"].T @ Pi["X"] / n
    pbar = Pi["X"].mean(axis=0)
    M1 = F["A"] @ pbar
    np.testing.assert_allclose(om.community_first_moment(G["A"]), M1, atol=1e-13)
    M2 = (a0 + 1) * F["A"] @ H @ F["A"].T - a0 * np.outer(M1, M1)
    np.testing.assert_allclose(om.community_second_moment(G["A"], G["B"], G["C"], k, a0), M2,
                               atol=1e-11)
    c1, c2, c3 = (a0 + 1) * (a0 + 2) / 2, a0 * (a0 + 1) / 2, a0 ** 2
    E = np.einsum("xi,xj,xk->ijk", Y, Y, Y) / n
    S = (np.einsum("xi,xj,k->ijk", Y, Y, M1) + np.einsum("xi,j,xk->ijk", Y, M1, Y)
         + np.einsum("i,xj,xk->ijk", M1, Y, Y)) / n
    M3 = c1 * E - c2 * S + c3 * np.einsum("i,j,k->ijk", M1, M1, M1)
    np.testing.assert_allclose(om.community_third_moment(G["A"], G["B"], G["C"], k, a0), M3,
                               atol=1e-11)


def test_dirichlet_pair_identity_makes_lemma2_diagonal():
    """Appendix B: E[pi_i^2] = a_i(a_i+1)/(a0(a0+1)), E[pi_i pi_j] = a_i a_j/(a0(a0+1)),
    hence (a0+1) E[pi pi^T] - a0 E[pi] E[pi]^T = diag(alpha/alpha0)."""
    alpha = np.array([0.2, 0.7, 1.1])
    a0 = alpha.sum()
    H = np.array([[_dirichlet_moment(alpha, np.eye(3, dtype=int)[i] + np.eye(3, dtype=int)[j])
                   for j in range(3)] for i in range(3)])
    m = alpha / a0
    np.testing.assert_allclose((a0 + 1) * H - a0 * np.outer(m, m), np.diag(m), atol=1e-14)
    g = np.random.default_rng(5).dirichlet(alpha, size=400000)
    np.testing.assert_allclose(g.T @ g / g.shape[0], H, atol=3e-3)


def test_coefficients_values():
    assert om.coefficients(1.0) == (3.0, 1.0, 1.0)
    assert om.coefficients(0.0) == (1.0, 0.0, 0.0)
    assert math.isclose(om.coefficients(0.5)[0], 1.5 * 2.5 / 2)
