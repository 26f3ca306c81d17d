"""CPU pins of the oracle's whitening (Section 3.1) and randomised low-rank
algebra (Section 4.2, Algorithms 2-3 as read in the oracle's module doc)."""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import moments as om
from oracle import whiten as ow


def _psd(seed, d, r, spread=10.0):
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((d, r)))
    lam = np.geomspace(spread, 1.0, r)
    return (U * lam) @ U.T, lam, U


def test_whiten_exact_identity_and_library_eigh():
    M2, _, _ = _psd(0, 30, 30)
    M2 -= 2.0 * np.eye(30)                      # indefinite, top-k still positive
    wh = ow.whiten_exact(M2, 6)
    np.testing.assert_allclose(wh["W"].T @ M2 @ wh["W"], np.eye(6), atol=1e-10)
    ref = scipy.linalg.eigh(M2, eigvals_only=True, subset_by_index=[24, 29])[::-1]
    np.testing.assert_allclose(wh["eig"], ref, rtol=1e-12)
    # W^+ is the pseudo-inverse of W^T
    np.testing.assert_allclose(wh["Wplus"], np.linalg.pinv(wh["W"].T), atol=1e-10)


def test_whiten_rejects_indefinite():
    M2 = np.diag([3.0, 1.0, -1.0, -2.0])
    with pytest.raises(ow.NotPositiveDefinite):
        ow.whiten_exact(M2, 3)


def test_range_finder_exact_for_low_rank():
    """For an exactly rank-r M2 with r <= k~, the range finder spans range(M2)
    and reproduces the exact whitening (up to column signs)."""
    M2, lam, _ = _psd(1, 80, 12)
    S = synth.gaussian(2, 80, 16, np.float64)
    r = ow.range_finder_whiten(lambda X: M2 @ X, S, 10, 2)
    e = ow.whiten_exact(M2, 10)
    np.testing.assert_allclose(r["eig"], lam[:10], rtol=1e-10)
    s = np.sign(np.sum(r["W"] * e["W"], axis=0))
    np.testing.assert_allclose(r["W"] * s, e["W"], atol=1e-9)
    np.testing.assert_allclose(r["W"].T @ M2 @ r["W"], np.eye(10), atol=1e-10)
    np.testing.assert_allclose(r["Q"].T @ r["Q"], np.eye(16), atol=1e-12)


def test_range_finder_topic_operator_whitens():
    c = synth.lda_corpus(4, 400, 40, 4, 0.25, 0.3, 30)
    X = c["X"]
    M2 = om.topic_second_moment(X, 1.0)
    S = synth.gaussian(5, 40, 14, np.float64)
    r = ow.range_finder_whiten(lambda Z: om.topic_second_moment_apply(X, Z, 1.0), S, 4, 2)
    np.testing.assert_allclose(r["W"].T @ M2 @ r["W"], np.eye(4), atol=1e-6)
    e = ow.whiten_exact(M2, 4)
    # same top-4 eigenvalues as the exact whitening, to the range finder's accuracy
    np.testing.assert_allclose(r["eig"], e["eig"], rtol=1e-6)


def test_randomized_svd_matches_library_svd():
    g = np.random.default_rng(3)
    A = g.standard_normal((50, 5)) @ np.diag([9, 5, 3, 2, 1.0]) @ g.standard_normal((5, 40))
    S = synth.gaussian(6, 40, 9, np.float64)
    U, s, V = ow.randomized_svd(lambda X: A @ X, lambda X: A.T @ X, S, 5, 2)
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False)[:5], rtol=1e-11)
    np.testing.assert_allclose((U * s) @ V.T, A, atol=1e-10)
    np.testing.assert_allclose(U.T @ U, np.eye(5), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-12)


def test_community_randomized_whitening_on_expected_graph():
    """On expected graphs (exact rank k) the randomised community whitening equals
    the exact whitening of the symmetric part of Eq. (10), and the whitened views
    coincide: W_B^T G_{x,B}^T = W^T Z_B G_{x,B}^T = W^T F_A pi_x = W^T G_{x,A}^T."""
    k, n, a0 = 3, 14, 0.8
    g = np.random.default_rng(21)
    Pi = {p: g.dirichlet(np.full(k, a0 / k), size=n) for p in "XABC"}
    P = g.uniform(0.1, 0.9, size=(k, k))
    G = {p: Pi["X"] @ P @ Pi[p].T for p in "ABC"}
    S1 = synth.gaussian(1, n, k + 2, np.float64)
    S2 = synth.gaussian(2, n, k + 2, np.float64)
    r = ow.community_whiten_randomized(G["A"], G["B"], G["C"], k, a0, S1, S2, 2)
    M2 = om.community_second_moment(G["A"], G["B"], G["C"], k, a0)
    M2s = 0.5 * (M2 + M2.T)
    np.testing.assert_allclose(r["apply_M2"](np.eye(n)), M2s, atol=1e-11)
    e = ow.whiten_exact(M2s, k)
    s = np.sign(np.sum(r["W"] * e["W"], axis=0))
    np.testing.assert_allclose(r["W"] * s, e["W"], atol=1e-8)
    YA = G["A"] @ r["W"]
    np.testing.assert_allclose(G["B"] @ r["W_B"], YA, atol=1e-9)
    np.testing.assert_allclose(G["C"] @ r["W_C"], YA, atol=1e-9)


# --- Algorithm 2 (Nystrom form), read as in the oracle's module doc ----------

@pytest.mark.parametrize("kind", ["selection", "gaussian"])
def test_nystrom_whiten_exact_on_rank_k(kind):
    """M2 of rank k: the Nystrom approximation O Omega^+ O^T is exact, so W
    whitens M2 exactly and W W^T is M2's pseudo-inverse (unique, whatever the
    rotation); Omega's eigenvalues from the library; Wplus = pinv(W^T)."""
    d, k, kt = 40, 5, 10
    M2, _, _ = _psd(3, d, k)
    S = (synth.signed_column_selection(4, d, kt) if kind == "selection"
         else synth.gaussian(4, d, kt)).astype(np.float64)
    wh = ow.nystrom_whiten(lambda Z: M2 @ Z, S, k)
    W = wh["W"]
    assert W.shape == (d, k)
    np.testing.assert_allclose(W.T @ M2 @ W, np.eye(k), atol=1e-9)
    P = np.linalg.pinv(M2, rcond=1e-10)
    assert np.linalg.norm(W @ W.T - P) < 1e-9 * np.linalg.norm(P)
    Om = S.T @ M2 @ S
    ref = scipy.linalg.eigh(0.5 * (Om + Om.T), eigvals_only=True,
                            subset_by_index=[kt - k, kt - 1])[::-1]
    np.testing.assert_allclose(wh["eig"], ref, rtol=1e-10)
    np.testing.assert_allclose(wh["Wplus"], np.linalg.pinv(W.T), atol=1e-9)


def test_nystrom_whiten_full_selection_is_exact_whitening():
    """S a signed permutation (k~ = d): Omega is M2 in permuted coordinates and
    the Nystrom W equals the exact whitening of the top-k eigenpairs."""
    d, k = 30, 6
    M2, _, _ = _psd(5, d, d)                   # full rank, distinct eigenvalues
    S = synth.signed_column_selection(6, d, d).astype(np.float64)
    wh = ow.nystrom_whiten(lambda Z: M2 @ Z, S, k)
    ex = ow.whiten_exact(M2, k)
    np.testing.assert_allclose(wh["W"] @ wh["W"].T, ex["W"] @ ex["W"].T, atol=1e-10)
    np.testing.assert_allclose(wh["eig"], ex["eig"], rtol=1e-12)


def test_nystrom_whiten_rejects_indefinite():
    M2, _, _ = _psd(7, 20, 20)
    S = synth.signed_column_selection(8, 20, 8).astype(np.float64)
    with pytest.raises(ow.NotPositiveDefinite):
        ow.nystrom_whiten(lambda Z: -M2 @ Z, S, 3)


def test_nystrom_gram_form_equals_printed_product():
    """The GPU evaluates Algorithm 2 from the eigenpairs of the small Gram
    matrix O^T O instead of an SVD of the tall O: W = O V_G,k diag(1/ev_G)
    V_G,k^T V_Om,k L_Om,k^{1/2} (U_O = O V_O L_O^{-1}), and (W^T)^+ = O C H^{-1}
    with H = C^T (O^T O) C.  Checked here in FP64 against the oracle's printed
    product on an indefinite, full-rank M2 (the general case)."""
    d, k, kt = 60, 6, 14
    g = np.random.default_rng(12)
    A = g.standard_normal((d, d))
    M2 = A @ A.T / d - 0.3 * np.eye(d)
    S = synth.signed_column_selection(13, d, kt).astype(np.float64)
    ref = ow.nystrom_whiten(lambda Z: M2 @ Z, S, k)
    O = M2 @ S
    evG, VG = np.linalg.eigh(O.T @ O)
    evG, VG = evG[::-1][:k], VG[:, ::-1][:, :k]
    lam, VO = ow.top_eigh(S.T @ O, k)
    C = VG @ np.diag(1.0 / evG) @ VG.T @ VO * np.sqrt(lam)
    W = O @ C
    np.testing.assert_allclose(W, ref["W"], rtol=1e-9, atol=1e-12)
    H = C.T @ (O.T @ O) @ C
    np.testing.assert_allclose(O @ C @ np.linalg.inv(H), ref["Wplus"], rtol=1e-8, atol=1e-10)
