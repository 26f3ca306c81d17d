"""CPU pins of the oracle's stochastic tensor gradient descent (Section 3.2,
Lemma 3, Appendix A) and post-processing (Section 3.3, Lemma 4)."""
import itertools

import numpy as np
import pytest

import synth
from oracle import moments as om
from oracle import post, stgd
from oracle import whiten as ow


def _samples(seed, n, k):
    g = np.random.default_rng(seed)
    Y = g.standard_normal((n, k)) + 0.3
    return Y, Y.mean(axis=0)


@pytest.mark.parametrize("alpha0,theta", [(0.0, 1.0), (1.0, 1.0), (0.6, 2.5)])
def test_implicit_gradient_is_third_of_explicit_loss_gradient(alpha0, theta):
    """Symmetric views: Lemma 3's implicit gradient equals (1/3) grad L~ computed
    from the explicit whitened tensor (different code path: einsum over T)."""
    Y, yb = _samples(1, 40, 5)
    V = np.random.default_rng(2).standard_normal((5, 5))
    T = stgd.whitened_tensor(Y, Y, Y, (yb, yb, yb), alpha0)
    G = stgd.grad_implicit(V, Y, Y, Y, (yb, yb, yb), theta, alpha0)
    np.testing.assert_allclose(3.0 * G, stgd.grad_explicit(V, T, theta), rtol=1e-11, atol=1e-11)


def test_explicit_gradient_matches_finite_differences():
    Y, yb = _samples(3, 30, 4)
    T = stgd.whitened_tensor(Y, Y, Y, (yb, yb, yb), 1.0)
    V = np.random.default_rng(4).standard_normal((4, 4))
    G = stgd.grad_explicit(V, T, 1.0)
    h = 1e-5
    FD = np.zeros_like(V)
    for a, b in itertools.product(range(4), range(4)):
        E = np.zeros_like(V)
        E[a, b] = h
        FD[a, b] = (stgd.loss_explicit(V + E, T, 1.0) - stgd.loss_explicit(V - E, T, 1.0)) / (2 * h)
    np.testing.assert_allclose(FD, G, rtol=1e-7, atol=1e-7 * np.abs(G).max())


def test_three_view_data_term_contracts_modes_one_and_two():
    """Three distinct views: the data term of Lemma 3 is T(v_i, v_i, I) of the
    explicit (non-symmetric) whitened tensor."""
    g = np.random.default_rng(5)
    YA, YB, YC = (g.standard_normal((25, 4)) + s for s in (0.1, -0.2, 0.3))
    yb = tuple(Y.mean(axis=0) for Y in (YA, YB, YC))
    V = g.standard_normal((4, 4))
    T = stgd.whitened_tensor(YA, YB, YC, yb, 0.8)
    G0 = stgd.grad_implicit(V, YA, YB, YC, yb, 1.0, 0.8)
    # Gram part alone from a zero-data problem (alpha0 = 0, all samples zero)
    Z = np.zeros_like(YA)
    gram = stgd.grad_implicit(V, Z, Z, Z, (Z[0], Z[0], Z[0]), 1.0, 0.0)
    np.testing.assert_allclose(gram - G0, stgd.contract(T, V), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("views,alpha0,theta", [(1, 1.0, 1.0), (3, 0.8, 1.0), (3, 0.0, 2.0),
                                               (1, 2.5, 0.5)])
def test_matrix_form_gradient_equals_explicit_tensor_contraction(views, alpha0, theta):
    """The matrix form of Lemma 3 (all components at once, products of the
    minibatch matrices) equals kappa V (V^T V)^o2 - T(V, V, I) with T formed
    explicitly by einsum; its SGD run equals the per-component one."""
    g = np.random.default_rng(21 + views)
    Ys = [g.standard_normal((30, 5)) + s for s in (0.2, -0.1, 0.4)]
    if views == 1:
        Ys = [Ys[0]] * 3
    yb = tuple(Y.mean(axis=0) for Y in Ys)
    V = g.standard_normal((5, 5))
    T = stgd.whitened_tensor(*Ys, yb, alpha0)
    G = stgd.grad_implicit_gemm(V, *Ys, yb, theta, alpha0)
    ref = stgd.kappa(theta) * V @ (V.T @ V) ** 2 - stgd.contract(T, V)
    np.testing.assert_allclose(G, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    perm = synth.epoch_permutations(3, 30, 2)
    V1, s1 = stgd.sgd_run(V, *Ys, yb, perm, 8, 0.01, theta, alpha0, snapshot_every=3)
    V2, s2 = stgd.sgd_run(V, *Ys, yb, perm, 8, 0.01, theta, alpha0, snapshot_every=3, gemm=True)
    np.testing.assert_allclose(V2, V1, rtol=1e-12, atol=1e-12)
    assert len(s1) == len(s2) == 2


def _orthogonal_atoms(seed, k):
    """Samples whose empirical third moment is exactly sum_i lam_i u_i^(x)3."""
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((k, k)))
    lam = g.uniform(1.5, 3.0, k)
    Y = ((k * lam) ** (1.0 / 3.0) * U).T
    return Y, U, lam


def test_stationary_point_of_orthogonal_tensor():
    """alpha0 = 0 (c1 = 1): T = sum lam_i u_i^(x)3 and V* = [(lam_i/kappa)^(1/3) u_i]
    has zero gradient (closed form)."""
    Y, U, lam = _orthogonal_atoms(6, 5)
    yb = Y.mean(axis=0)
    for theta in (1.0, 3.0):
        Vs = (lam / stgd.kappa(theta)) ** (1.0 / 3.0) * U
        G = stgd.grad_implicit(Vs, Y, Y, Y, (yb, yb, yb), theta, 0.0)
        assert np.abs(G).max() < 1e-12
        np.testing.assert_allclose(post.eigenvalues(Vs, theta), lam, rtol=1e-12)


def test_alpha0_zero_is_plain_third_moment():
    Y, yb = _samples(7, 20, 3)
    T = stgd.whitened_tensor(Y, Y, Y, (yb, yb, yb), 0.0)
    brute = np.zeros((3, 3, 3))
    for y in Y:
        for a, b, c in itertools.product(range(3), repeat=3):
            brute[a, b, c] += y[a] * y[b] * y[c] / len(Y)
    np.testing.assert_allclose(T, brute, atol=1e-12)


def test_whitened_tensor_equals_whitened_eq11_on_expected_graph():
    """Section 3.2's sample form of T (means of each view) equals Eq. (11)
    multilinearly whitened, M3(W, W, W), when the views coincide (expected graph)."""
    k, n, a0 = 3, 12, 0.7
    g = np.random.default_rng(8)
    Pi = {p: g.dirichlet(np.full(k, a0 / k), size=n) for p in "XABC"}
    P = g.uniform(0.1, 0.9, size=(k, k))
    G = {p: Pi["X"] @ P @ Pi[p].T for p in "ABC"}
    M2 = om.community_second_moment(G["A"], G["B"], G["C"], k, a0)
    W = ow.whiten_exact(0.5 * (M2 + M2.T), k)["W"]
    Z_B, Z_C = om.transition_matrices(G["A"], G["B"], G["C"], k)
    YA, YB, YC = G["A"] @ W, G["B"] @ Z_B.T @ W, G["C"] @ Z_C.T @ W
    yb = tuple(Y.mean(axis=0) for Y in (YA, YB, YC))
    T = stgd.whitened_tensor(YA, YB, YC, yb, a0)
    M3 = om.community_third_moment(G["A"], G["B"], G["C"], k, a0)
    np.testing.assert_allclose(T, np.einsum("abc,ai,bj,ck->ijk", M3, W, W, W), atol=1e-9)


def test_sgd_converges_locally_to_exact_decomposition():
    """Full-batch STGD started near the decomposition converges to it (error -> 0)."""
    k = 6
    Y, U, lam = _orthogonal_atoms(0, k)
    yb = Y.mean(axis=0)
    V0 = lam ** (1.0 / 3.0) * U + 0.1 * np.random.default_rng(1).standard_normal((k, k))
    V, _ = stgd.sgd_run(V0, Y, Y, Y, (yb, yb, yb), np.tile(np.arange(k), (300, 1)), k, 0.2,
                        1.0, 0.0)
    assert post.recon_error_from_V(V, 1.0, lam, U) < 1e-6
    perm, signs, err = post.match_components(V, U)
    assert err < 1e-5


def test_sgd_schedule_steps_and_partial_batch():
    """beta_t = beta0/sqrt(t) with t counted over the whole run; a partial last
    batch is one step averaged over its own size."""
    Y, yb = _samples(9, 10, 3)
    V0 = np.eye(3)
    perm = np.stack([np.arange(10), np.arange(10)[::-1]])
    V, _ = stgd.sgd_run(V0, Y, Y, Y, (yb, yb, yb), perm, 4, 0.01, 1.0, 0.5)
    Vm = V0.copy()
    t = 0
    for order in perm:
        for s in (0, 4, 8):
            t += 1
            idx = order[s:s + 4]
            Vm = Vm - 0.01 / np.sqrt(t) * stgd.grad_implicit(Vm, Y[idx], Y[idx], Y[idx],
                                                             (yb, yb, yb), 1.0, 0.5)
    assert t == 2 * stgd.steps_per_epoch(10, 4) == 6
    np.testing.assert_allclose(V, Vm, atol=1e-14)


def test_unwhiten_recovers_topics_from_population():
    """Population topic model: whiten M2 = mu diag(a) mu^T, decompose
    M3(W,W,W) = sum a_i^{-1/2} u_i^(x)3 exactly; Lemma 4 returns mu and alpha/alpha0."""
    g = np.random.default_rng(10)
    d, k = 9, 3
    mu = g.dirichlet(np.ones(d) * 0.7, size=k).T
    ah = np.array([0.2, 0.3, 0.5])
    M2 = (mu * ah) @ mu.T
    wh = ow.whiten_exact(M2, k)
    Umat = np.sqrt(ah) * (wh["W"].T @ mu)
    np.testing.assert_allclose(Umat.T @ Umat, np.eye(k), atol=1e-10)
    lam = ah ** -0.5
    for theta in (1.0, 2.0):
        Vs = (lam / stgd.kappa(theta)) ** (1.0 / 3.0) * Umat
        out = post.unwhiten(Vs, wh["Wplus"], theta, normalize=True)
        np.testing.assert_allclose(out["mu"], mu, atol=1e-10)
        np.testing.assert_allclose(out["alpha_hat"], ah, atol=1e-10)
        np.testing.assert_allclose(out["raw"], mu, atol=1e-10)
    # sign flip of a component is undone by the simplex normalisation
    out = post.unwhiten(-Vs, wh["Wplus"], 2.0, normalize=True)
    np.testing.assert_allclose(out["mu"], mu, atol=1e-10)


def test_recon_error_closed_form_matches_explicit_tensor():
    g = np.random.default_rng(11)
    k = 4
    lt, Ut = g.uniform(1, 3, k), g.standard_normal((k, k))
    lh, Uh = g.uniform(1, 3, k), g.standard_normal((k, k))
    Ut /= np.linalg.norm(Ut, axis=0)
    Uh /= np.linalg.norm(Uh, axis=0)
    Tt = post.tensor_from_components(lt, Ut)
    Th = post.tensor_from_components(lh, Uh)
    ref = np.linalg.norm(Th - Tt) / np.linalg.norm(Tt)
    assert abs(post.recon_error(lh, Uh, lt, Ut) - ref) < 1e-12
    assert post.recon_error(lt, Ut, lt, Ut) < 1e-7


def test_match_components_inverts_permutation_and_signs():
    g = np.random.default_rng(12)
    U, _ = np.linalg.qr(g.standard_normal((6, 6)))
    p = g.permutation(6)
    s = np.array([1, -1, 1, -1, -1, 1.0])
    Uh = np.empty_like(U)
    Uh[:, p] = U * s
    perm, signs, err = post.match_components(Uh, U)
    assert err < 1e-12
    np.testing.assert_array_equal(perm, p)
    np.testing.assert_array_equal(signs, s)


# --- exact self-token corrections (topic model, Eq. (3) kept whole) ---------

def _tiny_corpus(seed, n, d, lengths):
    """Count rows with the given document lengths (some below 3 on purpose)."""
    g = np.random.default_rng(seed)
    dense = np.zeros((n, d))
    for t in range(n):
        words = g.integers(0, d, size=lengths[t % len(lengths)])
        np.add.at(dense[t], words, 1.0)
    return synth.csr_from_dense(dense)


@pytest.mark.parametrize("alpha0,theta", [(0.0, 1.0), (1.0, 1.0), (0.7, 2.0)])
def test_exact_topic_gradient_is_third_of_explicit_eq3_gradient(alpha0, theta):
    """The implicit per-document formula equals (1/3) grad L~ of the explicit
    whitened tensor M3(W, W, W), with M3 from the brute-force-pinned Eq. (3)
    moments of the same documents (lengths 1 and 2 included: they add nothing
    to the terms they are too short for)."""
    d, k = 9, 4
    X = _tiny_corpus(3, 25, d, [1, 2, 3, 5, 8, 13])
    g = np.random.default_rng(4)
    W = g.standard_normal((d, k))
    V = g.standard_normal((k, k))
    M3 = om.topic_third_moment(X, alpha0)
    T = np.einsum("abc,ai,bj,ck->ijk", M3, W, W, W)
    G = stgd.grad_implicit_topic_exact(V, X, W, om.topic_first_moment(X), theta, alpha0)
    np.testing.assert_allclose(3.0 * G, stgd.grad_explicit(V, T, theta), rtol=1e-11,
                               atol=1e-11)


def test_exact_topic_gradient_approaches_sample_tensor_for_long_documents():
    """The self-token terms are O(1/l): for documents of l words the exact
    gradient and the sample-tensor gradient of Section 3.2 (y = W^T c / l)
    differ by a relative amount that shrinks like 1/l."""
    d, k, alpha0, theta = 30, 4, 1.0, 1.0
    g = np.random.default_rng(5)
    W = g.standard_normal((d, k))
    V = g.standard_normal((k, k))
    gaps = []
    for L in (50, 400):
        X = _tiny_corpus(6, 40, d, [L])
        M1 = om.topic_first_moment(X)
        Y = (om.as_sparse(X) @ W) / L
        yb = W.T @ M1
        G_exact = stgd.grad_implicit_topic_exact(V, X, W, M1, theta, alpha0)
        G_samp = stgd.grad_implicit(V, Y, Y, Y, (yb, yb, yb), theta, alpha0)
        gaps.append(np.linalg.norm(G_exact - G_samp) / np.linalg.norm(G_samp))
    assert gaps[1] < gaps[0] / 4.0                # 8x longer documents: ~8x smaller
    assert gaps[1] < 5e-2


def test_exact_topic_gradient_in_gathered_gemm_form():
    """The form a kernel would evaluate (all word occurrences e = (t, j) of the
    minibatch at once): gathered rows W_g (nnz x k), U_e = W_j V, per-document
    S = Y' V and q; then the self-token terms are ONE product W_g^T Coef with
    Coef_e = c_e U_e (2 w2_t mu - 2 w3_t S_t) + 2 w3_t c_e U_e^2, the sample terms
    Y'^T A with A_t = w3_t (S_t^2 - q_t) - 2 w2_t mu S_t, plus m terms.  Checked
    against the oracle's per-document loop (FP64)."""
    from oracle.moments import coefficients
    d, k, alpha0, theta = 20, 5, 0.8, 1.5
    X = _tiny_corpus(8, 30, d, [1, 2, 4, 7, 12])
    g = np.random.default_rng(9)
    W = g.standard_normal((d, k))
    V = g.standard_normal((k, k))
    M1 = om.topic_first_moment(X) + 0.01
    c1, c2, c3 = coefficients(alpha0)
    Xs = om.as_sparse(X)
    b = Xs.shape[0]
    rows = np.repeat(np.arange(b), np.diff(Xs.indptr))       # document of each occurrence
    cols, cnt = Xs.indices, Xs.data
    l = np.asarray(Xs.sum(axis=1)).ravel()
    w3 = np.where(l >= 3, c1 / np.maximum(l * (l - 1) * (l - 2), 1), 0.0)
    w2 = np.where(l >= 2, c2 / np.maximum(l * (l - 1), 1), 0.0)
    Wg = W[cols]                                              # nnz x k
    U = Wg @ V                                                # U_e[i] = <W_j, v_i>
    Yp = Xs @ W                                               # b x k, rows y'_t
    S = Yp @ V                                                # S[t, i] = <y'_t, v_i>
    q = np.zeros((b, k))
    np.add.at(q, rows, cnt[:, None] * U * U)
    m = W.T @ M1
    mu = m @ V                                                # mu_i = <m, v_i>
    coef = (cnt[:, None] * U * (2 * w2[rows, None] * mu - 2 * w3[rows, None] * S[rows])
            + 2 * w3[rows, None] * cnt[:, None] * U * U)
    A = w3[:, None] * (S * S - q) - 2 * w2[:, None] * mu * S
    data = (Wg.T @ coef + Yp.T @ A - np.outer(m, (w2[:, None] * (S * S - q)).sum(axis=0))) / b
    data += c3 * m[:, None] * mu ** 2
    Gm = V.T @ V
    G = stgd.kappa(theta) * V @ (Gm ** 2) - data
    np.testing.assert_allclose(G, stgd.grad_implicit_topic_exact(V, X, W, M1, theta, alpha0),
                               rtol=1e-11, atol=1e-11)


def test_exact_topic_run_is_the_schedule_over_the_exact_gradient():
    """sgd_run_topic_exact visits perm[e][s:s+b] with beta0/sqrt(t) and the
    gradient of grad_implicit_topic_exact; an index outside [0, n) is an empty
    document (it counts in the minibatch mean and adds nothing)."""
    corp = synth.lda_corpus(31, 30, 20, 3, 0.3, 0.3, 6, poisson_len=True)
    X = corp["X"]
    g = np.random.default_rng(32)
    W = g.standard_normal((20, 3))
    M1 = om.topic_first_moment(X)
    V0 = g.standard_normal((3, 3))
    perm = synth.epoch_permutations(33, 30, 2).copy()
    perm[1, 4] = -1
    V, snaps = stgd.sgd_run_topic_exact(V0, X, W, M1, perm, 8, 0.05, 1.0, 0.7, snapshot_every=4)
    Xs = om.as_sparse(X)
    Vm, t = V0.copy(), 0
    for e in range(2):
        for s in range(0, 30, 8):
            t += 1
            idx = perm[e][s:s + 8]
            rows = [Xs[i] if 0 <= i < 30 else None for i in idx]
            Xb = om.as_sparse(np.vstack([r.toarray() if r is not None else np.zeros((1, 20))
                                         for r in rows]))
            Vm = Vm - 0.05 / np.sqrt(t) * stgd.grad_implicit_topic_exact(Vm, Xb, W, M1, 1.0, 0.7)
    np.testing.assert_allclose(V, Vm, rtol=1e-12, atol=1e-12)
    assert len(snaps) == 2


@pytest.mark.parametrize("views,alpha0", [(1, 1.0), (3, 0.6), (1, 0.0)])
def test_chunked_tensor_and_matrix_contraction_equal_the_definitions(views, alpha0):
    """whitened_tensor_chunked (matrix products over sample chunks) equals the
    einsum definition; contract_all (Khatri-Rao form) equals contract."""
    g = np.random.default_rng(41 + views)
    Ys = [g.standard_normal((77, 6)) + s for s in (0.2, -0.3, 0.1)]
    if views == 1:
        Ys = [Ys[0]] * 3
    yb = tuple(Y.mean(axis=0) for Y in Ys)
    T = stgd.whitened_tensor(*Ys, yb, alpha0)
    np.testing.assert_allclose(stgd.whitened_tensor_chunked(*Ys, yb, alpha0, chunk=10), T,
                               rtol=1e-12, atol=1e-12)
    V = g.standard_normal((6, 6))
    np.testing.assert_allclose(stgd.contract_all(T, V), stgd.contract(T, V), rtol=1e-12,
                               atol=1e-12)
