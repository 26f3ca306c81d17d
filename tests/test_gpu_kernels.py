"""GPU parity of the individual C-ABI calls against the FP64 oracle.

Inputs come from ``synth`` (seeded) and are fed to both sides; expected values
come only from ``oracle``.  Tolerances follow from the arithmetic of each
kernel (float32 storage and FMAs, FP64 where the call promises FP64) and are
stated at each assertion.
"""
import numpy as np
import pytest

import synth
from oracle import moments as om
from oracle import post as opost
from oracle import stgd as ostgd
from tests._util import align_signs, grad_errs, rel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def otm():
    from paper_1309_0787_gb300 import otm as _otm
    return _otm


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _corpus(seed, n, d, k, L, poisson=True):
    return synth.lda_corpus(seed, n, d, k, 0.1, 0.2, L, poisson_len=poisson)


# ----------------------------------------------------------------------------
# moments, projection, sparse products
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,d,L", [(2000, 500, 100), (333, 97, 3), (50, 40, 1)])
def test_topic_moments(otm, n, d, L):
    X = _corpus(1, n, d, 10, L)["X"]
    # include an empty document and a one-word document
    dense = synth.csr_to_dense(X)
    dense[0] = 0.0
    dense[1] = 0.0
    dense[1, 3] = 1.0
    X = synth.csr_from_dense(dense)
    out = otm.topic_moments(otm.DeviceCSR.from_host(X))
    torch.cuda.synchronize()
    l = om.doc_lengths(X)
    # FP64 sums of exact integer counts: only summation order differs
    np.testing.assert_allclose(to_np(out["M1"]), om.topic_first_moment(X), rtol=1e-12, atol=1e-15)
    w = om.topic_pair_weights(l)
    np.testing.assert_allclose(to_np(out["delta"]), om.as_sparse(X).T @ w / n, rtol=1e-12,
                               atol=1e-15)
    # float32 outputs: one rounding of the FP64 value
    np.testing.assert_allclose(to_np(out["row_w"]), w, rtol=1e-7)
    np.testing.assert_allclose(to_np(out["row_invlen"]),
                               np.where(l > 0, 1 / np.maximum(l, 1), 0), rtol=1e-7)


@pytest.mark.parametrize("n,d,k", [(2000, 500, 10), (1001, 300, 100), (257, 50, 7),
                                   (300, 200, 130), (64, 30, 1)])
def test_project(otm, n, d, k):
    X = _corpus(2, n, d, 5, 40)["X"]
    W = synth.gaussian(3, d, k)
    scale = synth.gaussian(4, n, 1).ravel()
    Xd = otm.DeviceCSR.from_host(X)
    Y = otm.project(Xd, _dev(W), _dev(scale))
    Y0 = otm.project(Xd, _dev(W))
    torch.cuda.synchronize()
    ref = om.as_sparse(X) @ W.astype(np.float64)
    # float32 FMAs over <= l_t terms: relative error well below 1e-6 normwise
    assert rel(to_np(Y0), ref) < 1e-6
    assert rel(to_np(Y), ref * scale[:, None].astype(np.float64)) < 1e-6


@pytest.mark.parametrize("m", [30, 120, 13])
def test_topic_m2_apply(otm, m):
    c = _corpus(5, 1500, 300, 8, 60)
    X = c["X"]
    S = synth.gaussian(6, 300, m)
    Xd = otm.DeviceCSR.from_host(X)
    mom = otm.topic_moments(Xd)
    O = otm.topic_m2_apply(Xd, mom, 1.0, _dev(S))
    torch.cuda.synchronize()
    ref = om.topic_second_moment_apply(X, S.astype(np.float64), 1.0)
    # float32 products and atomics; the result is a difference of terms of the
    # same size as itself (pair moment minus diagonal), so ~1e-6 normwise
    assert rel(to_np(O), ref) < 1e-5


@pytest.mark.parametrize("m", [32, 120, 200])
def test_topic_m2_apply_over_transpose(otm, m):
    """X^T P as a gather over the transpose (the form the topic whitening uses)
    against the oracle: 3,000 documents with word 0 in every one (a column
    spread over a dozen warps of 256 nonzeros, summed with atomics), words 1-9
    in none (empty columns), empty and one-word documents, m of one to two
    float4 per lane."""
    c = _corpus(15, 3000, 400, 8, 40)
    dense = synth.csr_to_dense(c["X"])
    dense[:, 0] += 2.0
    dense[:, 1:10] = 0.0
    dense[5] = 0.0
    dense[6] = 0.0
    dense[6, 17] = 1.0
    X = synth.csr_from_dense(dense)
    S = synth.gaussian(16, 400, m)
    Xd = otm.DeviceCSR.from_host(X)
    mom = otm.topic_moments(Xd)
    Xt = otm.csr_transpose(Xd)
    O = otm.topic_m2_apply(Xd, mom, 1.0, _dev(S), Xt=Xt)
    torch.cuda.synchronize()
    ref = om.topic_second_moment_apply(X, S.astype(np.float64), 1.0)
    assert rel(to_np(O), ref) < 1e-5
    # every row (word) on its own, the empty ones included
    err = np.linalg.norm(to_np(O) - ref, axis=1)
    assert np.all(err <= 1e-5 * np.linalg.norm(ref, axis=1) + 1e-6 * np.linalg.norm(ref) / 20)


def _check_transpose(otm, X):
    sp = pytest.importorskip("scipy.sparse")
    Xt = otm.csr_transpose(otm.DeviceCSR.from_host(X))
    torch.cuda.synchronize()
    n, d = X.shape
    ref = sp.csr_matrix((X.val, X.col, X.row_ptr), shape=X.shape).T.tocsr()
    ref.sort_indices()
    cp, rt, vt = to_np(Xt.row_ptr), to_np(Xt.col), to_np(Xt.val)
    assert Xt.shape == (d, n)
    np.testing.assert_array_equal(cp, ref.indptr)
    # per word the (document, count) pairs as a set: order them by document
    key = np.repeat(np.arange(d, dtype=np.int64), np.diff(cp)) * (n + 1) + rt
    o = np.argsort(key, kind="stable")
    np.testing.assert_array_equal(rt[o], ref.indices)
    np.testing.assert_array_equal(vt[o], ref.data)


@pytest.mark.parametrize("n", [2000, 5000])
def test_csr_transpose_matches_scipy(otm, n):
    """colptr exact; per word the (document, count) pairs as a set (their order
    within a word is not fixed); 5,000 documents span three row blocks of the
    counting sort."""
    c = _corpus(17, n, 300, 6, 50)
    dense = synth.csr_to_dense(c["X"])
    dense[:, 3] = 1.0          # a word in every document
    dense[:, 7] = 0.0          # a word in none
    dense[11] = 0.0            # an empty document
    _check_transpose(otm, synth.csr_from_dense(dense))


def test_csr_transpose_in_word_phases(otm):
    """A corpus whose transpose (8 bytes per entry) is larger than 96 MB, so that
    the placement pass runs in two phases over ranges of words: 100,000
    documents of Poisson(150) words over 20,000 words (about 14 M entries), word 3
    in every document, word 7 in none, document 11 empty."""
    sp = pytest.importorskip("scipy.sparse")
    n, d = 100000, 20000
    X = _corpus(23, n, d, 8, 150)["X"]
    Xs = sp.csr_matrix((X.val.astype(np.float64), X.col, X.row_ptr), shape=(n, d))
    Xs = Xs + sp.csr_matrix((np.ones(n), (np.arange(n), np.full(n, 3))), shape=(n, d))
    cmask = np.ones(d)
    cmask[7] = 0.0
    rmask = np.ones(n)
    rmask[11] = 0.0
    Xs = (sp.diags(rmask) @ Xs @ sp.diags(cmask)).tocsr()
    Xs.eliminate_zeros()
    Xs.sort_indices()
    assert Xs.nnz * 8 > 96 << 20
    _check_transpose(otm, synth.CSR(Xs.indptr, Xs.indices, Xs.data, (n, d)))


def test_csr_transpose_word_ranges_capped(otm):
    """60,000 words, more than the 49,152 cursors of one placement phase: two
    phases by the word cap although the corpus is small (4,000 documents of 50
    words, uniform over the vocabulary; words 0, 49,151, 49,152 and 59,999, the
    edges of the phases, in every document)."""
    g = np.random.default_rng(29)
    n, d, per = 4000, 60000, 50
    edges = np.array([0, 49151, 49152, 59999])
    pool = np.setdiff1d(np.arange(d), edges)
    cols = np.stack([np.sort(np.concatenate([edges, g.choice(pool, per - 4, replace=False)]))
                     for _ in range(n)])
    row_ptr = np.arange(n + 1, dtype=np.int64) * per
    X = synth.CSR(row_ptr, cols.reshape(-1), g.integers(1, 5, n * per).astype(np.float64), (n, d))
    _check_transpose(otm, X)


def test_csr_transpose_wide_vocabulary(otm):
    """A vocabulary too wide for the per-block counts in shared memory (150,000
    words): the transpose takes one atomic position per entry, same result."""
    g = np.random.default_rng(19)
    n, d, per = 3000, 150000, 40
    cols = np.sort(np.stack([g.choice(d, per, replace=False) for _ in range(n)]), axis=1)
    cols[:, 0] = 0             # a word in every document
    cols = np.sort(cols, axis=1)
    row_ptr = np.arange(n + 1, dtype=np.int64) * per
    X = synth.CSR(row_ptr, cols.reshape(-1), g.integers(1, 4, n * per).astype(np.float64),
                  (n, d))
    _check_transpose(otm, X)


def test_pairs_apply(otm):
    g = synth.mmsb_graph(7, 600, 8, 0.05, 0.3, 0.02)
    S = synth.gaussian(8, 600, 28)
    A, B = (otm.DeviceCSR.from_host(g[x]) for x in ("G_XC", "G_XB"))
    O = otm.pairs_apply(A, B, _dev(S))
    torch.cuda.synchronize()
    ref = om.pairs(g["G_XC"], g["G_XB"]) @ S.astype(np.float64)
    assert rel(to_np(O), ref) < 1e-6


# ----------------------------------------------------------------------------
# dense kernels of the whitening
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("rows,m,cond", [(5000, 120, 1e2), (500, 30, 1e5), (161, 160, 10.0),
                                         (40, 1, 1.0), (3000, 77, 1e6), (2000, 64, 1e3),
                                         (1000, 128, 1e2), (33, 4, 1.0)])
def test_orthonormalize(otm, rows, m, cond):
    g = np.random.default_rng(9)
    U, _ = np.linalg.qr(g.standard_normal((rows, m)))
    Vt, _ = np.linalg.qr(g.standard_normal((m, m)))
    A = (U * np.geomspace(1.0, 1.0 / cond, m)) @ Vt
    At = _dev(A.astype(np.float32))
    otm.orthonormalize(At)
    torch.cuda.synchronize()
    Q = to_np(At).astype(np.float64)
    # float32 Cholesky-QR after the shifted first pass: orthogonality O(m u)
    assert np.abs(Q.T @ Q - np.eye(m)).max() < 2e-5
    # same column space as A
    assert rel(Q @ (Q.T @ A), A) < 1e-5 * max(1.0, np.log10(cond))


def _sym(seed, n, spread=1e3, clusters=False):
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.geomspace(1.0, 1.0 / spread, n) * np.where(g.random(n) < 0.2, -1, 1)
    if clusters and n >= 6:
        lam[1:4] = lam[1]
    return (U * lam) @ U.T


@pytest.mark.parametrize("n,spread,clusters", [(120, 1e3, False), (30, 1e6, False),
                                               (77, 10.0, True), (160, 1e2, False), (1, 1, False),
                                               (2, 5.0, False)])
def test_syev_fp64(otm, n, spread, clusters):
    A = _sym(10 + n, n, spread, clusters)
    ev, vec = otm.syev(_dev(A))
    torch.cuda.synchronize()
    ev, vec = to_np(ev), to_np(vec)
    ref = np.sort(np.linalg.eigvalsh(A))[::-1]
    scale = np.abs(ref).max()
    # FP64-accurate after refinement for eigenvalues separated from their
    # neighbours by more than the float32 starting point resolves (1e-5 ||A||);
    # closer groups keep an FP64-exact invariant subspace, their eigenvalues
    # are resolved to ~1e-9 ||A||.
    gap = np.minimum(np.abs(np.diff(ref, prepend=np.inf)), np.abs(np.diff(ref, append=-np.inf)))
    sep = gap > 1e-5 * scale
    assert np.abs(ev - ref)[sep].max(initial=0.0) < 1e-12 * scale
    assert np.abs(ev - ref).max() < 1e-9 * scale
    # six FP64 refinement steps: orthonormal to ~1e-12 even when float32 mixed
    # near-degenerate groups at the start
    assert np.abs(vec.T @ vec - np.eye(n)).max() < 1e-11
    H = vec.T @ A @ vec
    close = np.abs(ev[:, None] - ev[None, :]) <= 1e-5 * scale
    assert np.abs(np.where(close, 0.0, H)).max() < 1e-12 * scale
    # sign convention: largest-magnitude entry of every eigenvector positive
    idx = np.argmax(np.abs(vec), axis=0)
    assert np.all(vec[idx, np.arange(n)] > 0)


# ----------------------------------------------------------------------------
# the fused STGD step (Lemma 3)
# ----------------------------------------------------------------------------
def _grad_parts(V, YA, YB, YC, yb, theta, a0):
    G = ostgd.grad_implicit(V, YA, YB, YC, yb, theta, a0)
    gram = ostgd.kappa(theta) * V @ (V.T @ V) ** 2
    return G, gram, gram - G


@pytest.mark.parametrize("k,b,sym,a0", [(10, 256, True, 1.0), (100, 1024, False, 1.0),
                                        (100, 1024, True, 0.0), (17, 33, False, 0.7),
                                        (1, 5, True, 1.0), (128, 1000, False, 2.0),
                                        (64, 1, False, 1.0), (3, 4096, True, 1.0)])
def test_sgd_step_gradient(otm, k, b, sym, a0):
    g = np.random.default_rng(k * 7 + b)
    Ys = [g.standard_normal((b, k)).astype(np.float32) + 0.2 * s for s in (1, -1, 0.5)]
    if sym:
        Ys = [Ys[0]] * 3
    yb = np.stack([Y.astype(np.float64).mean(axis=0) for Y in Ys])
    V0 = (0.5 * g.standard_normal((k, k))).astype(np.float32)     # columns = components
    theta = 1.0
    beta = 1.0
    Yd = [_dev(Y) for Y in Ys]
    if sym:
        Yd = [Yd[0]] * 3
    Vd = _dev(V0.T.copy())                                         # row i = component i
    otm.sgd_step(Vd, Yd[0], Yd[1], Yd[2], _dev(yb), theta, beta, a0)
    torch.cuda.synchronize()
    V1 = to_np(Vd).T.astype(np.float64)
    Gk = (V0.astype(np.float64) - V1) / beta
    G, gram, data = _grad_parts(V0.astype(np.float64), *[Y.astype(np.float64) for Y in Ys],
                                tuple(yb), theta, a0)
    frob, col = grad_errs(Gk, G, gram)
    # FP32 path, tolerance 1e-5 (normwise, relative to the two gradient terms), for the
    # whole matrix and for every component on its own
    assert frob < 1e-5 and col < 1e-5, (frob, col)


def test_sgd_run_matches_oracle_schedule(otm):
    """Several epochs with permutations and a partial last batch, snapshots."""
    k, n, b, epochs = 12, 700, 128, 3
    o = synth.orthogonal_samples(11, k, n, 0.05)
    Y = o["Y"]
    yb = Y.astype(np.float64).mean(axis=0)
    perm = synth.epoch_permutations(12, n, epochs)
    V0 = synth.haar_orthonormal(13, k)
    Vd = _dev(V0.T.copy())
    Yd = _dev(Y)
    snaps = otm.sgd_run(Vd, Yd, Yd, Yd, _dev(np.stack([yb] * 3)), _dev(perm), epochs, b, 2e-3,
                        1.0, 0.0, snapshot_every=6)
    torch.cuda.synchronize()
    Vo, so = ostgd.sgd_run(V0, Y, Y, Y, (yb, yb, yb), perm, b, 2e-3, 1.0, 0.0, snapshot_every=6)
    # 18 float32 steps: rounding differences stay at the 1e-6 level
    assert rel(to_np(Vd).T, Vo) < 1e-5
    assert snaps.shape[0] == len(so) == 3
    for s_gpu, s_ref in zip(to_np(snaps), so):
        assert rel(s_gpu.T, s_ref) < 1e-5


def test_sgd_run_identity_order_and_three_views(otm):
    k, n, b = 20, 300, 64
    g = np.random.default_rng(14)
    Ys = [g.standard_normal((n, k)).astype(np.float32) * 0.3 for _ in range(3)]
    yb = np.stack([Y.astype(np.float64).mean(axis=0) for Y in Ys])
    V0 = synth.haar_orthonormal(15, k)
    Vd = _dev(V0.T.copy())
    otm.sgd_run(Vd, *[_dev(Y) for Y in Ys], _dev(yb), None, 2, b, 1e-2, 1.0, 1.0)
    torch.cuda.synchronize()
    perm = np.tile(np.arange(n, dtype=np.int32), (2, 1))
    Vo, _ = ostgd.sgd_run(V0, *Ys, tuple(yb), perm, b, 1e-2, 1.0, 1.0)
    assert rel(to_np(Vd).T, Vo) < 1e-5


@pytest.mark.parametrize("k,offset", [(100, 0), (128, 0), (37, 0), (64, 1)])
def test_sgd_run_large_batches_three_views(otm, k, offset):
    """Minibatches of 20000 samples (a CTA's slice is longer than its staged row
    indices), a partial last batch, three views; k = 128 runs with one sample
    buffer, k = 37 and views that are not 16-byte aligned take scalar loads."""
    n, b, epochs = 45000, 20000, 1
    g = np.random.default_rng(k + offset)
    Ys = [(g.standard_normal((n, k)) * 0.05 + 0.1 * g.standard_normal(k)).astype(np.float32)
          for _ in range(3)]
    yb = np.stack([Y.astype(np.float64).mean(axis=0) for Y in Ys])
    perm = synth.epoch_permutations(k + 3, n, epochs)
    V0 = synth.haar_orthonormal(k + 4, k)
    Vd = _dev(V0.T.copy())
    views = []
    for Y in Ys:
        buf = torch.zeros(n * k + offset, device="cuda", dtype=torch.float32)
        buf[offset:] = _dev(Y).reshape(-1)
        views.append(buf[offset:].view(n, k))
    otm.sgd_run(Vd, *views, _dev(yb), _dev(perm), epochs, b, 5e-2, 1.0, 1.0)
    torch.cuda.synchronize()
    Vo, _ = ostgd.sgd_run(V0, *Ys, tuple(yb), perm, b, 5e-2, 1.0, 1.0)
    assert rel(to_np(Vd).T, Vo) < 1e-5


# ----------------------------------------------------------------------------
# post-processing and the error measure
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("d,k,kt,normalize", [(500, 10, 30, True), (5000, 100, 120, False),
                                              (77, 5, 5, True)])
def test_unwhiten(otm, d, k, kt, normalize):
    g = np.random.default_rng(d + k)
    Q = np.linalg.qr(g.standard_normal((d, kt)))[0].astype(np.float32)
    Cp = g.standard_normal((kt, k))
    V = (g.standard_normal((k, k)) + 2 * np.eye(k)).astype(np.float32)
    out = otm.unwhiten(_dev(V.T.copy()), _dev(Q), _dev(Cp), 1.0, normalize)
    torch.cuda.synchronize()
    ref = opost.unwhiten(V.astype(np.float64), Q.astype(np.float64) @ Cp, 1.0, normalize)
    # FP64 arithmetic on float32 inputs: agreement to ~1e-12 relative
    assert rel(to_np(out["comps"]), ref["mu"]) < 1e-10
    np.testing.assert_allclose(to_np(out["lambda"]), ref["lambda"], rtol=1e-12)
    np.testing.assert_allclose(to_np(out["alpha_hat"]), ref["alpha_hat"], rtol=1e-12)


def test_unwhiten_product_elementwise(otm):
    """The d x k product Q M of the unwhitening is summed in double-float on the
    FP32 units: every entry within 2^-44 of the sum of its absolute terms
    (|Q| |M|), which a float32 accumulation (about 2^-24 of it) misses by far.
    M = Cp (V / ||v_i||) diag(lambda) in FP64 (Lemma 4); columns of M of very
    different scales and the signs of Q make the sums cancel."""
    g = np.random.default_rng(77)
    d, k, kt = 3000, 30, 40
    Q = np.linalg.qr(g.standard_normal((d, kt)))[0].astype(np.float32)
    Cp = g.standard_normal((kt, k)) * np.exp(3.0 * g.standard_normal((1, k)))
    V = (g.standard_normal((k, k)) + 2 * np.eye(k)).astype(np.float32)
    out = otm.unwhiten(_dev(V.T.copy()), _dev(Q), _dev(Cp), 1.0, False)
    torch.cuda.synchronize()
    Q64, V64 = Q.astype(np.float64), V.astype(np.float64)
    norms = np.linalg.norm(V64, axis=0)
    M = Cp @ (V64 / norms) * (0.5 * (1.0 + 1.0) * norms ** 3)
    ref = Q64 @ M
    np.testing.assert_allclose(ref, opost.unwhiten(V64, Q64 @ Cp, 1.0, False)["mu"],
                               rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    bound = 2.0 ** -44 * (np.abs(Q64) @ np.abs(M)) + 1e-300
    assert np.all(np.abs(to_np(out["comps"]) - ref) <= bound)


@pytest.mark.parametrize("k", [4, 64, 100])
def test_recon_error(otm, k):
    g = np.random.default_rng(k)
    U = np.linalg.qr(g.standard_normal((k, k)))[0]
    lam = g.uniform(1, 3, k)
    V = ((lam ** (1 / 3)) * U + 0.01 * g.standard_normal((k, k))).astype(np.float32)
    err = otm.recon_error(_dev(V.T.copy()), _dev(U.T.copy()), _dev(lam), 1.0)
    torch.cuda.synchronize()
    ref = opost.recon_error_from_V(V.astype(np.float64), 1.0, lam, U)
    assert abs(float(to_np(err)[0]) - ref) < 1e-9 * max(ref, 1e-3)


def test_recon_error_of_diverged_components_is_nan(otm):
    """A diverged iterate (inf or NaN in V) reports NaN, not a clamped zero."""
    k = 8
    g = np.random.default_rng(3)
    U = np.linalg.qr(g.standard_normal((k, k)))[0]
    lam = g.uniform(1, 3, k)
    for bad in (np.inf, np.nan):
        V = (lam ** (1 / 3) * U).astype(np.float32)
        V[2, 5] = bad
        err = otm.recon_error(_dev(V.T.copy()), _dev(U.T.copy()), _dev(lam), 1.0)
        torch.cuda.synchronize()
        assert np.isnan(float(to_np(err)[0]))
