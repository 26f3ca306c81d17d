"""GPU parity of the whitening composites and of the whole hot path (whiten ->
project -> STGD -> unwhiten) against the oracle run on the same seeded inputs.

Workloads: the synthetic LDA corpus (d = 500, k = 10, 2,000 documents of 100
words; oracle finishes in seconds) and the synthetic MMSB graph (four parts of
5,000 nodes, k = 100, p = 0.1, q = 0.005), the latter compared at full size on
the outputs the oracle computes directly.
"""
import numpy as np
import pytest

import synth
from oracle import moments as om
from oracle import post as opost
from oracle import stgd as ostgd
from oracle import whiten as ow
from tests._util import align_signs, rel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def otm():
    from paper_1309_0787_gb300 import otm as _otm
    return _otm


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _subspace_gap(A, B):
    """sin of the largest principal angle between span(A) and span(B)."""
    qa = np.linalg.qr(A)[0]
    qb = np.linalg.qr(B)[0]
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - s.min() ** 2)))


@pytest.fixture(scope="module")
def lda1():
    c = synth.lda_corpus(0, 2000, 500, 10, 0.1, 0.1, 100)
    S = synth.gaussian(1, 500, 30)
    return c, S


def test_whiten_topic_matches_oracle(otm, lda1):
    c, S = lda1
    X = c["X"]
    wh = otm.whiten_topic(otm.DeviceCSR.from_host(X), _dev(S), 10, 2, 1.0)
    torch.cuda.synchronize()
    ref = ow.range_finder_whiten(lambda Z: om.topic_second_moment_apply(X, Z, 1.0),
                                 S.astype(np.float64), 10, 2)
    M2 = om.topic_second_moment(X, 1.0)
    W = to_np(wh["W"]).astype(np.float64)
    # float32 range finder: eigenvalues and W agree to ~1e-5 relative
    np.testing.assert_allclose(to_np(wh["eig"]), ref["eig"], rtol=1e-4)
    assert rel(align_signs(W, ref["W"]), ref["W"]) < 1e-3
    assert np.abs(W.T @ M2 @ W - np.eye(10)).max() < 1e-3
    assert _subspace_gap(to_np(wh["Q"]).astype(np.float64), ref["Q"]) < 1e-3
    np.testing.assert_allclose(to_np(wh["M1"]), om.topic_first_moment(X), rtol=1e-12)
    # the per-document weights of the whitening's moments equal the standalone call's
    mom = otm.topic_moments(otm.DeviceCSR.from_host(X))
    np.testing.assert_array_equal(to_np(wh["row_invlen"]), to_np(mom["row_invlen"]))
    np.testing.assert_array_equal(to_np(wh["row_w"]), to_np(mom["row_w"]))
    # factored forms: W = Q Cw and (W^T)^+ = Q Cp
    Q = to_np(wh["Q"]).astype(np.float64)
    assert rel(Q @ to_np(wh["Cw"]), W) < 1e-6
    assert rel(Q @ to_np(wh["Cp"]), ref["Wplus"] * np.sign(np.sum(Q @ to_np(wh["Cp"]) * ref["Wplus"], 0))) < 1e-3


def test_whiten_topic_rejects_too_large_k(otm):
    # a corpus whose M2 has rank < k: the k-th eigenvalue is not positive
    dense = np.zeros((40, 20))
    dense[:, :3] = 5.0
    X = synth.csr_from_dense(dense)
    S = synth.gaussian(2, 20, 12)
    with pytest.raises(otm.OtmError, match="OTM_ENOTPSD"):
        otm.whiten_topic(otm.DeviceCSR.from_host(X), _dev(S), 8, 2, 1.0)


@pytest.mark.parametrize("kt,kind", [(20, "selection"), (30, "selection"), (20, "gaussian")])
def test_whiten_topic_nystrom_matches_oracle(otm, lda1, kt, kind):
    """Algorithm 2 on the GPU against the oracle's, same float32 S.  The float32
    O = M2 S (SpMM sums, float32 storage) carries ~1e-6 relative error, which
    the rank-k pseudo-inverse of O^T O (condition ~500 here) amplifies to ~1e-5
    on W (3e-6 from float32 rounding alone, emulated on the CPU); the bounds
    below leave two orders of margin."""
    c, _ = lda1
    X = c["X"]
    k = 10
    S = (synth.signed_column_selection(5, 500, kt) if kind == "selection"
         else synth.gaussian(6, 500, kt))
    wh = otm.whiten_topic_nystrom(otm.DeviceCSR.from_host(X), _dev(S), k, 1.0)
    torch.cuda.synchronize()
    ref = ow.nystrom_whiten(lambda Z: om.topic_second_moment_apply(X, Z, 1.0),
                            S.astype(np.float64), k)
    W = to_np(wh["W"]).astype(np.float64)
    np.testing.assert_allclose(to_np(wh["eig"]), ref["eig"], rtol=1e-4)
    assert rel(align_signs(W, ref["W"]), ref["W"]) < 1e-3
    O = to_np(wh["Q"]).astype(np.float64)
    O_ref = om.topic_second_moment_apply(X, S.astype(np.float64), 1.0)
    assert rel(O, O_ref) < 1e-5
    assert rel(O @ to_np(wh["Cw"]), W) < 1e-6
    Wp = O @ to_np(wh["Cp"])
    assert rel(align_signs(Wp, ref["Wplus"]), ref["Wplus"]) < 1e-3
    # (W^T)^+ is a left inverse of W^T: W^T (W^T)^+ = I
    assert np.abs(W.T @ Wp - np.eye(k)).max() < 1e-4


def test_whiten_topic_nystrom_rejects_too_large_k(otm):
    dense = np.zeros((40, 20))
    dense[:, :3] = 5.0
    X = synth.csr_from_dense(dense)
    S = synth.signed_column_selection(2, 20, 12)
    with pytest.raises(otm.OtmError, match="OTM_ENOTPSD"):
        otm.whiten_topic_nystrom(otm.DeviceCSR.from_host(X), _dev(S), 8, 1.0)


def test_topic_pipeline_end_to_end(otm, lda1):
    """Config: d = 500, k = 10, 2,000 x 100-word documents, b = 256, beta = 1e-2/sqrt(t),
    theta = 1, 20 epochs, alpha0 = 1.  Each side runs the whole path itself."""
    c, S = lda1
    X = c["X"]
    k, b, epochs = 10, 256, 20
    perm = synth.epoch_permutations(2, 2000, epochs)
    V0 = synth.haar_orthonormal(3, k)
    Xd = otm.DeviceCSR.from_host(X)
    wh = otm.whiten_topic(Xd, _dev(S), k, 2, 1.0)
    Y = otm.project(Xd, wh["W"], wh["row_invlen"])
    yb = otm.column_mean(Y)
    Vd = _dev(V0.T.copy())
    otm.sgd_run(Vd, Y, Y, Y, torch.stack([yb] * 3), _dev(perm), epochs, b, 1e-2, 1.0, 1.0)
    out = otm.unwhiten(Vd, wh["Q"], wh["Cp"], 1.0, True)
    torch.cuda.synchronize()

    ref = ow.range_finder_whiten(lambda Z: om.topic_second_moment_apply(X, Z, 1.0),
                                 S.astype(np.float64), k, 2)
    Xs = om.as_sparse(X)
    l = om.doc_lengths(Xs)
    Yo = (Xs @ ref["W"]) / l[:, None]
    ybo = Yo.mean(axis=0)
    # projection and means of the GPU path agree with the oracle's up to the
    # whitening's float32 accuracy
    assert rel(to_np(yb), ybo) < 1e-3
    Vo, _ = ostgd.sgd_run(V0, Yo, Yo, Yo, (ybo, ybo, ybo), perm, b, 1e-2, 1.0, 1.0)
    assert rel(to_np(Vd).T, Vo) < 2e-3
    uo = opost.unwhiten(Vo, ref["Wplus"], 1.0, True)
    assert rel(to_np(out["comps"]), uo["mu"]) < 5e-3
    np.testing.assert_allclose(to_np(out["lambda"]), uo["lambda"], rtol=5e-3)


@pytest.fixture(scope="module")
def mmsb_full():
    g = synth.mmsb_graph(0, 5000, 100, 0.01, 0.1, 0.005)
    S_pairs = synth.gaussian(1, 5000, 120)
    S_w = synth.gaussian(2, 5000, 120)
    return g, S_pairs, S_w


def test_whiten_community_full_size(otm, mmsb_full):
    """MMSB, four parts of 5,000 nodes, k = 100, oversampling 20, 2 power
    iterations: the GPU whitening against the oracle's on the same projections."""
    g, S_pairs, S_w = mmsb_full
    k = 100
    D = {x: otm.DeviceCSR.from_host(g[x]) for x in ("G_XA", "G_XB", "G_XC")}
    wh = otm.whiten_community(D["G_XA"], D["G_XB"], D["G_XC"], _dev(S_pairs), _dev(S_w), k, 2, 1.0)
    torch.cuda.synchronize()
    ref = ow.community_whiten_randomized(g["G_XA"], g["G_XB"], g["G_XC"], k, 1.0,
                                         S_pairs.astype(np.float64), S_w.astype(np.float64), 2)
    np.testing.assert_allclose(to_np(wh["sigma"]), ref["sigma"], rtol=1e-3)
    np.testing.assert_allclose(to_np(wh["eig"]), ref["eig"], rtol=1e-3)
    W = to_np(wh["W"]).astype(np.float64)
    # whitening identity with the oracle's (factored) M2
    WtMW = W.T @ ref["apply_M2"](W)
    assert np.abs(WtMW - np.eye(k)).max() < 1e-2
    # the three whitened views, projected by each side
    YA = to_np(otm.project(D["G_XA"], wh["W"]))
    YB = to_np(otm.project(D["G_XB"], wh["W_B"]))
    YAo = om.as_sparse(g["G_XA"]) @ ref["W"]
    YBo = om.as_sparse(g["G_XB"]) @ ref["W_B"]
    # whitened data agree up to per-coordinate signs
    s = np.sign(np.sum(YA * YAo, axis=0))
    assert rel(YA * s, YAo) < 2e-2
    assert rel(YB * s, YBo) < 2e-2


def test_community_sgd_step_full_size(otm, mmsb_full):
    """One fused step at the full MMSB minibatch (b = 1,024, k = 100, three
    distinct views) against the oracle's Lemma 3 on the same inputs."""
    g, _, _ = mmsb_full
    k, b = 100, 1024
    rng = np.random.default_rng(3)
    Ys = [(rng.standard_normal((b, k)) * 0.5 + 0.1).astype(np.float32) for _ in range(3)]
    yb = np.stack([Y.astype(np.float64).mean(axis=0) for Y in Ys])
    V0 = synth.haar_orthonormal(4, k) * np.float32(1.3)
    Vd = _dev(V0.T.copy())
    otm.sgd_step(Vd, *[_dev(Y) for Y in Ys], _dev(yb), 1.0, 1.0, 1.0)
    torch.cuda.synchronize()
    G = ostgd.grad_implicit(V0.astype(np.float64), *[Y.astype(np.float64) for Y in Ys],
                            tuple(yb), 1.0, 1.0)
    gram = V0.astype(np.float64) @ (V0.astype(np.float64).T @ V0.astype(np.float64)) ** 2
    Gk = V0.astype(np.float64) - to_np(Vd).T
    assert np.linalg.norm(Gk - G) / (np.linalg.norm(gram) + np.linalg.norm(gram - G)) < 1e-5
