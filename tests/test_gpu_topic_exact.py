"""GPU parity of the STGD on the whole third moment of Section 2.1, Eq. (3)
(otm_sgd_run_topic_exact: the self-token terms kept) against the FP64 oracle
(oracle.stgd.grad_implicit_topic_exact and its run loop), on the same seeded
corpora, whitening matrices and starts.

Tolerance: the FP32 one of the other STGD kernels, 1e-5 normwise relative to
the two gradient terms (||G - G64|| / (||kappa G_gram|| + ||G_data||)), for the
whole matrix and for every component; runs against the oracle's run at 1e-5.
The products are FP32 tiles accumulated in FP64 and the per-document sums s, q
are FP64, so the cancellation in s^2 - q (pairs of distinct tokens) costs no
accuracy.
"""
import numpy as np
import pytest

import synth
from oracle import moments as om
from oracle import stgd as ostgd
from tests._util import grad_errs, rel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def otm():
    from paper_1309_0787_gb300 import otm as _otm
    return _otm


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _corpus(seed, n, d, k, L, short=True):
    """LDA counts with, if `short`, an empty document and documents of one, two
    and three words among the first rows."""
    X = synth.lda_corpus(seed, n, d, k, 0.2, 0.2, L, poisson_len=True)["X"]
    if not short:
        return X
    dense = synth.csr_to_dense(X)
    dense[0] = 0.0
    for r, words in ((1, [3]), (2, [5, 5]), (3, [1, 7]), (4, [2, 2, 9])):
        dense[r] = 0.0
        for w in words:
            dense[r, w] += 1.0
    return synth.csr_from_dense(dense)


@pytest.mark.parametrize("n,d,k,L,a0,theta", [(90, 60, 6, 12, 1.0, 1.0), (70, 40, 9, 5, 0.5, 2.0),
                                              (400, 300, 17, 40, 0.0, 1.0)])
def test_exact_gradient_one_step(otm, n, d, k, L, a0, theta):
    """One step over all documents (b = n, beta = 1): V0 - V1 is the gradient."""
    X = _corpus(n + d, n, d, k, L)
    g = np.random.default_rng(n + k)
    W = (g.standard_normal((d, k)) * 0.3).astype(np.float32)
    M1 = om.topic_first_moment(X)
    V0 = (0.7 * g.standard_normal((k, k))).astype(np.float32)     # columns = components
    Vd = _dev(V0.T.copy())
    otm.sgd_run_topic_exact(Vd, otm.DeviceCSR.from_host(X), _dev(W), _dev(M1), None, 1, n, 1.0,
                            theta, a0)
    torch.cuda.synchronize()
    V64 = V0.astype(np.float64)
    Gk = V64 - to_np(Vd).T.astype(np.float64)
    G = ostgd.grad_implicit_topic_exact(V64, X, W.astype(np.float64), M1, theta, a0)
    frob, col = grad_errs(Gk, G, ostgd.kappa(theta) * V64 @ (V64.T @ V64) ** 2)
    assert frob < 1e-5 and col < 1e-5, (frob, col)


def test_exact_run_matches_oracle_run(otm):
    """Two epochs with permutations, minibatches of 48 documents (the last one
    partial), snapshots; documents of zero to three words included."""
    n, d, k, b, epochs = 150, 80, 5, 48, 2
    X = _corpus(5, n, d, k, 20)
    g = np.random.default_rng(6)
    W = (g.standard_normal((d, k)) * 0.4).astype(np.float32)
    M1 = om.topic_first_moment(X)
    V0 = synth.haar_orthonormal(7, k)
    perm = synth.epoch_permutations(8, n, epochs)
    Vd = _dev(V0.T.copy())
    snaps = otm.sgd_run_topic_exact(Vd, otm.DeviceCSR.from_host(X), _dev(W), _dev(M1), _dev(perm),
                                    epochs, b, 0.05, 1.0, 1.0, snapshot_every=4)
    torch.cuda.synchronize()
    Vo, so = ostgd.sgd_run_topic_exact(V0, X, W.astype(np.float64), M1, perm, b, 0.05, 1.0, 1.0,
                                       snapshot_every=4)
    assert rel(to_np(Vd).T, Vo) < 1e-5
    assert snaps.shape[0] == len(so) == 2
    for s_gpu, s_ref in zip(to_np(snaps), so):
        assert rel(s_gpu.T, s_ref) < 1e-5


def test_exact_gradient_k100_lda_documents(otm):
    """k = 100 on LDA documents (256 documents of Poisson(100) words over 2,000
    words, Zipf-skewed topics) with a fixed random W of whitened scale: one step
    over all of them from a Haar-random start."""
    n, d, k = 256, 2000, 100
    X = synth.lda_corpus(11, n, d, k, 0.01, 0.05, 100, poisson_len=True, zipf=True)["X"]
    W = (synth.gaussian(12, d, k) * 0.5).astype(np.float32)
    M1 = om.topic_first_moment(X)
    V0 = synth.haar_orthonormal(13, k)
    Vd = _dev(V0.T.copy())
    otm.sgd_run_topic_exact(Vd, otm.DeviceCSR.from_host(X), _dev(W), _dev(M1), None, 1, n, 1.0,
                            1.0, 1.0)
    torch.cuda.synchronize()
    V64 = V0.astype(np.float64)
    Gk = V64 - to_np(Vd).T.astype(np.float64)
    G = ostgd.grad_implicit_topic_exact(V64, X, W.astype(np.float64), M1, 1.0, 1.0)
    frob, col = grad_errs(Gk, G, V64 @ (V64.T @ V64) ** 2)
    assert frob < 1e-5 and col < 1e-5, (frob, col)


def test_exact_rejects_too_small_capacity(otm):
    """A minibatch with more word occurrences than the workspace holds is not
    processed and the call returns OTM_EINVAL (the kernels write nothing past
    the capacity)."""
    n, d, k = 50, 30, 4
    X = _corpus(21, n, d, k, 10, short=False)
    Xd = otm.DeviceCSR.from_host(X)
    W = _dev(np.ones((d, k), np.float32) * 0.1)
    M1 = _dev(om.topic_first_moment(X))
    V = _dev(np.eye(k, dtype=np.float32))
    cap = int(X.nnz) // 2
    for prec in (0, otm.PREC_BF16):
        ws = torch.empty(int(otm._lib.otm_sgd_topic_exact_workspace(k, n, cap, prec)),
                         dtype=torch.uint8, device="cuda")
        st = otm._lib.otm_sgd_run_topic_exact(otm._ptr(V), Xd.ref(), otm._ptr(W), otm._ptr(M1),
                                              k, None, 1, n, cap, 1e-3, 1.0, 1.0, prec, None, 0,
                                              otm._ptr(ws), ws.numel(), otm._stream())
        assert st == 1 and b"nnz_b_max" in otm._lib.otm_last_error()


@pytest.mark.parametrize("n,d,k,L,a0,theta", [(90, 60, 6, 12, 1.0, 1.0), (400, 300, 17, 40, 0.0, 1.0),
                                              (3000, 2000, 100, 100, 1.0, 1.0)])
def test_exact_gradient_one_step_bf16(otm, n, d, k, L, a0, theta):
    """The BF16 tensor-core form (U = W_g V^T and W_g^T Coef on tcgen05): one
    full-batch step within the 2e-2 of the low-precision paths, whole matrix and
    every component; 3,000 documents of 100 words hold about 3e5 occurrences,
    more than 190 slices of the W_g^T Coef product."""
    X = _corpus(n + d, n, d, k, L, short=(n < 1000))
    g = np.random.default_rng(n + k)
    W = (g.standard_normal((d, k)) * (0.3 if k < 50 else 0.05)).astype(np.float32)
    M1 = om.topic_first_moment(X)
    V0 = (0.7 * g.standard_normal((k, k))).astype(np.float32)
    Vd = _dev(V0.T.copy())
    otm.sgd_run_topic_exact(Vd, otm.DeviceCSR.from_host(X), _dev(W), _dev(M1), None, 1, n, 1.0,
                            theta, a0, precision=otm.PREC_BF16)
    torch.cuda.synchronize()
    V64 = V0.astype(np.float64)
    Gk = V64 - to_np(Vd).T.astype(np.float64)
    G = ostgd.grad_implicit_topic_exact(V64, X, W.astype(np.float64), M1, theta, a0)
    frob, col = grad_errs(Gk, G, ostgd.kappa(theta) * V64 @ (V64.T @ V64) ** 2)
    assert frob < 2e-2 and col < 2e-2, (frob, col)


def test_exact_run_bf16_tracks_fp32(otm):
    """Two epochs with permutations and snapshots in BF16 against the FP32 form
    and the oracle's run: both within 2e-2 of the oracle."""
    n, d, k, b, epochs = 150, 80, 5, 48, 2
    X = _corpus(5, n, d, k, 20)
    g = np.random.default_rng(6)
    W = (g.standard_normal((d, k)) * 0.4).astype(np.float32)
    M1 = om.topic_first_moment(X)
    V0 = synth.haar_orthonormal(7, k)
    perm = synth.epoch_permutations(8, n, epochs)
    Vd = _dev(V0.T.copy())
    snaps = otm.sgd_run_topic_exact(Vd, otm.DeviceCSR.from_host(X), _dev(W), _dev(M1),
                                    _dev(perm), epochs, b, 0.05, 1.0, 1.0, snapshot_every=4,
                                    precision=otm.PREC_BF16)
    torch.cuda.synchronize()
    Vo, so = ostgd.sgd_run_topic_exact(V0, X, W.astype(np.float64), M1, perm, b, 0.05, 1.0, 1.0,
                                       snapshot_every=4)
    assert rel(to_np(Vd).T, Vo) < 2e-2
    for s_gpu, s_ref in zip(to_np(snaps), so):
        assert rel(s_gpu.T, s_ref) < 2e-2
