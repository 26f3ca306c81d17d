"""GPU parity of the tensor-core (BF16 / FP8) STGD against the FP64 oracle.

The low-precision path quantises the samples, V and B (per-sample and
per-component scales) and accumulates in FP32; FP8 keeps V as two e4m3 terms,
and the two-term FP8 form the samples and B as well.  The oracle computes
Lemma 3 in FP64 from the unquantised samples.  Tolerance for every precision:
2e-2 normwise relative,
||G - G64||_F / (||kappa G_gram||_F + ||G_data||_F), and the same ratio for
every column (component) of G on its own, so that one wrong component or tile
cannot hide inside the Frobenius norm.
"""
import numpy as np
import pytest

import synth
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


def _grad_err(otm, prec, k, b, sym, a0, seed):
    g = np.random.default_rng(seed)
    Ys = [(g.standard_normal((b, k)) * 0.5 + 0.2 * s).astype(np.float32) for s in (1, -1, 0.5)]
    if sym:
        Ys = [Ys[0]] * 3
    yb = np.stack([Y.astype(np.float64).mean(axis=0) for Y in Ys])
    V0 = (synth.haar_orthonormal(seed + 1, k) * np.float32(1.2)).astype(np.float32)
    qs = [otm.quantize_samples(_dev(Y), prec) for Y in (Ys[:1] if sym else Ys)]
    if sym:
        qs = qs * 3
    Vd = _dev(V0.T.copy())
    otm.sgd_run_lp(Vd, qs[0], qs[1], qs[2], _dev(yb), None, 1, b, 1.0, 1.0, a0, prec)
    torch.cuda.synchronize()
    V64 = V0.astype(np.float64)
    G = ostgd.grad_implicit(V64, *[Y.astype(np.float64) for Y in Ys], tuple(yb), 1.0, a0)
    return _errs(V64, V64 - to_np(Vd).T.astype(np.float64), G)


def _errs(V64, Gk, G):
    """(Frobenius, worst column) error of Gk against the oracle's G; theta = 1."""
    return grad_errs(Gk, G, ostgd.kappa(1.0) * V64 @ (V64.T @ V64) ** 2)


@pytest.mark.parametrize("k,b,sym,a0", [(100, 1024, False, 1.0), (100, 1024, True, 1.0),
                                        (10, 256, True, 1.0), (17, 100, False, 0.5),
                                        (64, 2000, True, 0.0), (128, 512, True, 1.0)])
def test_tc_bf16_gradient(otm, k, b, sym, a0):
    frob, col = _grad_err(otm, otm.PREC_BF16, k, b, sym, a0, 3 * k + b)
    assert frob < 2e-2 and col < 2e-2, (frob, col)


@pytest.mark.parametrize("k,b,sym,a0", [(100, 1024, False, 1.0), (100, 1024, True, 1.0),
                                        (33, 300, False, 1.0), (128, 1024, True, 1.0)])
def test_tc_fp8_gradient(otm, k, b, sym, a0):
    frob, col = _grad_err(otm, otm.PREC_FP8, k, b, sym, a0, 5 * k + b)
    assert frob < 2e-2 and col < 2e-2, (frob, col)


@pytest.mark.parametrize("k,b,sym,a0", [(100, 1024, False, 1.0), (100, 1024, True, 1.0),
                                        (33, 300, False, 1.0), (128, 1024, True, 1.0),
                                        (200, 512, True, 1.0), (256, 512, True, 0.5)])
def test_tc_fp8x2_gradient(otm, k, b, sym, a0):
    """FP8 with two-term samples and B: within 2e-2, and closer to the oracle than
    the one-term FP8 on the same inputs."""
    frob, col = _grad_err(otm, otm.PREC_FP8X2, k, b, sym, a0, 7 * k + b)
    assert frob < 2e-2 and col < 2e-2, (frob, col)
    frob1, _ = _grad_err(otm, otm.PREC_FP8, k, b, sym, a0, 7 * k + b)
    assert frob < frob1, (frob, frob1)


def test_quantize_samples_two_terms(otm):
    """PREC_FP8X2 stores the e4m3 residual in a second plane at the same scale:
    hi + lo reproduces the row within the two-term rounding (about 2^-8 of the
    row's largest entry), and the first plane equals the one-term FP8 rows."""
    g = np.random.default_rng(41)
    Y = (g.standard_normal((300, 70)) * np.exp(g.standard_normal((300, 1)))).astype(np.float32)
    q2, s2 = otm.quantize_samples(_dev(Y), otm.PREC_FP8X2)
    q1, s1 = otm.quantize_samples(_dev(Y), otm.PREC_FP8)
    torch.cuda.synchronize()
    assert tuple(q2.shape) == (600, 80)
    np.testing.assert_array_equal(to_np(q2[:300]), to_np(q1))
    np.testing.assert_array_equal(to_np(s2), to_np(s1))
    f8 = lambda q: q.view(torch.float8_e4m3fn).float().cpu().numpy().astype(np.float64)  # noqa: E731
    rec = (f8(q2[:300]) + f8(q2[300:]))[:, :70] * to_np(s2)[:, None]
    amax = np.abs(Y).max(axis=1, keepdims=True)
    assert np.all(np.abs(rec - Y) <= amax * 2.0 ** -8 + 1e-30)
    assert np.abs(rec - Y).max() < np.abs(f8(q1)[:, :70] * to_np(s1)[:, None] - Y).max()


@pytest.fixture(scope="module")
def lda_samples():
    """Whitened samples of a synthetic LDA corpus (6,000 documents of Poisson(300)
    words over 2,000 words, Zipf-skewed Dir(0.05) topics, k = 50, alpha0 = 0.5),
    whitened and projected by the oracle (FP64), stored as float32."""
    from oracle import moments as om
    from oracle import whiten as ow
    n, d, k = 6000, 2000, 50
    c = synth.lda_corpus(0, n, d, k, 0.01, 0.05, 300, poisson_len=True, zipf=True)
    a0 = 0.01 * k
    S = synth.gaussian(1, d, k + 20).astype(np.float64)
    wh = ow.range_finder_whiten(lambda Z: om.topic_second_moment_apply(c["X"], Z, a0), S, k, 2)
    Xs = om.as_sparse(c["X"])
    Y = ((Xs @ wh["W"]) / om.doc_lengths(Xs)[:, None]).astype(np.float32)
    return Y, a0


@pytest.mark.parametrize("prec_name", ["PREC_BF16", "PREC_FP8", "PREC_FP8X2"])
def test_tc_gradient_on_lda_samples(otm, lda_samples, prec_name):
    """One step on a minibatch of whitened LDA samples (Section 3.1): the whitened
    documents share a large mean and carry word-sampling noise, so the
    alpha0-corrected terms of Lemma 3 cancel much more than on Gaussian samples.
    Full-data means, Haar-random V."""
    Y, a0 = lda_samples
    k, b = Y.shape[1], 1024
    prec = getattr(otm, prec_name)
    yb = np.stack([Y.astype(np.float64).mean(axis=0)] * 3)
    Yb = np.ascontiguousarray(Y[:b])
    V0 = synth.haar_orthonormal(4, k).astype(np.float32)
    q = otm.quantize_samples(_dev(Yb), prec)
    Vd = _dev(V0.T.copy())
    otm.sgd_run_lp(Vd, q, q, q, _dev(yb), None, 1, b, 1.0, 1.0, a0, prec)
    torch.cuda.synchronize()
    V64 = V0.astype(np.float64)
    Y64 = Yb.astype(np.float64)
    G = ostgd.grad_implicit(V64, Y64, Y64, Y64, tuple(yb), 1.0, a0)
    frob, col = _errs(V64, V64 - to_np(Vd).T.astype(np.float64), G)
    assert frob < 2e-2 and col < 2e-2, (frob, col)


def test_tc_bf16_run_tracks_fp32_run(otm):
    """Several epochs with permutations: the BF16 iterate stays close to the
    FP32 oracle iterate (errors do not accumulate beyond the per-step level)."""
    k, n, b, epochs = 16, 2000, 256, 4
    o = synth.orthogonal_samples(7, k, n, 0.05)
    Y = o["Y"]
    yb = Y.astype(np.float64).mean(axis=0)
    perm = synth.epoch_permutations(8, n, epochs)
    V0 = synth.haar_orthonormal(9, k)
    q = otm.quantize_samples(_dev(Y), otm.PREC_BF16)
    Vd = _dev(V0.T.copy())
    snaps = otm.sgd_run_lp(Vd, q, q, q, _dev(np.stack([yb] * 3)), _dev(perm), epochs, b, 5e-3,
                           1.0, 0.0, otm.PREC_BF16, snapshot_every=8)
    torch.cuda.synchronize()
    Vo, so = ostgd.sgd_run(V0, Y, Y, Y, (yb, yb, yb), perm, b, 5e-3, 1.0, 0.0, snapshot_every=8)
    assert rel(to_np(Vd).T, Vo) < 2e-2
    assert snaps.shape[0] == len(so)


def test_quantize_samples_roundtrip(otm):
    g = np.random.default_rng(1)
    Y = (g.standard_normal((300, 37)) * np.exp(g.standard_normal((300, 1)))).astype(np.float32)
    qb, sb = otm.quantize_samples(_dev(Y), otm.PREC_BF16)
    qf, sf = otm.quantize_samples(_dev(Y), otm.PREC_FP8)
    torch.cuda.synchronize()
    yb = to_np(qb.view(torch.bfloat16).float())[:, :37]
    assert np.abs(yb - Y).max() <= 2 ** -8 * np.abs(Y).max()
    yf = to_np(qf.view(torch.float8_e4m3fn).float())[:, :37] * to_np(sf)[:, None]
    # e4m3: 3 mantissa bits -> relative rounding error <= 2^-4 of each value's scale
    assert np.all(np.abs(yf - Y) <= 2 ** -4 * np.abs(Y) + 2 ** -9 * to_np(sf)[:, None] * 448)
    assert np.all(to_np(qb)[:, 74:] == 0) and np.all(to_np(qf)[:, 37:] == 0)


@pytest.mark.parametrize("k,b,prec_name", [(200, 512, "PREC_BF16"), (256, 1024, "PREC_BF16"),
                                           (256, 512, "PREC_FP8"), (200, 1024, "PREC_FP8")])
def test_tc_gradient_beyond_128_components(otm, k, b, prec_name):
    """k > 128: 256 padded coordinates, products per 128-row block (symmetric views)."""
    frob, col = _grad_err(otm, getattr(otm, prec_name), k, b, True, 1.0, 7 * k + b)
    assert frob < 2e-2 and col < 2e-2, (frob, col)


@pytest.mark.parametrize("prec_name", ["PREC_BF16", "PREC_FP8"])
def test_tc_three_views_beyond_128(otm, prec_name):
    """k > 128 with three distinct views (16-CTA cluster, one sample stage of
    three views): one step against the oracle's implicit gradient."""
    frob, col = _grad_err(otm, getattr(otm, prec_name), 160, 512, False, 1.0, 41)
    assert frob < 2e-2 and col < 2e-2, (frob, col)


@pytest.mark.parametrize("prec_name,tol,sym", [("PREC_BF16", 2e-2, True), ("PREC_FP8", 2e-2, True),
                                               ("PREC_BF16", 2e-2, False),
                                               ("PREC_FP8", 2e-2, False)])
def test_tc_run_beyond_128_tracks_oracle(otm, prec_name, tol, sym):
    """k > 128 over twelve steps with a partial last minibatch: the cluster's
    shared V image alternates between two global buffers, read back for the
    Gram term of every step.  beta0 = 0.2 moves V by about 60 %; a Gram term
    one step stale would leave the iterate about 9 % from the oracle's, 1 %
    random gradient noise about 0.3 %."""
    prec = getattr(otm, prec_name)
    k, n, b, epochs = 160, 1500, 256, 2
    g = np.random.default_rng(13)
    Y = (g.standard_normal((n, k)) * 0.3 + 0.1).astype(np.float32)
    Ys = [Y] * 3 if sym else [Y, (Y + 0.05 * g.standard_normal(Y.shape)).astype(np.float32),
                              Y[::-1].copy()]
    yb = np.stack([Z.astype(np.float64).mean(axis=0) for Z in Ys])
    perm = synth.epoch_permutations(15, n, epochs)
    V0 = synth.haar_orthonormal(16, k)
    qs = [otm.quantize_samples(_dev(Z), prec) for Z in (Ys[:1] if sym else Ys)]
    if sym:
        qs = qs * 3
    Vd = _dev(V0.T.copy().astype(np.float32))
    otm.sgd_run_lp(Vd, qs[0], qs[1], qs[2], _dev(yb), _dev(perm), epochs, b, 0.2, 1.0, 1.0, prec)
    torch.cuda.synchronize()
    Vo, _ = ostgd.sgd_run(V0, *Ys, tuple(yb), perm, b, 0.2, 1.0, 1.0)
    assert rel(to_np(Vd).T, Vo) < tol
