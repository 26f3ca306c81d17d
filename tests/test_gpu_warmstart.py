"""GPU parity of the learned warm start against the FP64 oracle.

Tolerances: FP32 kernels (Gram-Schmidt, its backward, the loss, Adam, the
initial scaling) 1e-4 relative or tighter; BF16 tensor-core paths (GEMM
inputs rounded to BF16, sketches, MLP activations) 2e-2 normwise relative, the
tolerance the precision form uses; the GEMM itself is checked against the
exact product of its BF16-rounded operands at FP32-accumulation accuracy.
"""
import numpy as np
import pytest

import synth
from oracle import stgd as ostgd
from oracle import warmstart as ows
from tests._util import to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def otm():
    from paper_1309_0787_gb300 import otm as _otm
    return _otm


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).cuda()


def _bf(a):
    """float64 values of the BF16 rounding of a."""
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def _flat(p):
    return np.concatenate([p[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def _unflat(v, din, h, dout):
    out, o = {}, 0
    for key, shape in (("W1", (h, din)), ("b1", (h,)), ("W2", (h, h)), ("b2", (h,)),
                       ("W3", (dout, h)), ("b3", (dout,))):
        n = int(np.prod(shape))
        out[key] = v[o:o + n].reshape(shape)
        o += n
    return out


def _relnorm(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("nb,M,N,K", [(1, 256, 512, 1024), (1, 200, 136, 72), (3, 64, 320, 2000),
                                      (2, 130, 8, 8)])
def test_gemm_bf16_matches_exact_product(otm, nb, M, N, K):
    g = np.random.default_rng(M + N + K)
    A = g.standard_normal((nb, M, K)).astype(np.float32)
    B = g.standard_normal((nb, N, K)).astype(np.float32)
    C, _ = otm.gemm_bf16(_dev(A, torch.bfloat16), _dev(B, torch.bfloat16), alpha=0.5)
    ref = 0.5 * np.einsum("zmk,znk->zmn", _bf(A), _bf(B))
    bound = 0.5 * np.einsum("zmk,znk->zmn", np.abs(_bf(A)), np.abs(_bf(B)))
    assert np.all(np.abs(to_np(C) - ref) <= 1e-5 * bound + 1e-6)


def test_gemm_bf16_bias_gelu_epilogue(otm):
    g = np.random.default_rng(3)
    A = g.standard_normal((256, 96)).astype(np.float32) / 8
    B = g.standard_normal((264, 96)).astype(np.float32) / 8
    bias = g.standard_normal(264).astype(np.float32)
    C, H = otm.gemm_bf16(_dev(A, torch.bfloat16), _dev(B, torch.bfloat16), epilogue=2,
                         bias=_dev(bias), want_h=True)
    z = _bf(A) @ _bf(B).T + bias
    assert np.abs(to_np(C) - z).max() < 1e-5 * np.abs(z).max()
    h = to_np(H.float())
    assert np.abs(h - ows.gelu(z)).max() <= 2 ** -8 * np.abs(ows.gelu(z)).max() + 1e-6


def test_generator_matches_counter_definition(otm):
    """The GPU generator reproduces synth's counter-based samples (same Philox
    counters and gamma algorithm); float32 math functions may differ by an
    ulp, so rows agree to 1e-4 except for (rare) flipped acceptance tests."""
    inst = synth.whitened_lda_instances(5, 3, 16)
    n = 2000
    Yc = synth.whitened_lda_samples(inst, n, 77, first=0)
    Yg = to_np(otm.ws_generate(_dev(inst["m"]), _dev(inst["alpha32"]), n, 77))
    err = np.linalg.norm(Yg - Yc, axis=2) / np.linalg.norm(Yc, axis=2)
    assert np.mean(err < 1e-4) > 0.999, np.sort(err.reshape(-1))[-10:]
    # instance offset: instances 1..2 generated alone equal the batch's 1..2
    Yo = to_np(otm.ws_generate(_dev(inst["m"][1:]), _dev(inst["alpha32"][1:]), n, 77, first=1))
    np.testing.assert_array_equal(Yo, Yg[1:])


def test_sketch_matches_explicit_tensor(otm):
    k, n, J = 8, 3000, 4
    inst = synth.whitened_lda_instances(9, 2, k)
    Y = synth.whitened_lda_samples(inst, n, 10)
    th = synth.unit_vectors(11, J, k)
    S, x16 = otm.ws_sketch(_dev(Y), _dev(inst["alpha0"]), _dev(th))
    S = to_np(S)
    for i in range(2):
        y = Y[i].astype(np.float64)
        ref = ows.sketches(y, y.mean(axis=0), inst["alpha0"][i], th.astype(np.float64))
        assert _relnorm(S[i], ref) < 2e-2
        x = ows.mlp_input(ref)
        assert _relnorm(to_np(x16[i].float()), x) < 2e-2


def test_gram_schmidt_forward_backward_loss(otm):
    k, nb = 24, 5
    g = np.random.default_rng(4)
    M = g.standard_normal((nb, k, k)).astype(np.float32) + 3 * np.eye(k, dtype=np.float32)
    Us = np.stack([synth.haar_orthonormal(20 + b, k) for b in range(nb)])
    lam = g.uniform(0.5, 3.0, (nb, k)).astype(np.float32)
    U, R = otm.gram_schmidt(_dev(M))
    loss, dU = otm.ws_loss_grad(U, _dev(Us), _dev(lam), scale=0.25)
    dUin = g.standard_normal((nb, k, k)).astype(np.float32)
    dM = otm.gram_schmidt_backward(U, R, _dev(dUin))
    U, R, loss, dU, dM = map(to_np, (U, R, loss, dU, dM))
    for b in range(nb):
        Uo, Ro = ows.gram_schmidt(M[b].astype(np.float64))
        assert np.abs(U[b] - Uo).max() < 1e-5 and np.abs(R[b] - Ro).max() < 1e-5 * np.abs(Ro).max()
        Lo = ows.warmstart_loss(Uo, lam[b].astype(np.float64), Us[b].astype(np.float64))
        Go = ows.warmstart_loss_grad(Uo, lam[b].astype(np.float64), Us[b].astype(np.float64))
        assert abs(loss[b] - Lo) < 1e-5 * abs(Lo)
        assert _relnorm(dU[b], 0.25 * Go) < 1e-4
        dMo = ows.gram_schmidt_backward(Uo, Ro, dUin[b].astype(np.float64))
        assert _relnorm(dM[b], dMo) < 1e-4


def test_init_components_match_explicit_tensor(otm):
    k, n = 8, 2000
    inst = synth.whitened_lda_instances(13, 2, k)
    Y = synth.whitened_lda_samples(inst, n, 14)
    U0 = np.stack([synth.haar_orthonormal(30 + b, k) for b in range(2)])
    V0 = to_np(otm.ws_init_components(_dev(U0), _dev(Y), _dev(inst["alpha0"]), 1.0))
    for b in range(2):
        y = Y[b].astype(np.float64)
        yb = y.mean(axis=0)
        T = ostgd.whitened_tensor(y, y, y, (yb, yb, yb), inst["alpha0"][b])
        ref = ows.initial_components(U0[b].astype(np.float64), T, 1.0)   # columns
        assert _relnorm(V0[b].T, ref) < 1e-4


def _net(otm, seed, din, h, dout):
    p = ows.init_params(seed, din, h, dout)
    g = np.random.default_rng(seed + 1)
    for key in ("b1", "b2", "b3"):
        p[key] = 0.1 * g.standard_normal(p[key].shape)
    # the reference uses the BF16-rounded weights the kernels multiply with
    pb = {key: (_bf(v) if key.startswith("W") else v.astype(np.float32).astype(np.float64))
          for key, v in p.items()}
    return otm.Mlp(din, h, dout, _flat(p).astype(np.float32)), pb


def test_mlp_forward_backward_match_oracle(otm):
    din, h, dout, B = 256, 64, 64, 32
    net, pb = _net(otm, 40, din, h, dout)
    g = np.random.default_rng(41)
    x = _bf(g.standard_normal((B, din)))
    x16 = _dev(x.astype(np.float32), torch.bfloat16)
    out = to_np(net.forward(x16))
    ref, cache = ows.mlp_forward(x, pb)
    assert _relnorm(out, ref) < 2e-2
    dout_ = g.standard_normal((B, dout))
    grad = to_np(net.backward(x16, _dev(dout_.astype(np.float32))))
    gref = ows.mlp_backward(dout_, pb, cache)
    gg = _unflat(grad, din, h, dout)
    for key in gref:
        assert _relnorm(gg[key], gref[key]) < 2e-2, key


def test_adam_matches_oracle(otm):
    din, h, dout = 16, 8, 16
    net, _ = _net(otm, 50, din, h, dout)
    P = net.p.numel()
    g = np.random.default_rng(51)
    p0 = to_np(net.p).astype(np.float64)
    m = np.zeros(P)
    v = np.zeros(P)
    p = p0.copy()
    for t in (1, 2, 3):
        gr = g.standard_normal(P)
        net.grad.copy_(_dev(gr.astype(np.float32)))
        net.adam(1e-2)
        p, m, v = ows.adam_step(p, gr.astype(np.float32).astype(np.float64), m, v, t, 1e-2)
    assert np.abs(to_np(net.p) - p).max() < 1e-5
    assert np.all(to_np(net.p16.float()) == to_np(net.p.to(torch.bfloat16).float()))


def test_train_step_gradient_matches_oracle(otm):
    """otm_ws_train_step's gradient (before its Adam update) equals the oracle's
    composite gradient MLP -> Gram-Schmidt -> loss on the same BF16 weights."""
    k, J, h, B = 4, 4, 32, 16
    din, dout = J * k * k, k * k
    net, pb = _net(otm, 60, din, h, dout)
    g = np.random.default_rng(61)
    x = _bf(g.standard_normal((B, din)))
    Us = np.stack([synth.haar_orthonormal(70 + b, k) for b in range(B)])
    lam = g.uniform(0.5, 2.0, (B, k)).astype(np.float32)
    loss = to_np(net.train_step(_dev(x.astype(np.float32), torch.bfloat16), _dev(Us), _dev(lam),
                                k, 1e-3))
    Lo, gref = ows.batch_loss_and_grad(pb, x, Us.astype(np.float64), lam.astype(np.float64), k)
    assert abs(loss.mean() - Lo) < 2e-2 * abs(Lo)
    gg = _unflat(to_np(net.grad), din, h, dout)
    for key in gref:
        assert _relnorm(gg[key], gref[key]) < 3e-2, key


def test_canonical_frame_matches_oracle(otm):
    """E, the eigenvalues and the rotated input against eigh on first sketches
    with a known, separated spectrum (the other sketches arbitrary)."""
    k, J, nb = 16, 4, 3
    g = np.random.default_rng(90)
    S = g.standard_normal((nb, J, k, k))
    S = 0.5 * (S + S.transpose(0, 1, 3, 2))
    for b in range(nb):
        Q = synth.haar_orthonormal(91 + b, k).astype(np.float64)
        S[b, 0] = (Q * np.linspace(3.0, -1.0, k)) @ Q.T
    S = S.astype(np.float32)
    E, ev, x16 = otm.ws_canonicalize(_dev(S))
    E, ev, x = to_np(E), to_np(ev), to_np(x16.float())
    for b in range(nb):
        Eo, wo = ows.canonical_frame(S[b, 0].astype(np.float64))
        assert np.abs(ev[b] - wo).max() < 1e-5 * np.abs(wo).max()
        assert np.abs(E[b] - Eo).max() < 1e-4
        xo, _ = ows.canonical_input(S[b].astype(np.float64))
        assert _relnorm(x[b], xo) < 2e-2
    U = np.random.default_rng(93).standard_normal((3, k, k)).astype(np.float32)
    R0 = to_np(otm.ws_rotate(_dev(E), _dev(U)))
    R1 = to_np(otm.ws_rotate(_dev(E), _dev(U), transpose=True))
    for b in range(3):
        assert np.abs(R0[b] - E[b] @ U[b]).max() < 1e-5
        assert np.abs(R1[b] - E[b].T @ U[b]).max() < 1e-5


def test_training_lowers_loss_and_beats_random_init(otm):
    """A short training run on generated instances (k = 8), started at the
    canonical frame, lowers the loss; on held-out instances the network's
    directions (rotated back from the frame) capture far more of T* (mean of
    -L) than Haar-random ones and no less than the frame alone."""
    k, J, h, n, ntr, nte, B = 8, 4, 256, 1000, 2048, 256, 128
    din, dout = J * k * k, k * k
    inst = synth.whitened_lda_instances(80, ntr + nte, k)
    th = _dev(synth.unit_vectors(81, J, k))
    Y = otm.ws_generate(_dev(inst["m"]), _dev(inst["alpha32"]), n, 82)
    S, _ = otm.ws_sketch(Y, _dev(inst["alpha0"]), th)
    E, _, X = otm.ws_canonicalize(S)
    Us = _dev(inst["U"].astype(np.float32))
    Ut = otm.ws_rotate(E, Us, transpose=True)        # targets in the canonical frame
    lam = _dev(inst["lam"].astype(np.float32))
    # start at the canonical frame: b3 = vec(I), W3 small (the network learns
    # corrections to the frame)
    p0 = ows.init_params(83, din, h, dout)
    p0["W3"] *= 0.01
    p0["b3"] = np.eye(k).reshape(-1)
    net = otm.Mlp(din, h, dout, _flat(p0).astype(np.float32))
    first, last = [], []
    for step in range(300):
        i0 = (step * B) % ntr
        loss = net.train_step(X[i0:i0 + B], Ut[i0:i0 + B], lam[i0:i0 + B], k, 1e-3)
        (first if step < 10 else last).append(float(loss.mean()))
    net.check(B)
    assert np.mean(last[-10:]) < np.mean(first)
    U0 = otm.ws_rotate(E[ntr:], net.infer(X[ntr:ntr + nte], k))
    l_net = float(otm.ws_loss_grad(U0, Us[ntr:], lam[ntr:])[0].mean())
    Ur = _dev(np.stack([synth.haar_orthonormal(900 + b, k) for b in range(nte)]))
    l_rand = float(otm.ws_loss_grad(Ur, Us[ntr:], lam[ntr:])[0].mean())
    l_frame = float(otm.ws_loss_grad(E[ntr:].contiguous(), Us[ntr:], lam[ntr:])[0].mean())
    print(f"held-out -L: network {-l_net:.4f}, canonical frame {-l_frame:.4f}, random {-l_rand:.4f}")
    assert l_net < l_rand - 0.5
    assert l_net < l_frame + 0.01


def _steps_to_1e3(otm, Y, a0, V0, U_ref, lam_ref, beta0, max_steps):
    """First full-batch STGD step (b = n) whose iterate is within 1e-3 relative
    reconstruction error of the reference, or None."""
    yb = torch.stack([Y.double().mean(0)] * 3).contiguous()
    V = V0.clone()
    sn = otm.sgd_run(V, Y, Y, Y, yb, None, max_steps, Y.shape[0], beta0, 1.0, a0,
                     snapshot_every=1)
    for j in range(sn.shape[0]):
        if float(otm.recon_error(sn[j].contiguous(), U_ref, lam_ref, 1.0)[0]) <= 1e-3:
            return j + 1
    return None


def test_trained_network_beats_frame_on_held_out(otm):
    """The learned start against the canonical frame alone and a Haar-random start
    (k = 8), after training on 65,536 generated instances (8 epochs, batch 256):
      * captured mass -L on 1,000 held-out instances: the network's mean exceeds
        the frame's by at least 0.005 and by at least four standard errors of the
        paired differences;
      * full-batch STGD (b = n = 4,000, beta0 = 0.1) to 1e-3 of a converged
        reference (6,000 steps from the frame start) on 200 of them: the network's
        start reaches 1e-3 on at least 99 % of the instances, in at most 0.9 times
        the frame start's mean number of steps and by at least two standard errors
        of the paired differences; the random start reaches it within 600 steps on
        fewer than half of them."""
    k, J, h, n_train, ntr, B, epochs = 8, 4, 256, 1000, 65536, 256, 8
    nte, n_test, nsgd, beta0 = 1000, 4000, 200, 0.1
    din, dout = J * k * k, k * k
    inst = synth.whitened_lda_instances(300, ntr + nte, k)
    th = _dev(synth.unit_vectors(301, J, k))
    m, al = _dev(inst["m"]), _dev(inst["alpha32"])
    a0 = _dev(inst["alpha0"])
    Us = _dev(inst["U"].astype(np.float32))
    lam = _dev(inst["lam"].astype(np.float32))
    X = torch.empty(ntr, din, dtype=torch.bfloat16, device="cuda")
    E = torch.empty(ntr, k, k, dtype=torch.float32, device="cuda")
    for c0 in range(0, ntr, 1024):
        c1 = min(c0 + 1024, ntr)
        Yc = otm.ws_generate(m[c0:c1].contiguous(), al[c0:c1].contiguous(), n_train, 302,
                             first=c0)
        S, _ = otm.ws_sketch(Yc, a0[c0:c1].contiguous(), th)
        Ec, _, Xc = otm.ws_canonicalize(S)
        X[c0:c1], E[c0:c1] = Xc, Ec
    Ut = otm.ws_rotate(E, Us[:ntr].contiguous(), transpose=True)
    p0 = ows.init_params(303, din, h, dout)
    p0["W3"] *= 0.01
    p0["b3"] = np.eye(k).reshape(-1)
    net = otm.Mlp(din, h, dout, _flat(p0).astype(np.float32))
    steps = epochs * ntr // B
    for st in range(steps):
        i0 = (st * B) % ntr
        net.train_step(X[i0:i0 + B], Ut[i0:i0 + B], lam[i0:i0 + B], k,
                       1e-3 if st < 0.7 * steps else 2e-4)
    net.check(B)
    lo = ntr
    Yt = otm.ws_generate(m[lo:].contiguous(), al[lo:].contiguous(), n_test, 304, first=lo)
    St, _ = otm.ws_sketch(Yt, a0[lo:].contiguous(), th)
    Et, _, Xt = otm.ws_canonicalize(St)
    U0 = otm.ws_rotate(Et, net.infer(Xt, k).contiguous())
    Ur = _dev(np.stack([synth.haar_orthonormal(5000 + b, k) for b in range(nte)]))

    def captured(U):
        return -to_np(otm.ws_loss_grad(U.contiguous(), Us[lo:].contiguous(),
                                       lam[lo:].contiguous())[0]).astype(np.float64)
    cn, cf, cr = captured(U0), captured(Et), captured(Ur)
    d = cn - cf
    sem = d.std() / np.sqrt(nte)
    print(f"held-out -L: network {cn.mean():.4f}, frame {cf.mean():.4f}, random {cr.mean():.4f}; "
          f"network - frame {d.mean():.4f} +- {sem:.4f}")
    assert d.mean() >= 0.005 and d.mean() >= 4 * sem

    a0t = a0[lo:].contiguous()
    starts = {"net": otm.ws_init_components(U0, Yt, a0t, 1.0),
              "frame": otm.ws_init_components(Et.contiguous(), Yt, a0t, 1.0),
              "random": otm.ws_init_components(Ur, Yt, a0t, 1.0)}
    res = {nm: [] for nm in starts}
    for i in range(nsgd):
        Y = Yt[i].contiguous()
        a0i = float(a0t[i])
        yb = torch.stack([Y.double().mean(0)] * 3).contiguous()
        Vref = starts["frame"][i].clone()
        otm.sgd_run(Vref, Y, Y, Y, yb, None, 6000, n_test, beta0, 1.0, a0i)
        nr = Vref.double().norm(dim=1)
        lam_ref, U_ref = (nr ** 3).contiguous(), (Vref.double() / nr[:, None]).contiguous()
        for nm, V0 in starts.items():
            res[nm].append(_steps_to_1e3(otm, Y, a0i, V0[i], U_ref, lam_ref, beta0,
                                         600 if nm == "random" else 1000))
    reached = {nm: np.mean([s is not None for s in v]) for nm, v in res.items()}
    both = [(a, b) for a, b in zip(res["net"], res["frame"]) if a is not None and b is not None]
    sn = np.array([a for a, _ in both], dtype=float)
    sf = np.array([b for _, b in both], dtype=float)
    dd = sn - sf
    print(f"steps to 1e-3: reached {reached}; mean network {sn.mean():.1f}, frame {sf.mean():.1f}; "
          f"paired {dd.mean():.2f} +- {dd.std() / np.sqrt(len(dd)):.2f}")
    assert reached["net"] >= 0.99
    assert sn.mean() <= 0.9 * sf.mean()
    assert dd.mean() <= -2 * dd.std() / np.sqrt(len(dd))
    assert reached["random"] < 0.5
