"""CPU pins of the warm-start oracle: finite differences of the MLP, of the
Gram-Schmidt backward and of the loss; library QR; closed-form optimum."""
import itertools

import numpy as np

from oracle import stgd, warmstart as ws


def _fd(f, x, h=1e-6):
    g = np.zeros_like(x)
    for idx in itertools.product(*[range(s) for s in x.shape]):
        e = np.zeros_like(x)
        e[idx] = h
        g[idx] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def test_gelu_matches_definition_and_derivative():
    z = np.linspace(-4, 4, 41)
    from scipy.stats import norm
    np.testing.assert_allclose(ws.gelu(z), z * norm.cdf(z), atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(ws.gelu_grad(z), (ws.gelu(z + h) - ws.gelu(z - h)) / (2 * h),
                               atol=1e-8)


def test_mlp_backward_finite_differences():
    p = ws.init_params(0, 6, 5, 4)
    for key in p:
        p[key] = p[key] + 0.1 * np.random.default_rng(1).standard_normal(p[key].shape)
    x = np.random.default_rng(2).standard_normal((3, 6))
    w = np.random.default_rng(3).standard_normal((3, 4))   # L = sum(w * out)
    out, cache = ws.mlp_forward(x, p)
    g = ws.mlp_backward(w, p, cache)
    for key in p:
        def f(v, key=key):
            q = dict(p)
            q[key] = v
            return float((w * ws.mlp_forward(x, q)[0]).sum())
        np.testing.assert_allclose(g[key], _fd(f, p[key]), rtol=1e-6, atol=1e-8)


def test_gram_schmidt_is_library_qr():
    M = np.random.default_rng(4).standard_normal((7, 7))
    U, R = ws.gram_schmidt(M)
    Q, Rl = np.linalg.qr(M)
    s = np.sign(np.diag(Rl))
    np.testing.assert_allclose(U, Q * s, atol=1e-12)
    np.testing.assert_allclose(R, (Rl.T * s).T, atol=1e-12)


def test_gram_schmidt_backward_finite_differences():
    g = np.random.default_rng(5)
    M = g.standard_normal((5, 5)) + 3 * np.eye(5)
    W = g.standard_normal((5, 5))                      # L = sum(W * U(M))
    U, R = ws.gram_schmidt(M)
    dM = ws.gram_schmidt_backward(U, R, W)
    np.testing.assert_allclose(dM, _fd(lambda X: float((W * ws.gram_schmidt(X)[0]).sum()), M),
                               rtol=1e-6, atol=1e-8)


def test_loss_optimum_and_gradient():
    g = np.random.default_rng(6)
    k = 5
    Us, _ = np.linalg.qr(g.standard_normal((k, k)))
    lam = g.uniform(1, 3, k)
    # the true components (any order, any signs... signs enter squared) give -1
    perm = g.permutation(k)
    assert abs(ws.warmstart_loss(Us[:, perm] * np.array([1, -1, 1, 1, -1.0]), lam, Us) + 1.0) < 1e-12
    U = g.standard_normal((k, k))
    np.testing.assert_allclose(ws.warmstart_loss_grad(U, lam, Us),
                               _fd(lambda X: ws.warmstart_loss(X, lam, Us), U), rtol=1e-6,
                               atol=1e-7)


def test_sketch_and_initial_components_on_orthogonal_tensor():
    g = np.random.default_rng(7)
    k = 4
    Us, _ = np.linalg.qr(g.standard_normal((k, k)))
    lam = g.uniform(1, 3, k)
    T = np.einsum("j,aj,bj,cj->abc", lam, Us, Us, Us)
    th = g.standard_normal(k)
    # T(I,I,theta) = sum_j lam_j <u_j, theta> u_j u_j^T
    np.testing.assert_allclose(ws.sketch(T, th), (Us * (lam * (Us.T @ th))) @ Us.T, atol=1e-12)
    V0 = ws.initial_components(-Us, T, 1.0)
    Vs = (lam / stgd.kappa(1.0)) ** (1 / 3) * Us
    np.testing.assert_allclose(V0, Vs, atol=1e-12)
