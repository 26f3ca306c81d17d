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


def test_batch_loss_and_grad_finite_differences():
    """The composite training gradient (MLP -> Gram-Schmidt -> loss, batch
    mean) equals central differences of the composite loss."""
    k, B = 3, 2
    p = ws.init_params(4, 2 * k * k, 6, k * k)
    g = np.random.default_rng(5)
    X = g.standard_normal((B, 2 * k * k))
    Us = np.stack([np.linalg.qr(g.standard_normal((k, k)))[0] for _ in range(B)])
    lam = g.uniform(0.5, 2.0, (B, k))
    _, grads = ws.batch_loss_and_grad(p, X, Us, lam, k)
    for key in ("W1", "b2", "W3"):
        def f(v, key=key):
            q = dict(p)
            q[key] = v
            return ws.batch_loss_and_grad(q, X, Us, lam, k)[0]
        np.testing.assert_allclose(grads[key], _fd(f, p[key]), rtol=1e-5, atol=1e-8)


def test_adam_matches_first_steps_by_hand():
    """Adam's bias correction: the first step moves every coordinate by
    lr * sign(g) (up to eps), the second by lr * mh / sqrt(vh) written out."""
    p = np.array([1.0, -2.0, 0.5])
    g1 = np.array([0.3, -4.0, 1e-3])
    p1, m, v = ws.adam_step(p, g1, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g1), atol=1e-7)
    g2 = np.array([-0.1, 2.0, 1e-3])
    p2, _, _ = ws.adam_step(p1, g2, m, v, 2, 0.01)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(p2, p1 - 0.01 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-12)


def test_mlp_input_unit_rms():
    S = np.random.default_rng(6).standard_normal((4, 5, 5)) * 7.0
    x = ws.mlp_input(S)
    assert x.shape == (100,)
    np.testing.assert_allclose(np.sqrt((x ** 2).mean()), 1.0, rtol=1e-12)
    np.testing.assert_allclose(x / x[0], S.reshape(-1) / S.reshape(-1)[0], rtol=1e-12)


def test_infer_orthonormal_columns():
    k = 4
    p = ws.init_params(7, 8, 6, k * k)
    U0 = ws.infer(p, np.random.default_rng(8).standard_normal((3, 8)), k)
    for U in U0:
        np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)


def test_canonical_frame_diagonalises_first_sketch():
    g = np.random.default_rng(9)
    A = g.standard_normal((6, 6))
    S = np.stack([A + A.T, g.standard_normal((6, 6))])
    E, w = ws.canonical_frame(S[0])
    D = E.T @ S[0] @ E
    np.testing.assert_allclose(D, np.diag(np.diag(D)), atol=1e-12)
    np.testing.assert_allclose(np.diag(D), w, atol=1e-12)
    assert np.all(np.diff(w) <= 0)
    idx = np.argmax(np.abs(E), axis=0)
    assert np.all(E[idx, np.arange(6)] > 0)
    x, E2 = ws.canonical_input(S)
    np.testing.assert_array_equal(E, E2)
    np.testing.assert_allclose(np.linalg.norm(x), np.linalg.norm(ws.mlp_input(S)), rtol=1e-12)


def test_sketches_match_implicit_formula():
    """The sketches built from the explicit whitened tensor equal the implicit
    form S_j = (1/n) Y^T diag(c1 Y th_j - c2 <th_j, yb>) Y - c2 (m_j yb^T + yb m_j^T)
    + c3 <th_j, yb> yb yb^T with m_j = (1/n) Y^T (Y th_j) (Section 3.2's tensor
    contracted in its third mode; no k^3 tensor)."""
    from oracle.moments import coefficients
    g = np.random.default_rng(9)
    n, k, alpha0 = 60, 5, 0.8
    Y = g.standard_normal((n, k)) + 0.2
    yb = Y.mean(axis=0)
    th = g.standard_normal((3, k))
    c1, c2, c3 = coefficients(alpha0)
    S = ws.sketches(Y, yb, alpha0, th)
    for j in range(3):
        a = Y @ th[j]
        m = Y.T @ a / n
        p = th[j] @ yb
        want = (Y.T * (c1 * a - c2 * p)) @ Y / n - c2 * (np.outer(m, yb) + np.outer(yb, m)) \
            + c3 * p * np.outer(yb, yb)
        np.testing.assert_allclose(S[j], want, rtol=1e-12, atol=1e-12)
