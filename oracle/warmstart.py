"""Learned warm start for the STGD (not in the paper), FP64 (oracle).

A small MLP maps sketches of the whitened tensor, S_j = T(I, I, theta_j) for a
few random unit theta_j, to an initial component matrix: its k x k output M is
orthonormalised by Gram-Schmidt (U0 = GS(M)) and each column is scaled to the
stationary norm of Lemma 3, v_i = (T(u_i, u_i, u_i) / kappa)^{1/3} u_i (with
u_i -> -u_i when T(u_i, u_i, u_i) < 0).  Training minimises the permutation-
and sign-invariant loss
    L(U) = - sum_i T*(u_i, u_i, u_i)^2 / sum_j lam_j^2,
T* = sum_j lam_j u*_j^(x)3 the instance's known decomposition; L = -1 exactly
when U recovers the components.  Test infrastructure only.

MLP: x (4 k^2) -> GELU(W1 x + b1) (512) -> GELU(W2 h1 + b2) (512) -> W3 h2 + b3
(k^2, read row-major as the k x k matrix M whose columns are Gram-Schmidt'ed).
GELU(z) = z Phi(z) (exact, Phi the standard normal CDF).  The input is the
concatenated sketches scaled to unit root-mean-square (mlp_input).  Training:
the batch-mean loss, its gradient through Gram-Schmidt and the MLP, and Adam
(Kingma & Ba 2015, Algorithm 1).  The network works in a canonical frame: the
eigenvectors E of the first sketch (canonical_frame); its input is the
sketches E^T S_j E and its output directions are rotated back by E, so the
map it learns does not depend on the arbitrary orientation of the whitened
coordinates.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .stgd import kappa, whitened_tensor

__all__ = ["sketch", "sketches", "gelu", "gelu_grad", "init_params", "mlp_forward",
           "mlp_backward", "gram_schmidt", "gram_schmidt_backward", "tensor_eval",
           "warmstart_loss", "warmstart_loss_grad", "initial_components", "mlp_input",
           "adam_step", "batch_loss_and_grad", "infer", "canonical_frame",
           "canonical_input"]


def sketch(T: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """S = T(I, I, theta): contraction of mode 3 with theta (definition)."""
    return np.einsum("abc,c->ab", T, theta)


def sketches(Y, ybar, alpha0: float, thetas: np.ndarray) -> np.ndarray:
    """Sketches of the symmetric whitened tensor of Section 3.2 (explicit T)."""
    T = whitened_tensor(Y, Y, Y, (ybar, ybar, ybar), alpha0)
    return np.stack([sketch(T, th) for th in thetas])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def init_params(seed: int, d_in: int, width: int, d_out: int) -> dict:
    g = np.random.default_rng(seed)
    return {"W1": g.standard_normal((width, d_in)) / math.sqrt(d_in), "b1": np.zeros(width),
            "W2": g.standard_normal((width, width)) / math.sqrt(width), "b2": np.zeros(width),
            "W3": g.standard_normal((d_out, width)) / math.sqrt(width), "b3": np.zeros(d_out)}


def mlp_forward(x: np.ndarray, p: dict):
    """x: batch x d_in.  Returns the output and the cache for the backward pass."""
    z1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (x, z1, h1, z2, h2)


def mlp_backward(dout: np.ndarray, p: dict, cache) -> dict:
    """Gradients of the parameters given dL/d(out) (batch x d_out)."""
    x, z1, h1, z2, h2 = cache
    g = {"W3": dout.T @ h2, "b3": dout.sum(axis=0)}
    dz2 = (dout @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return g


def gram_schmidt(M: np.ndarray):
    """Modified Gram-Schmidt on the columns of M: M = U R, U orthonormal,
    R upper triangular with positive diagonal."""
    k = M.shape[1]
    U = np.array(M, dtype=np.float64, copy=True)
    R = np.zeros((k, k))
    for i in range(k):
        for j in range(i):
            R[j, i] = U[:, j] @ U[:, i]
            U[:, i] -= R[j, i] * U[:, j]
        R[i, i] = np.linalg.norm(U[:, i])
        U[:, i] /= R[i, i]
    return U, R


def gram_schmidt_backward(U: np.ndarray, R: np.ndarray, dU: np.ndarray) -> np.ndarray:
    """dL/dM from dL/dU for M = U R (thin QR with R's diagonal positive):
    dM = (dU + U copyltu(-dU^T U)) R^{-T}, copyltu(A) = tril(A) + tril(A, -1)^T."""
    A = -dU.T @ U
    C = np.tril(A) + np.tril(A, -1).T
    return np.linalg.solve(R, (dU + U @ C).T).T


def tensor_eval(lam: np.ndarray, Ustar: np.ndarray, U: np.ndarray):
    """T*(u_i, u_i, u_i) and T*(u_i, u_i, I) for T* = sum_j lam_j u*_j^(x)3."""
    C = Ustar.T @ U                    # C[j, i] = <u*_j, u_i>
    t3 = (lam[:, None] * C ** 3).sum(axis=0)
    t2 = Ustar @ (lam[:, None] * C ** 2)   # column i = sum_j lam_j <u*_j,u_i>^2 u*_j
    return t3, t2


def warmstart_loss(U, lam, Ustar) -> float:
    t3, _ = tensor_eval(lam, Ustar, U)
    return float(-(t3 ** 2).sum() / (lam ** 2).sum())


def warmstart_loss_grad(U, lam, Ustar) -> np.ndarray:
    """dL/dU: column i = -6 T*(u_i,u_i,u_i) T*(u_i,u_i,I) / sum lam^2."""
    t3, t2 = tensor_eval(lam, Ustar, U)
    return -6.0 * t2 * t3 / (lam ** 2).sum()


def initial_components(U0: np.ndarray, T: np.ndarray, theta: float) -> np.ndarray:
    """V0 column i = (T(u_i,u_i,u_i)/kappa)^{1/3} u_i, sign chosen so that
    T(u_i,u_i,u_i) >= 0 (explicit tensor; Lemma 3 stationary scaling)."""
    t = np.einsum("abc,ai,bi,ci->i", T, U0, U0, U0)
    s = np.where(t < 0, -1.0, 1.0)
    return (U0 * s) * (np.abs(t) / kappa(theta)) ** (1.0 / 3.0)


def mlp_input(S: np.ndarray) -> np.ndarray:
    """Network input of one instance: vec(S_1, ..., S_J) (row-major) scaled so
    that its root-mean-square is 1."""
    x = np.asarray(S, dtype=np.float64).reshape(-1)
    return x * math.sqrt(x.size) / np.linalg.norm(x)


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def batch_loss_and_grad(params: dict, X: np.ndarray, Ustar: np.ndarray, lam: np.ndarray,
                        k: int):
    """Batch-mean warm-start loss of the network outputs and its parameter
    gradient.  X: B x d_in inputs, Ustar: B x k x k (columns u*_i), lam: B x k."""
    out, cache = mlp_forward(X, params)
    B = X.shape[0]
    dout = np.zeros_like(out)
    loss = 0.0
    for b in range(B):
        U, R = gram_schmidt(out[b].reshape(k, k))
        loss += warmstart_loss(U, lam[b], Ustar[b]) / B
        dU = warmstart_loss_grad(U, lam[b], Ustar[b])
        dout[b] = gram_schmidt_backward(U, R, dU).reshape(-1) / B
    return loss, mlp_backward(dout, params, cache)


def infer(params: dict, X: np.ndarray, k: int) -> np.ndarray:
    """Orthonormal initial directions U0 (B x k x k, columns) for inputs X."""
    out, _ = mlp_forward(X, params)
    return np.stack([gram_schmidt(o.reshape(k, k))[0] for o in out])


def canonical_frame(S1: np.ndarray):
    """Eigenvectors of the symmetric part of S1 (library eigh), ordered by
    descending eigenvalue, each with its largest-magnitude entry positive."""
    w, V = np.linalg.eigh(0.5 * (S1 + S1.T))
    order = np.argsort(-w, kind="stable")
    E = V[:, order]
    idx = np.argmax(np.abs(E), axis=0)
    E = E * np.where(E[idx, np.arange(E.shape[1])] < 0, -1.0, 1.0)
    return E, w[order]


def canonical_input(S: np.ndarray):
    """Network input in the canonical frame of S[0] and the frame E:
    mlp_input([E^T S_j E]_j)."""
    E, _ = canonical_frame(S[0])
    return mlp_input(np.stack([E.T @ Sj @ E for Sj in S])), E
