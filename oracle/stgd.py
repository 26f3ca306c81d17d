"""Stochastic tensor gradient descent on the implicit whitened tensor, FP64 (oracle).

Section 3.2: the whitened tensor T, the loss Eq. (15), the stochastic update of
Lemma 3 / Eq. (16); Appendix A (gradient and the alpha0 "shift" terms).
Test infrastructure only (see the package docstring).

Readings of the paper used here:
  * Gram coefficient kappa.  Lemma 3 writes (1+theta)/2, Appendix A writes
    theta; they agree at theta = 1 (the paper's choice).  We use
    kappa = (1+theta)/2 (Lemma 3).
  * The factor 3 from differentiating the cubic is absorbed into the step size:
    the gradient is G = kappa V ((V^T V) o (V^T V)) - T(V, V, I), where column i
    of T(V, V, I) is T(v_i, v_i, I), and the update is V <- V - beta G.  The
    matching explicit loss is
        L~(V) = (kappa/2) sum_ij <v_i, v_j>^3 - <sum_i v_i^(x)3, T>,
    whose gradient is 3 G when the three views coincide.
  * The unit-norm constraint of Definition 1 is not enforced during SGD
    (Section 3.3 reads eigenvalues off the norms).
  * Lemma 3 contracts views A and B and leaves view C free; with three distinct
    views (community model) we follow it literally.
  * "y_B^t" in the alpha0^2 term of Lemma 3 is read as the mean y_B-bar.
  * y-bar is the full-data mean of each view (computed once).
  * A step uses the mean of the per-sample updates over a minibatch of b
    samples (the Gram term once per step); the last, partial minibatch of an
    epoch is kept and averaged over its own size.
  * Step size beta_t = beta0 / sqrt(t), t the global step counted from 1.
  * grad_implicit_topic_exact keeps the self-token terms of Eq. (3) that the
    sample tensor of Section 3.2 drops (its bias is O(1/l)): the data tensor is
    M3(W, W, W) of Eq. (3) estimated on the minibatch documents (per-document
    normalisation as for the moments, documents too short for a term add zero
    to it, the average over all b documents), M1 the full-data first moment.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .moments import as_sparse, coefficients

__all__ = [
    "kappa", "whitened_tensor", "whitened_tensor_chunked", "contract", "contract_all",
    "loss_explicit", "grad_explicit",
    "grad_implicit", "grad_implicit_gemm", "grad_implicit_topic_exact", "sgd_step", "sgd_run",
    "sgd_run_topic_exact", "steps_per_epoch",
]


def kappa(theta: float) -> float:
    """Gram-term coefficient of Lemma 3: (1 + theta) / 2."""
    return 0.5 * (1.0 + float(theta))


def whitened_tensor(YA, YB, YC, ybar3, alpha0: float) -> np.ndarray:
    """Section 3.2: T = c1 E_t[yA (x) yB (x) yC]
                        - c2 E_t[yA (x) yB (x) ybC + yA (x) ybB (x) yC + ybA (x) yB (x) yC]
                        + c3 ybA (x) ybB (x) ybC   (explicit k^3; small k)."""
    YA, YB, YC = (np.asarray(Y, dtype=np.float64) for Y in (YA, YB, YC))
    ybA, ybB, ybC = (np.asarray(y, dtype=np.float64) for y in ybar3)
    n = YA.shape[0]
    c1, c2, c3 = coefficients(alpha0)
    E = np.einsum("ti,tj,tk->ijk", YA, YB, YC) / n
    S = (np.einsum("ti,tj,k->ijk", YA, YB, ybC) + np.einsum("ti,j,tk->ijk", YA, ybB, YC)
         + np.einsum("i,tj,tk->ijk", ybA, YB, YC)) / n
    return c1 * E - c2 * S + c3 * np.einsum("i,j,k->ijk", ybA, ybB, ybC)


def whitened_tensor_chunked(YA, YB, YC, ybar3, alpha0: float, chunk: int = 8192) -> np.ndarray:
    """The tensor of whitened_tensor for many samples: the three sample sums of
    Section 3.2 formed chunk by chunk as matrix products, e.g.
    sum_t yA_t (x) yB_t (x) yC_t = reshape(YA^T [YB (row-wise x) YC]), and the mean
    terms from the full-data sums; same definition, other summation order."""
    YA, YB, YC = (np.asarray(Y, dtype=np.float64) for Y in (YA, YB, YC))
    ybA, ybB, ybC = (np.asarray(y, dtype=np.float64) for y in ybar3)
    n, k = YA.shape
    c1, c2, c3 = coefficients(alpha0)
    E = np.zeros((k, k * k))
    for t0 in range(0, n, chunk):
        a, bb, c = YA[t0:t0 + chunk], YB[t0:t0 + chunk], YC[t0:t0 + chunk]
        E += a.T @ (bb[:, :, None] * c[:, None, :]).reshape(len(a), k * k)
    E = E.reshape(k, k, k) / n
    AB = YA.T @ YB / n
    AC = YA.T @ YC / n
    BC = YB.T @ YC / n
    S = (np.einsum("ij,k->ijk", AB, ybC) + np.einsum("ik,j->ijk", AC, ybB)
         + np.einsum("jk,i->ijk", BC, ybA))
    return c1 * E - c2 * S + c3 * np.einsum("i,j,k->ijk", ybA, ybB, ybC)


def contract_all(T: np.ndarray, V: np.ndarray) -> np.ndarray:
    """contract(T, V) as one matrix product: column i = T_(3)^T (v_i (x) v_i), with
    T_(3) the k^2 x k unfolding of T and the Khatri-Rao columns v_i (x) v_i."""
    k = T.shape[0]
    KR = (V[:, None, :] * V[None, :, :]).reshape(k * k, V.shape[1])
    return T.reshape(k * k, k).T @ KR


def contract(T: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Column i = T(v_i, v_i, I): contraction of modes 1 and 2 with v_i."""
    return np.einsum("abc,ai,bi->ci", T, V, V)


def loss_explicit(V: np.ndarray, T: np.ndarray, theta: float) -> float:
    """L~(V) = (kappa/2) sum_ij <v_i, v_j>^3 - sum_i T(v_i, v_i, v_i)."""
    G = V.T @ V
    return 0.5 * kappa(theta) * np.sum(G ** 3) - np.einsum("abc,ai,bi,ci->", T, V, V, V)


def grad_explicit(V: np.ndarray, T: np.ndarray, theta: float) -> np.ndarray:
    """Gradient of L~ with respect to each v_i (all three modes of T)."""
    G = V.T @ V
    gram = 3.0 * kappa(theta) * V @ (G ** 2)
    t = (np.einsum("abc,bi,ci->ai", T, V, V) + np.einsum("abc,ai,ci->bi", T, V, V)
         + np.einsum("abc,ai,bi->ci", T, V, V))
    return gram - t


def grad_implicit(V, YA, YB, YC, ybar3, theta: float, alpha0: float) -> np.ndarray:
    """Lemma 3 (Eq. (16)) written per component i, averaged over the minibatch.

    For each i with phi = v_i:
      data_i = c1 mean_t[<phi,yA_t><phi,yB_t> yC_t] + c3 <phi,ybA><phi,ybB> ybC
             - c2 mean_t[<phi,yA_t><phi,yB_t>] ybC
             - c2 <phi,ybB> mean_t[<phi,yA_t> yC_t]
             - c2 <phi,ybA> mean_t[<phi,yB_t> yC_t]
      gram_i = sum_j <phi_j, phi>^2 phi_j
      G[:, i] = kappa gram_i - data_i.
    The tensor is never formed: only inner products with the samples.
    """
    V = np.asarray(V, dtype=np.float64)
    YA, YB, YC = (np.asarray(Y, dtype=np.float64) for Y in (YA, YB, YC))
    ybA, ybB, ybC = (np.asarray(y, dtype=np.float64) for y in ybar3)
    c1, c2, c3 = coefficients(alpha0)
    kap = kappa(theta)
    k = V.shape[1]
    G = np.empty_like(V)
    for i in range(k):
        phi = V[:, i]
        a = YA @ phi
        b = YB @ phi
        pa = phi @ ybA
        pb = phi @ ybB
        data = (c1 * np.mean((a * b)[:, None] * YC, axis=0)
                + c3 * pa * pb * ybC
                - c2 * np.mean(a * b) * ybC
                - c2 * pb * np.mean(a[:, None] * YC, axis=0)
                - c2 * pa * np.mean(b[:, None] * YC, axis=0))
        gram = np.zeros(V.shape[0])
        for j in range(k):
            gram += (V[:, j] @ phi) ** 2 * V[:, j]
        G[:, i] = kap * gram - data
    return G


def grad_implicit_gemm(V, YA, YB, YC, ybar3, theta: float, alpha0: float) -> np.ndarray:
    """Lemma 3 (Eq. (16)) for all components at once: the same sums as
    grad_implicit, grouped into products of the minibatch matrices (b x k):
      A_A = Y_A V, A_B = Y_B V, a_A = V^T ybar_A, a_B = V^T ybar_B,
      B = c1 A_A o A_B - c2 (A_A diag(a_B) + A_B diag(a_A)),
      data = Y_C^T B / b + ybar_C (c3 a_A o a_B - c2 mean_t (A_A o A_B))^T,
      G = kappa V ((V^T V) o (V^T V)) - data.
    Column i of every matrix is component i."""
    V = np.asarray(V, dtype=np.float64)
    YA, YB, YC = (np.asarray(Y, dtype=np.float64) for Y in (YA, YB, YC))
    ybA, ybB, ybC = (np.asarray(y, dtype=np.float64) for y in ybar3)
    c1, c2, c3 = coefficients(alpha0)
    b = YA.shape[0]
    AA = YA @ V
    AB = AA if YB is YA else YB @ V
    aA = V.T @ ybA
    aB = V.T @ ybB
    P = AA * AB
    B = c1 * P - c2 * (AA * aB[None, :] + AB * aA[None, :])
    data = YC.T @ B / b + np.outer(ybC, c3 * aA * aB - c2 * P.mean(axis=0))
    H = V.T @ V
    return kappa(theta) * V @ (H * H) - data


def grad_implicit_topic_exact(V, Xb, W, M1, theta: float, alpha0: float) -> np.ndarray:
    """Implicit gradient (Lemma 3 form, G = kappa V((V^T V)o2) - T(V, V, I)) for
    the topic model with the exact third moment of Eq. (3) whitened by W
    (d x k), estimated on the minibatch count rows Xb, without forming it.

    For component v, u = W v, and document t with counts c (length l),
    y' = W^T c, s = <c, u>, q = sum_j c_j u_j^2, r = W^T (c o u),
    z = W^T (c o u o u), m = W^T M1, mu = <m, v>:
      bracket of Eq. (3) at (u, u, W):   s^2 y' - q y' - 2 s r + 2 z
      pair moment P2 at (u, u):          s^2 - q
      P2 W v (positions (1,3) and (2,3)): s y' - r
      T_t(v, v, I) = c1 [s^2 y' - q y' - 2 s r + 2 z] / (l (l-1) (l-2))
                     - c2 ([s^2 - q] m + 2 mu [s y' - r]) / (l (l-1)),
    averaged over the b documents, plus c3 mu^2 m.
    """
    V = np.asarray(V, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    m = W.T @ np.asarray(M1, dtype=np.float64)
    Xs = as_sparse(Xb)
    n = Xs.shape[0]
    c1, c2, c3 = coefficients(alpha0)
    kap = kappa(theta)
    k = V.shape[1]
    G = np.empty_like(V)
    for i in range(k):
        v = V[:, i]
        u = W @ v
        mu = m @ v
        acc = np.zeros(V.shape[0])
        for t in range(n):
            lo, hi = Xs.indptr[t], Xs.indptr[t + 1]
            idx = Xs.indices[lo:hi]
            c = Xs.data[lo:hi]
            l = c.sum()
            Wt = W[idx]
            ut = u[idx]
            yp = Wt.T @ c
            s_ = yp @ v
            q = c @ (ut * ut)
            r = Wt.T @ (c * ut)
            z = Wt.T @ (c * ut * ut)
            if l >= 3:
                acc += c1 * (s_ * s_ * yp - q * yp - 2.0 * s_ * r + 2.0 * z) / (
                    l * (l - 1.0) * (l - 2.0))
            if l >= 2:
                acc -= c2 * ((s_ * s_ - q) * m + 2.0 * mu * (s_ * yp - r)) / (l * (l - 1.0))
        data = acc / n + c3 * mu * mu * m
        gram = np.zeros(V.shape[0])
        for j in range(k):
            gram += (V[:, j] @ v) ** 2 * V[:, j]
        G[:, i] = kap * gram - data
    return G


def sgd_step(V, YA, YB, YC, ybar3, theta: float, beta: float, alpha0: float,
             gemm: bool = False) -> np.ndarray:
    """One update of Lemma 3 over a minibatch: V <- V - beta G (G per component,
    or in the matrix form of grad_implicit_gemm when gemm is set)."""
    grad = grad_implicit_gemm if gemm else grad_implicit
    return np.asarray(V, dtype=np.float64) - beta * grad(V, YA, YB, YC, ybar3, theta, alpha0)


def steps_per_epoch(n: int, b: int) -> int:
    return (n + b - 1) // b


def sgd_run(V0, YA, YB, YC, ybar3, perm: np.ndarray, b: int, beta0: float,
            theta: float, alpha0: float, snapshot_every: int = 0, max_steps: int = -1,
            gemm: bool = False):
    """The STGD loop (Section 3.2): for each epoch e the samples are visited in the
    order perm[e], in minibatches of b; beta_t = beta0/sqrt(t).

    Returns the final V and, if snapshot_every > 0, the list of V after every
    snapshot_every-th step.  max_steps >= 0 stops early (bounded CPU samples).
    gemm selects the matrix form of the gradient (grad_implicit_gemm).
    """
    V = np.asarray(V0, dtype=np.float64).copy()
    YA, YB, YC = (np.asarray(Y, dtype=np.float64) for Y in (YA, YB, YC))
    n = YA.shape[0]
    snaps = []
    t = 0
    for order in perm:
        for s in range(0, n, b):
            if 0 <= max_steps <= t:
                return V, snaps
            idx = order[s:s + b]
            t += 1
            V = sgd_step(V, YA[idx], YB[idx], YC[idx], ybar3, theta,
                         beta0 / np.sqrt(t), alpha0, gemm=gemm)
            if snapshot_every and t % snapshot_every == 0:
                snaps.append(V.copy())
    return V, snaps


def sgd_run_topic_exact(V0, X, W, M1, perm: np.ndarray, b: int, beta0: float, theta: float,
                        alpha0: float, snapshot_every: int = 0):
    """The STGD loop of sgd_run (same visiting order, minibatches, partial last
    batch and beta_t = beta0/sqrt(t)) with the gradient of
    grad_implicit_topic_exact: the minibatch is the count rows perm[e][s:s+b] of
    X; an index outside [0, n) is an empty document."""
    V = np.asarray(V0, dtype=np.float64).copy()
    Xs = as_sparse(X)
    n = Xs.shape[0]
    Xz = sp.vstack([Xs, sp.csr_matrix((1, Xs.shape[1]))]).tocsr()  # row n: an empty document
    snaps = []
    t = 0
    for order in perm:
        for s in range(0, n, b):
            idx = np.asarray(order[s:s + b], dtype=np.int64)
            idx = np.where((idx >= 0) & (idx < n), idx, n)
            t += 1
            V = V - (beta0 / np.sqrt(t)) * grad_implicit_topic_exact(V, Xz[idx], W, M1, theta,
                                                                     alpha0)
            if snapshot_every and t % snapshot_every == 0:
                snaps.append(V.copy())
    return V, snaps

