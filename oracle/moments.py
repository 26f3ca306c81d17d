"""Empirical moments of the topic and community models, FP64 (oracle).

Topic model, Section 2.1 Eqs. (1)-(3); community model (MMSB), Section 2.2
Eqs. (7)-(11).  Test infrastructure only (see the package docstring).

Readings of the paper used here:
  * Document-length normalisation (topic model).  Eqs. (1)-(3) as printed use raw
    counts, but Lemma 1 (E[M2] = sum_i alpha_hat_i mu_i mu_i^T) only holds for
    counts normalised per document.  We weight the first moment by 1/l_t, the
    pair term by 1/(l_t (l_t - 1)) and the triple term by
    1/(l_t (l_t - 1) (l_t - 2)).  Documents too short for a term (l_t < 1, < 2,
    < 3) contribute zero to it; n is always the number of documents.
  * The alpha0 correction of Eq. (3) is printed with diag(c_t) (x) M1; we read it
    as the pair moment (x) M1 in each of the three positions, which is the
    correction that makes Lemma 1 hold.
  * Pairs(Y1, Y2) = (1/n_X) G_{X,Y1}^T G_{X,Y2}; the pseudo-inverses in Eqs. (7)-(8)
    are taken at rank k.
  * Eq. (10): the symmetric part of M2 is what gets whitened.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = [
    "as_sparse", "coefficients", "doc_lengths", "topic_first_moment",
    "topic_pair_weights", "topic_pair_moment", "topic_second_moment",
    "topic_second_moment_apply", "topic_triple_moment", "topic_third_moment",
    "pairs", "pinv_rank", "transition_matrices", "community_first_moment",
    "community_second_moment", "community_third_moment", "outer3",
]


def as_sparse(X) -> sp.csr_matrix:
    """CSR-like object (row_ptr/col/val/shape), scipy matrix or dense -> float64 CSR."""
    if sp.issparse(X):
        return sp.csr_matrix(X, dtype=np.float64)
    if hasattr(X, "row_ptr"):
        return sp.csr_matrix((np.asarray(X.val, np.float64), np.asarray(X.col),
                              np.asarray(X.row_ptr)), shape=tuple(X.shape))
    return sp.csr_matrix(np.asarray(X, dtype=np.float64))


def coefficients(alpha0: float):
    """The Dirichlet weights of the whitened tensor (Section 3.2) and Eq. (16):
    c1 = (a0+1)(a0+2)/2, c2 = a0(a0+1)/2, c3 = a0^2."""
    a0 = float(alpha0)
    return (a0 + 1.0) * (a0 + 2.0) / 2.0, a0 * (a0 + 1.0) / 2.0, a0 * a0


def outer3(a, b, c) -> np.ndarray:
    return np.einsum("i,j,k->ijk", a, b, c)


def _doc_weights(n: int, weights):
    """Per-document averaging weights: 1/n by default (Eqs. (1)-(3))."""
    if weights is None:
        return np.full(n, 1.0 / n)
    w = np.asarray(weights, dtype=np.float64)
    return w / w.sum()


def doc_lengths(X) -> np.ndarray:
    """l_t = sum_w c_{w,t} (number of words in document t)."""
    return np.asarray(as_sparse(X).sum(axis=1)).ravel()


def topic_first_moment(X, weights=None) -> np.ndarray:
    """Eq. (1), length-normalised: M1 = (1/n) sum_t c_t / l_t."""
    Xs = as_sparse(X)
    l = doc_lengths(Xs)
    inv = np.where(l > 0, 1.0 / np.maximum(l, 1.0), 0.0)
    return Xs.T @ (inv * _doc_weights(Xs.shape[0], weights))


def topic_pair_weights(l: np.ndarray) -> np.ndarray:
    """1 / (l (l - 1)) for documents with at least two words, else 0."""
    l = np.asarray(l, dtype=np.float64)
    return np.where(l >= 2, 1.0 / np.maximum(l * (l - 1.0), 1.0), 0.0)


def topic_pair_moment(X, weights=None) -> np.ndarray:
    """E[x1 (x) x2] estimated as (1/n) sum_t (c_t c_t^T - diag(c_t)) / (l_t (l_t-1)).

    The bracket counts ordered pairs of distinct word positions (Eq. (2))."""
    Xs = as_sparse(X)
    n = Xs.shape[0]
    w = topic_pair_weights(doc_lengths(Xs)) * _doc_weights(n, weights)
    Xw = sp.diags(w) @ Xs
    out = (Xs.T @ Xw).toarray()
    out -= np.diag(np.asarray(Xw.sum(axis=0)).ravel())
    return out


def topic_second_moment(X, alpha0: float, weights=None) -> np.ndarray:
    """Eq. (2): M2 = (a0+1) * pair moment - a0 M1 M1^T (dense d x d; small d only)."""
    M1 = topic_first_moment(X, weights)
    return (alpha0 + 1.0) * topic_pair_moment(X, weights) - alpha0 * np.outer(M1, M1)


def topic_second_moment_apply(X, S: np.ndarray, alpha0: float) -> np.ndarray:
    """M2 @ S for Eq. (2) without forming M2 (same algebra, any d):
    (a0+1) [X^T diag(w) (X S) - diag(X^T w) S] / n - a0 M1 (M1^T S)."""
    Xs = as_sparse(X)
    n = Xs.shape[0]
    S = np.asarray(S, dtype=np.float64)
    w = topic_pair_weights(doc_lengths(Xs)) / n
    delta = Xs.T @ w
    M1 = topic_first_moment(Xs)
    pair = Xs.T @ (w[:, None] * (Xs @ S)) - delta[:, None] * S
    return (alpha0 + 1.0) * pair - alpha0 * np.outer(M1, M1 @ S)


def topic_triple_moment(X, weights=None) -> np.ndarray:
    """E[x1 (x) x2 (x) x3]: ordered triples of distinct word positions (Eq. (3)
    bracket), per document divided by l(l-1)(l-2), averaged.  Dense d^3."""
    Xs = as_sparse(X)
    n, d = Xs.shape
    wd = _doc_weights(n, weights)
    out = np.zeros((d, d, d))
    eye = np.eye(d)
    for t in range(n):
        c = Xs.getrow(t).toarray().ravel()
        l = c.sum()
        if l < 3:
            continue
        cc = np.outer(c, c)
        term = outer3(c, c, c)
        term -= np.einsum("ij,ia->iaj", cc, eye)      # sum_ij c_i c_j e_i e_i e_j
        term -= np.einsum("ij,ia->ija", cc, eye)      # sum_ij c_i c_j e_i e_j e_i
        term -= np.einsum("ij,ja->ija", cc, eye)      # sum_ij c_i c_j e_i e_j e_j
        term += 2.0 * np.einsum("i,ia,ib->iab", c, eye, eye)
        out += wd[t] * term / (l * (l - 1.0) * (l - 2.0))
    return out


def topic_third_moment(X, alpha0: float, weights=None) -> np.ndarray:
    """Eq. (3): M3 = c1 E[x1x2x3] - c2 (P2 (x) M1 + perms) + c3 M1^(x)3."""
    c1, c2, c3 = coefficients(alpha0)
    M1 = topic_first_moment(X, weights)
    P2 = topic_pair_moment(X, weights)
    E3 = topic_triple_moment(X, weights)
    corr = (np.einsum("ij,k->ijk", P2, M1) + np.einsum("ik,j->ijk", P2, M1)
            + np.einsum("jk,i->ijk", P2, M1))
    return c1 * E3 - c2 * corr + c3 * outer3(M1, M1, M1)


# --------------------------------------------------------------------------
# Community model (MMSB), Section 2.2
# --------------------------------------------------------------------------

def pairs(G_XY1, G_XY2) -> np.ndarray:
    """Pairs(Y1, Y2) = (1/n_X) G_{X,Y1}^T G_{X,Y2} (dense; small graphs)."""
    a = as_sparse(G_XY1)
    b = as_sparse(G_XY2)
    return (a.T @ b).toarray() / a.shape[0]


def pinv_rank(M: np.ndarray, k: int) -> np.ndarray:
    """Rank-k pseudo-inverse from the top-k singular triplets (Section 4.1)."""
    U, s, Vt = np.linalg.svd(M)
    return (Vt[:k].T / s[:k]) @ U[:, :k].T


def transition_matrices(G_XA, G_XB, G_XC, k: int):
    """Eqs. (7)-(8): Z_B = Pairs(A,C) Pairs(B,C)^+, Z_C = Pairs(A,B) Pairs(C,B)^+."""
    Z_B = pairs(G_XA, G_XC) @ pinv_rank(pairs(G_XB, G_XC), k)
    Z_C = pairs(G_XA, G_XB) @ pinv_rank(pairs(G_XC, G_XB), k)
    return Z_B, Z_C


def community_first_moment(G_XA) -> np.ndarray:
    """Eq. (9): M1 = (1/n_X) sum_x G_{x,A}^T."""
    a = as_sparse(G_XA)
    return np.asarray(a.sum(axis=0)).ravel() / a.shape[0]


def community_second_moment(G_XA, G_XB, G_XC, k: int, alpha0: float) -> np.ndarray:
    """Eq. (10): M2 = (a0+1) Z_C Pairs(C,B) Z_B^T - a0 M1 M1^T (as printed; not
    symmetrised -- callers whiten its symmetric part)."""
    Z_B, Z_C = transition_matrices(G_XA, G_XB, G_XC, k)
    M1 = community_first_moment(G_XA)
    return (alpha0 + 1.0) * Z_C @ pairs(G_XC, G_XB) @ Z_B.T - alpha0 * np.outer(M1, M1)


def community_third_moment(G_XA, G_XB, G_XC, k: int, alpha0: float) -> np.ndarray:
    """Eq. (11), explicit n_A^3 tensor (tiny graphs only)."""
    c1, c2, c3 = coefficients(alpha0)
    Z_B, Z_C = transition_matrices(G_XA, G_XB, G_XC, k)
    M1 = community_first_moment(G_XA)
    yA = as_sparse(G_XA).toarray()
    yB = as_sparse(G_XB).toarray() @ Z_B.T
    yC = as_sparse(G_XC).toarray() @ Z_C.T
    n = yA.shape[0]
    E = np.einsum("xi,xj,xk->ijk", yA, yB, yC) / n
    corr = (np.einsum("xi,xj,k->ijk", yA, yB, M1) + np.einsum("xi,j,xk->ijk", yA, M1, yC)
            + np.einsum("i,xj,xk->ijk", M1, yB, yC)) / n
    return c1 * E - c2 * corr + c3 * outer3(M1, M1, M1)
