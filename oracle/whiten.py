"""Whitening and randomised low-rank linear algebra, FP64 (oracle).

Section 3.1 (W^T M2 W = I, W = U Sigma^{-1/2} from the top-k eigenpairs) and
Section 4.2 (random projection of M2, tall-thin QR, Algorithms 2 and 3).
Test infrastructure only (see the package docstring).

Readings of the paper used here:
  * M2 may be indefinite (it is an empirical estimate): we take the symmetric
    eigendecomposition and keep the k LARGEST eigenvalues; if the k-th is not
    positive the whitening does not exist (error).
  * Eigenvector signs: the entry of largest magnitude of each eigenvector is
    made positive.
  * Randomised whitening, default form: the randomised range finder with
    oversampling p and q power iterations (Q = orth(M2 S), then
    Q <- orth(M2 Q) q times), Rayleigh-Ritz on Omega = Q^T M2 Q, truncation to
    k.  On the GPU the range finder uses the tall-thin QR of Section 4.2.
  * Randomised whitening, the paper's Nystrom form (Algorithm 2): O = M2 S,
    Omega = S^T O, W = U_O L_O^{-1} V_O^T V_Omega L_Omega^{1/2} with both
    decompositions truncated to rank k (O has rank k when M2 has, so its
    remaining singular values are rounding noise and L_O^{-1} would amplify
    them), Omega symmetrised and decomposed as a symmetric matrix (its SVD
    for a positive semi-definite Omega), its k largest eigenvalues required
    positive (relative to the largest, as for the exact whitening), and the
    trailing U_Omega^T of the printed formula dropped: it rotates the k
    columns back into k~ coordinates, and without it W is d x k with
    W^T M2 W = I_k whenever M2 has rank k.  (W^T)^+ = W (W^T W)^{-1}.
  * Randomised pseudo-inverse (Algorithm 3): its printed formula
    (J^+)^T Psi J^+ is a pseudo-inverse only for symmetric matrices; Pairs is
    not symmetric, so we compute the rank-k SVD P ~ U Sigma V^T by randomised
    subspace iteration with the same random projection and use
    P^+ = V Sigma^{-1} U^T.
"""
from __future__ import annotations

import numpy as np

from .moments import as_sparse, community_first_moment

__all__ = [
    "NotPositiveDefinite", "sign_fix", "orth", "top_eigh", "whiten_exact",
    "range_finder_whiten", "nystrom_whiten", "randomized_svd", "community_whiten_randomized",
]


class NotPositiveDefinite(ValueError):
    """Fewer than k positive eigenvalues: no whitening exists (Section 3.1)."""


def sign_fix(U: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude entry of every column positive."""
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s


def orth(Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Y) (library Householder QR, R diag >= 0)."""
    Q, R = np.linalg.qr(Y)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def top_eigh(A: np.ndarray, k: int):
    """The k largest eigenpairs of the symmetric part of A, descending, sign-fixed."""
    A = 0.5 * (A + A.T)
    lam, U = np.linalg.eigh(A)
    idx = np.argsort(lam)[::-1][:k]
    return lam[idx], sign_fix(U[:, idx])


def whiten_exact(M2: np.ndarray, k: int) -> dict:
    """Section 3.1: W = U_k Lambda_k^{-1/2}; W^+ := (W^T)^+ = U_k Lambda_k^{1/2}."""
    lam, U = top_eigh(M2, k)
    if lam[-1] <= 0:
        raise NotPositiveDefinite(f"k-th eigenvalue of M2 is {lam[-1]:.3e}")
    return {"W": U / np.sqrt(lam), "Wplus": U * np.sqrt(lam), "eig": lam, "U": U}


def range_finder_whiten(apply_M2, S: np.ndarray, k: int, power_iters: int) -> dict:
    """Section 4.2 randomised whitening (range-finder reading, see module doc).

    apply_M2(X) returns M2 @ X.  S is the d x k~ random projection (k~ = k + p).
    Returns W (d x k), W^+ (d x k), the basis Q (d x k~), the small factors
    Cw = U_k Lambda^{-1/2} and Cp = U_k Lambda^{1/2} (k~ x k) with
    W = Q Cw, W^+ = Q Cp, and the k eigenvalues of Omega = Q^T M2 Q.
    """
    Q = orth(apply_M2(np.asarray(S, dtype=np.float64)))
    for _ in range(power_iters):
        Q = orth(apply_M2(Q))
    Om = Q.T @ apply_M2(Q)
    lam, U = top_eigh(Om, k)
    if lam[-1] <= 0:
        raise NotPositiveDefinite(f"k-th eigenvalue of Omega is {lam[-1]:.3e}")
    Cw = U / np.sqrt(lam)
    Cp = U * np.sqrt(lam)
    return {"W": Q @ Cw, "Wplus": Q @ Cp, "Q": Q, "Cw": Cw, "Cp": Cp, "eig": lam,
            "Omega": 0.5 * (Om + Om.T)}


def nystrom_whiten(apply_M2, S: np.ndarray, k: int) -> dict:
    """Algorithm 2 (randomised tall-thin SVD), read as in the module doc:
    W (d x k), Wplus = (W^T)^+, eig = the k largest eigenvalues of Omega."""
    S = np.asarray(S, dtype=np.float64)
    O = apply_M2(S)                                     # O = M2 S
    U_O, L_O, Vt_O = np.linalg.svd(O, full_matrices=False)
    Omega = S.T @ O                                     # Omega = S^T O
    lam, V_Om = top_eigh(Omega, k)
    if not lam[-1] > 1e-5 * abs(lam[0]):
        raise NotPositiveDefinite(f"k-th eigenvalue of Omega is {lam[-1]:.3e}")
    W = (U_O[:, :k] / L_O[:k]) @ Vt_O[:k] @ (V_Om * np.sqrt(lam))
    Wplus = W @ np.linalg.inv(W.T @ W)
    return {"W": W, "Wplus": Wplus, "eig": lam}


def randomized_svd(apply_A, apply_AT, S: np.ndarray, k: int, power_iters: int):
    """Rank-k SVD A ~ U diag(sigma) V^T by randomised subspace iteration
    (Algorithm 3 reading, see module doc).  S is n_cols x k~."""
    Q = orth(apply_A(np.asarray(S, dtype=np.float64)))
    for _ in range(power_iters):
        Qt = orth(apply_AT(Q))
        Q = orth(apply_A(Qt))
    Bt = apply_AT(Q)                       # (Q^T A)^T, n_cols x k~
    ev, Ub = top_eigh(Bt.T @ Bt, k)        # B B^T = Ub diag(sigma^2) Ub^T
    if ev[-1] <= 0:
        raise NotPositiveDefinite("rank of Pairs is below k")
    sigma = np.sqrt(ev)
    return Q @ Ub, sigma, (Bt @ Ub) / sigma


def community_whiten_randomized(G_XA, G_XB, G_XC, k: int, alpha0: float,
                                S_pairs: np.ndarray, S_whiten: np.ndarray,
                                power_iters: int) -> dict:
    """Randomised whitening of the community model (Sections 4.1-4.2, Eq. (10)).

    1. Rank-k SVD of Pairs(C,B) = (1/n_X) G_XC^T G_XB ~ U_C Sigma V_B^T.
    2. Z_B = Pairs(A,C) Pairs(B,C)^+ = L_B V_B^T with L_B = Pairs(A,C) U_C Sigma^-1;
       Z_C = Pairs(A,B) Pairs(C,B)^+ = L_C U_C^T with L_C = Pairs(A,B) V_B Sigma^-1.
    3. M2 = (a0+1) Z_C Pairs(C,B) Z_B^T - a0 M1 M1^T = (a0+1) L_C K L_B^T - a0 M1 M1^T,
       K = U_C^T Pairs(C,B) V_B; its symmetric part is applied in factored form
       (no n x n product is ever formed, Section 4.1).
    4. Range-finder whitening of M2 (see range_finder_whiten).
    5. Whitening of the other views: W_B = Z_B^T W, W_C = Z_C^T W, so that
       y_B = W^T Z_B G_{x,B}^T = W_B^T G_{x,B}^T (Section 4.1, Appendix A).
    """
    A = as_sparse(G_XA)
    B = as_sparse(G_XB)
    C = as_sparse(G_XC)
    nX = A.shape[0]
    U_C, sigma, V_B = randomized_svd(lambda X: C.T @ (B @ X) / nX,
                                     lambda X: B.T @ (C @ X) / nX,
                                     S_pairs, k, power_iters)
    CU = C @ U_C
    BV = B @ V_B
    L_B = (A.T @ CU) / nX / sigma
    L_C = (A.T @ BV) / nX / sigma
    K = CU.T @ BV / nX
    M1 = community_first_moment(A)

    def apply_M2(X):
        t1 = L_C @ (K @ (L_B.T @ X))
        t2 = L_B @ (K.T @ (L_C.T @ X))
        return 0.5 * (alpha0 + 1.0) * (t1 + t2) - alpha0 * np.outer(M1, M1 @ X)

    out = range_finder_whiten(apply_M2, S_whiten, k, power_iters)
    out.update({"U_C": U_C, "sigma": sigma, "V_B": V_B, "L_B": L_B, "L_C": L_C,
                "K": K, "M1": M1,
                "W_B": V_B @ (L_B.T @ out["W"]), "W_C": U_C @ (L_C.T @ out["W"]),
                "apply_M2": apply_M2})
    return out
