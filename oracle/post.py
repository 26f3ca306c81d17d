"""Post-processing and error measures, FP64 (oracle).

Section 3.3 Lemma 4: eigenvalues lambda_i = ||phi_i||^3, topic estimate
mu = (W^T)^+ Phi, Dirichlet weights alpha_i ~ lambda_i^{-2} normalised to sum 1.
The reconstruction error is not in the paper; it measures convergence.
Test infrastructure only (see the package docstring).

Readings of the paper used here:
  * With the Gram coefficient kappa of Lemma 3 the stationary components have
    ||v_i||^3 = lambda_i / kappa, so lambda_i = kappa ||v_i||^3 (equal to the
    paper's ||phi_i||^3 at theta = 1).
  * mu_i = lambda_i (W^T)^+ u_i with u_i = v_i / ||v_i||: the exact inverse of the
    whitening when the population tensor is sum_i alpha_hat_i^{-1/2} u_i^(x)3.
    For topics each column is then sign-flipped to a non-negative sum and
    divided by its sum (a distribution over words).
  * No thresholding of the estimate (a tuning knob for real data).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment

from .stgd import kappa

__all__ = ["eigenvalues", "unwhiten", "tensor_from_components", "recon_error",
           "recon_error_from_V", "match_components"]


def eigenvalues(V: np.ndarray, theta: float) -> np.ndarray:
    """lambda_i = kappa ||v_i||^3 (Section 3.3)."""
    return kappa(theta) * np.linalg.norm(V, axis=0) ** 3


def unwhiten(V: np.ndarray, Wplus: np.ndarray, theta: float, normalize: bool) -> dict:
    """Lemma 4: mu_hat_i = lambda_i W^+ u_i; alpha_hat_i = lambda_i^-2 / sum_j lambda_j^-2."""
    V = np.asarray(V, dtype=np.float64)
    norms = np.linalg.norm(V, axis=0)
    lam = kappa(theta) * norms ** 3
    mu = (np.asarray(Wplus, dtype=np.float64) @ (V / norms)) * lam
    raw = mu.copy()
    if normalize:
        s = mu.sum(axis=0)
        mu = mu * np.where(s < 0, -1.0, 1.0)
        mu = mu / np.abs(s)
    a = lam ** -2.0
    return {"mu": mu, "raw": raw, "lambda": lam, "alpha_hat": a / a.sum()}


def tensor_from_components(lam: np.ndarray, U: np.ndarray) -> np.ndarray:
    """sum_i lam_i u_i (x) u_i (x) u_i (explicit; small k)."""
    return np.einsum("i,ai,bi,ci->abc", lam, U, U, U)


def recon_error(lam_hat, U_hat, lam_true, U_true) -> float:
    """||sum lam_hat u_hat^(x)3 - sum lam u^(x)3||_F / ||sum lam u^(x)3||_F in closed
    form, using <x^(x)3, y^(x)3> = <x, y>^3."""
    lh, Uh, lt, Ut = (np.asarray(a, dtype=np.float64) for a in (lam_hat, U_hat, lam_true, U_true))
    hh = lh @ (Uh.T @ Uh) ** 3 @ lh
    ht = lh @ (Uh.T @ Ut) ** 3 @ lt
    tt = lt @ (Ut.T @ Ut) ** 3 @ lt
    return float(np.sqrt(max(hh - 2.0 * ht + tt, 0.0) / tt))


def recon_error_from_V(V, theta, lam_true, U_true) -> float:
    """Reconstruction error of the SGD iterate: lam_hat u_hat^(x)3 = kappa v^(x)3."""
    V = np.asarray(V, dtype=np.float64)
    norms = np.linalg.norm(V, axis=0)
    return recon_error(kappa(theta) * norms ** 3, V / norms, lam_true, U_true)


def match_components(U_hat: np.ndarray, U_true: np.ndarray):
    """Permutation and signs matching estimated to true components (Hungarian
    assignment on |cos|).  Returns (perm, signs, max_abs_error) with
    U_hat[:, perm] * signs ~ U_true."""
    Uh = U_hat / np.linalg.norm(U_hat, axis=0)
    Ut = U_true / np.linalg.norm(U_true, axis=0)
    C = np.abs(Ut.T @ Uh)
    rows, cols = linear_sum_assignment(-C)
    perm = cols[np.argsort(rows)]
    signs = np.sign(np.sum(Uh[:, perm] * Ut, axis=0))
    signs[signs == 0] = 1.0
    err = float(np.max(np.abs(Uh[:, perm] * signs - Ut)))
    return perm, signs, err
