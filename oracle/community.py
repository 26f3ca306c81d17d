"""Community membership estimate and its validation, FP64 (oracle).

Section 3.3 Lemma 4 (community case): from the STGD components Phi and their
eigenvalues Lambda, the membership of the nodes of A^c is
    Pi_hat_{A^c} = diag(gamma)^{1/3} diag(Lambda)^{-1} Phi^T W^T G_{A,A^c},
followed by thresholding.  Section "Validation methods": Pearson correlation of
every estimated row Pi_hat_i with every ground-truth row Pi_j, Student-t
statistic T_ij = rho sqrt(n-2) / sqrt(1 - rho^2), right p-value against
t_{n-2}, a bipartite graph of pairs whose p-value is at most 0.01, the recovery
ratio R (fraction of ground-truth communities with at least one pair) and the
average error E (per pair, the l1 distance of the two rows divided by n,
summed over pairs, divided by k).
Test infrastructure only (see the package docstring).

Readings of the paper used here:
  * Phi holds unit columns u_i = v_i / ||v_i|| and Lambda the eigenvalues
    lambda_i = kappa ||v_i||^3 of the post-processing step.  With those, for
    the population moments Phi^T W^T E[G_{A,x}] = diag(Lambda) pi_x, so the
    formula returns pi_x exactly; keeping the norm ||v_i|| inside Phi would
    scale row i by lambda_i^{1/3} and give no such identity.
  * gamma is the one scalar fixed by the normalisation of the Dirichlet
    estimate: alpha_hat_i = gamma^2 lambda_i^-2 with sum_i alpha_hat_i = 1,
    so gamma = (sum_i lambda_i^-2)^{-1/2} and diag(gamma) = gamma I (it equals
    1 for population moments).
  * G_{A,A^c} restricted to the X nodes is G_{X,A}^T (an undirected graph), so
    Phi^T W^T G_{A,X} = (Y_A Phi)^T with Y_A = G_{X,A} W the whitened samples
    of view A: the membership of the X nodes is computed from Y_A.
  * Thresholding: entries below tau are set to 0; tau = -inf keeps every
    entry.  The rows are not renormalised afterwards (the paper does not say).
  * The printed p-value "1 - P(t > T)" contradicts the rule that pairs with a
    p-value at most 0.01 are the significant ones; the right p-value is read
    as P(t_{n-2} > T), small for strongly positive correlation.
  * rho of a row with zero variance (for instance an all-zero thresholded row)
    is taken as 0 (no evidence of dependence), so its p-value is 1/2.
  * Indices: rows i run over the k_hat estimated communities, columns j over
    the k ground-truth communities; a pair (i, j) is an edge when
    p(i, j) <= threshold; the degree of ground-truth community j counts its
    edges.
"""
from __future__ import annotations

import numpy as np
from scipy import special

from .post import eigenvalues

__all__ = ["membership", "pearson", "t_statistic", "right_pvalue", "pvalue_matrix",
           "match_scores"]


def membership(YA, V, theta: float, tau: float = -np.inf) -> np.ndarray:
    """Lemma 4, community case: Pi_hat (k x n) for the n nodes whose whitened
    view-A rows are YA (n x k); V holds the STGD components v_i as columns."""
    YA = np.asarray(YA, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    lam = eigenvalues(V, theta)
    Phi = V / np.linalg.norm(V, axis=0)
    gamma = np.sum(lam ** -2.0) ** -0.5
    Pi_hat = gamma ** (1.0 / 3.0) * (np.diag(1.0 / lam) @ Phi.T @ YA.T)
    return np.where(Pi_hat >= tau, Pi_hat, 0.0)


def pearson(a, b) -> float:
    """Pearson correlation of two length-n vectors; 0 when either is constant."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    da = a - a.mean()
    db = b - b.mean()
    saa = float(da @ da)
    sbb = float(db @ db)
    if saa == 0.0 or sbb == 0.0:
        return 0.0
    return float(da @ db) / np.sqrt(saa * sbb)


def t_statistic(rho: float, n: int) -> float:
    """T = rho sqrt(n-2) / sqrt(1 - rho^2), infinite at |rho| = 1."""
    if rho >= 1.0:
        return np.inf
    if rho <= -1.0:
        return -np.inf
    return rho * np.sqrt(n - 2.0) / np.sqrt(1.0 - rho * rho)


def right_pvalue(T: float, dof: float) -> float:
    """P(t_dof > T) for Student's t distribution (the library CDF at -T)."""
    return float(special.stdtr(dof, -T))


def pvalue_matrix(Pi_hat, Pi) -> np.ndarray:
    """p(i, j) = right p-value of the correlation of Pi_hat_i with Pi_j
    (k_hat x k), over the n columns (nodes)."""
    Pi_hat = np.asarray(Pi_hat, dtype=np.float64)
    Pi = np.asarray(Pi, dtype=np.float64)
    n = Pi.shape[1]
    if n < 3:
        raise ValueError("the t statistic needs n >= 3 nodes")
    P = np.empty((Pi_hat.shape[0], Pi.shape[0]))
    for i in range(Pi_hat.shape[0]):
        for j in range(Pi.shape[0]):
            P[i, j] = right_pvalue(t_statistic(pearson(Pi_hat[i], Pi[j]), n), n - 2)
    return P


def match_scores(Pi_hat, Pi, threshold: float = 0.01) -> dict:
    """Recovery ratio R and average error E over the p-value graph."""
    Pi_hat = np.asarray(Pi_hat, dtype=np.float64)
    Pi = np.asarray(Pi, dtype=np.float64)
    k, n = Pi.shape
    P = pvalue_matrix(Pi_hat, Pi)
    edges = P <= threshold
    l1 = np.abs(Pi_hat[:, None, :] - Pi[None, :, :]).sum(axis=2) / n
    degree = edges.sum(axis=0)
    R = float(np.count_nonzero(degree > 0)) / k
    E = float(l1[edges].sum()) / k
    return {"pvalues": P, "edges": edges, "l1": l1, "degree": degree, "recovery": R,
            "error": E}
