"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np


def rel(a, b):
    """Normwise relative difference ||a - b|| / ||b||."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def align_signs(A, B):
    """Flip the columns of A to best match B (eigenvector sign ambiguity)."""
    s = np.sign(np.sum(np.asarray(A) * np.asarray(B), axis=0))
    s[s == 0] = 1.0
    return np.asarray(A) * s


def to_np(t):
    return t.detach().cpu().numpy()


def grad_rel_err(G, G64, V, theta, kappa_gram_data):
    """Normwise error of a gradient relative to its two terms:
    ||G - G64||_F / (||kappa G_gram||_F + ||G_data||_F)."""
    gram, data = kappa_gram_data
    return float(np.linalg.norm(G - G64) / (np.linalg.norm(gram) + np.linalg.norm(data)))


def grad_errs(Gk, G, gram):
    """(Frobenius, worst column) of ||Gk - G|| / (||kappa G_gram|| + ||G_data||),
    with G_data = gram - G; columns are components.  The column-wise ratio keeps a
    wrong component from hiding inside the Frobenius norm."""
    Gk, G, gram = (np.asarray(x, dtype=np.float64) for x in (Gk, G, gram))
    data = gram - G
    frob = np.linalg.norm(Gk - G) / (np.linalg.norm(gram) + np.linalg.norm(data))
    col = np.linalg.norm(Gk - G, axis=0) / (np.linalg.norm(gram, axis=0)
                                            + np.linalg.norm(data, axis=0))
    return float(frob), float(col.max())
