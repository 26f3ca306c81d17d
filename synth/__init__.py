"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random inputs: it holds none of the method's
arithmetic (no moments, no whitening, no gradients).  Everything it returns is
plain NumPy data that either side (the CPU oracle or the CUDA library) consumes
as an input array.

Generators:
  * :func:`lda_corpus`          -- LDA bag-of-words corpus as a CSR count matrix
                                   (the topic model of Section 2.1).
  * :func:`mmsb_graph`          -- mixed-membership stochastic blockmodel with
                                   Bernoulli edges, partitioned into X, A, B, C
                                   (Section 2.2); the three blocks X->A, X->B,
                                   X->C as CSR matrices.
  * :func:`orthogonal_samples`  -- whitened samples of an orthogonal tensor plus
                                   Gaussian noise (batched decomposition
                                   problems, already whitened).
  * :func:`gaussian`            -- seeded Gaussian test matrices (the random
                                   projection S of Section 4.2).
  * :func:`haar_orthonormal`    -- Haar-random orthonormal k x k matrix (the
                                   random initial components of the SGD).
  * :func:`epoch_permutations`  -- per-epoch sample orders for the SGD.

All generators use NumPy's PCG64 bit generator seeded with the given integer,
so both sides see bit-identical inputs.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "CSR", "lda_corpus", "mmsb_graph", "orthogonal_samples", "gaussian",
    "haar_orthonormal", "epoch_permutations", "csr_from_dense", "csr_to_dense",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


class CSR:
    """Compressed sparse row matrix: int32 row_ptr/col, float32 values."""

    __slots__ = ("row_ptr", "col", "val", "shape")

    def __init__(self, row_ptr, col, val, shape):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float32)
        self.shape = (int(shape[0]), int(shape[1]))

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def row_slice(self, r0: int, r1: int) -> "CSR":
        a, b = int(self.row_ptr[r0]), int(self.row_ptr[r1])
        return CSR(self.row_ptr[r0:r1 + 1] - a, self.col[a:b], self.val[a:b],
                   (r1 - r0, self.shape[1]))


def _csr_from_pairs(rows: np.ndarray, cols: np.ndarray, n_rows: int, n_cols: int) -> CSR:
    """Counts of (row, col) pairs as a CSR matrix with sorted columns per row."""
    key = rows.astype(np.int64) * n_cols + cols.astype(np.int64)
    uk, cnt = np.unique(key, return_counts=True)
    r = (uk // n_cols).astype(np.int64)
    c = (uk % n_cols).astype(np.int32)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(row_ptr, c, cnt.astype(np.float32), (n_rows, n_cols))


def csr_from_dense(a: np.ndarray) -> CSR:
    a = np.asarray(a)
    rows, cols = np.nonzero(a)
    row_ptr = np.zeros(a.shape[0] + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return CSR(np.cumsum(row_ptr), cols, a[rows, cols], a.shape)


def csr_to_dense(x: CSR, dtype=np.float64) -> np.ndarray:
    out = np.zeros(x.shape, dtype=dtype)
    rows = np.repeat(np.arange(x.shape[0]), np.diff(x.row_ptr))
    out[rows, x.col] = x.val
    return out


def lda_corpus(seed: int, n_docs: int, d: int, k: int, alpha_i: float,
               word_conc: float, doc_len: int, poisson_len: bool = False,
               zipf: bool = False) -> dict:
    """LDA corpus (Section 2.1): h_t ~ Dir(alpha_i * 1_k), words i.i.d. from mu h_t.

    Topic-word columns mu_j ~ Dir(word_conc * 1_d); with ``zipf`` the
    concentration is skewed as Dir(word_conc * d * z) with z_w proportional to
    1/w (same total concentration).  Document lengths are exactly ``doc_len``
    or Poisson(doc_len).  Returns the CSR count matrix (documents x vocabulary)
    and the ground truth (mu: d x k, alpha: k, h: n x k).
    """
    g = rng(seed)
    if zipf:
        z = 1.0 / np.arange(1, d + 1, dtype=np.float64)
        conc = word_conc * d * z / z.sum()
    else:
        conc = np.full(d, word_conc)
    mu = np.stack([g.dirichlet(conc) for _ in range(k)], axis=1)          # d x k
    alpha = np.full(k, float(alpha_i))
    h = g.dirichlet(alpha, size=n_docs)                                    # n x k
    if poisson_len:
        lens = g.poisson(doc_len, size=n_docs).astype(np.int64)
    else:
        lens = np.full(n_docs, int(doc_len), dtype=np.int64)
    # per-document topic counts, then per-topic word draws (vectorised)
    tok_doc = np.repeat(np.arange(n_docs, dtype=np.int64), lens)
    topic_counts = g.multinomial(lens, h)                                 # n x k
    # token topic ids in document order
    tok_topic = np.repeat(np.tile(np.arange(k), n_docs), topic_counts.ravel())
    words = np.empty(tok_doc.shape[0], dtype=np.int64)
    cdf = np.cumsum(mu, axis=0)
    cdf[-1, :] = 1.0
    for j in range(k):
        sel = np.nonzero(tok_topic == j)[0]
        if sel.size:
            words[sel] = np.searchsorted(cdf[:, j], g.random(sel.size), side="right")
    words = np.minimum(words, d - 1)
    X = _csr_from_pairs(tok_doc, words, n_docs, d)
    return {"X": X, "mu": mu, "alpha": alpha, "h": h, "lens": lens}


def mmsb_graph(seed: int, n_per: int, k: int, alpha_i: float, p: float, q: float,
               chunk: int = 1024) -> dict:
    """Bernoulli MMSB (Section 2.2), nodes split into four parts X, A, B, C.

    pi_u ~ Dir(alpha_i * 1_k); P = q 11^T + (p - q) I; G_ij ~ Ber(pi_i^T P pi_j).
    Returns CSR blocks G_XA, G_XB, G_XC (n_per x n_per each) and the ground
    truth memberships Pi[part] (n_per x k) and P.
    """
    g = rng(seed)
    alpha = np.full(k, float(alpha_i))
    Pi = {part: g.dirichlet(alpha, size=n_per) for part in ("X", "A", "B", "C")}
    P = np.full((k, k), float(q)) + (float(p) - float(q)) * np.eye(k)
    blocks = {}
    for part in ("A", "B", "C"):
        rows, cols = [], []
        right = Pi[part] @ P.T                                # n_per x k
        for r0 in range(0, n_per, chunk):
            r1 = min(n_per, r0 + chunk)
            prob = Pi["X"][r0:r1] @ right.T                   # rows x n_per
            hit = g.random(prob.shape) < prob
            rr, cc = np.nonzero(hit)
            rows.append(rr + r0)
            cols.append(cc)
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        blocks["G_X" + part] = _csr_from_pairs(rows, cols, n_per, n_per)
    return {**blocks, "Pi": Pi, "P": P, "alpha": alpha}


def orthogonal_samples(seed: int, k: int, n: int, sigma: float) -> dict:
    """Whitened samples of an orthogonal tensor plus Gaussian noise.

    w ~ Dir(1_k), U a Haar-random orthonormal k x k matrix, h_t ~ Cat(w),
    y_t = w_h^{-1/2} u_h + sigma * eps_t.  Returns Y (n x k, float32) and the
    ground truth (U: columns u_h, w).
    """
    g = rng(seed)
    w = g.dirichlet(np.ones(k))
    U = _haar(g, k)
    h = g.choice(k, size=n, p=w)
    Y = (U[:, h] / np.sqrt(w[h])).T + sigma * g.standard_normal((n, k))
    return {"Y": Y.astype(np.float32), "U": U, "w": w, "h": h}


def gaussian(seed: int, rows: int, cols: int, dtype=np.float32) -> np.ndarray:
    return rng(seed).standard_normal((rows, cols)).astype(dtype)


def _haar(g: np.random.Generator, k: int) -> np.ndarray:
    a = g.standard_normal((k, k))
    q, r = np.linalg.qr(a)
    return q * np.where(np.diag(r) < 0, -1.0, 1.0)


def haar_orthonormal(seed: int, k: int, dtype=np.float32) -> np.ndarray:
    """Haar-random orthonormal k x k matrix (random initial components)."""
    return _haar(rng(seed), k).astype(dtype)


def epoch_permutations(seed: int, n: int, epochs: int) -> np.ndarray:
    """epochs x n int32 array; row e is the sample order of epoch e."""
    g = rng(seed)
    return np.stack([g.permutation(n) for _ in range(epochs)]).astype(np.int32)
