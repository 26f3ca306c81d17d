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
  * :func:`whitened_lda_instances` / :func:`whitened_lda_samples` --
                                   decomposition instances of an exact-mixture
                                   LDA model drawn directly in whitened
                                   coordinates (training and evaluation data
                                   of the learned warm start).  The samples
                                   come from a counter-based generator
                                   (:func:`philox4x32`, Marsaglia-Tsang gamma
                                   draws) that the CUDA library implements
                                   from the same published definitions.

All generators use NumPy's PCG64 bit generator seeded with the given integer,
so both sides see bit-identical inputs.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "CSR", "lda_corpus", "mmsb_graph", "orthogonal_samples", "gaussian",
    "haar_orthonormal", "epoch_permutations", "csr_from_dense", "csr_to_dense",
    "philox4x32", "bits_to_unit", "whitened_lda_instances", "whitened_lda_samples",
    "unit_vectors", "signed_column_selection",
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


def orthogonal_samples(seed: int, k: int, n: int, sigma: float, conc: float = 1.0) -> dict:
    """Whitened samples of an orthogonal tensor plus Gaussian noise.

    w ~ Dir(conc 1_k), U a Haar-random orthonormal k x k matrix, h_t ~ Cat(w),
    y_t = w_h^{-1/2} u_h + sigma * eps_t.  Returns Y (n x k, float32) and the
    ground truth (U: columns u_h, w, the draws h).
    """
    g = rng(seed)
    w = g.dirichlet(np.full(k, float(conc)))
    U = _haar(g, k)
    h = g.choice(k, size=n, p=w)
    Y = (U[:, h] / np.sqrt(w[h])).T + sigma * g.standard_normal((n, k))
    return {"Y": Y.astype(np.float32), "U": U, "w": w, "h": h}


def gaussian(seed: int, rows: int, cols: int, dtype=np.float32) -> np.ndarray:
    return rng(seed).standard_normal((rows, cols)).astype(dtype)


def signed_column_selection(seed: int, rows: int, cols: int, dtype=np.float32) -> np.ndarray:
    """rows x cols matrix with one entry +-1 per column, in distinct rows chosen
    uniformly without replacement (the random projection for a sparse second
    moment, Section 4.2)."""
    g = rng(seed)
    idx = g.choice(rows, size=cols, replace=False)
    sign = np.where(g.random(cols) < 0.5, -1.0, 1.0)
    S = np.zeros((rows, cols), dtype=dtype)
    S[idx, np.arange(cols)] = sign
    return S


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


# ---------------------------------------------------------------------------
# Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
# "Parallel random numbers: as easy as 1, 2, 3", SC 2011).
# ---------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = 10):
    """Philox4x32 with `rounds` rounds on uint32 counters (arrays broadcast)
    and a 2 x 32-bit key.  Returns the four uint32 output words."""
    c = [np.asarray(x, dtype=np.uint32) for x in np.broadcast_arrays(c0, c1, c2, c3)]
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for r in range(rounds):
            if r > 0:
                k0 = np.uint32(k0 + _PHILOX_W0)
                k1 = np.uint32(k1 + _PHILOX_W1)
            p0 = _PHILOX_M0 * c[0].astype(np.uint64)
            p1 = _PHILOX_M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def bits_to_unit(x) -> np.ndarray:
    """uint32 -> float32 uniform strictly inside (0, 1): ((x >> 9) + 0.5) * 2^-23
    (every step exact in float32)."""
    return ((np.asarray(x, dtype=np.uint32) >> np.uint32(9)).astype(np.float32)
            + np.float32(0.5)) * np.float32(2.0 ** -23)


# Marsaglia-Tsang attempts per gamma draw; after that many rejections (a
# probability below 1e-20) the draw takes the mode-like value d.
GAMMA_ATTEMPTS = 16


def _log_gamma_draws(alpha: np.ndarray, t: np.ndarray, c: np.ndarray, inst: int, key):
    """log of Gamma(alpha_c) draws for samples t (vector) and components c,
    Marsaglia & Tsang, "A simple method for generating gamma variables"
    (ACM TOMS 2000), with the alpha < 1 boost G(a) = G(a + 1) U^(1/a).
    Counter (t, c, instance, attempt), key (seed lo, seed hi).  float32."""
    f = np.float32
    T, C = np.meshgrid(t.astype(np.uint32), c.astype(np.uint32), indexing="ij")
    a = alpha.astype(np.float32)[None, :] * np.ones_like(T, dtype=np.float32)
    small = a < f(1)
    ab = np.where(small, a + f(1), a).astype(np.float32)
    d = (ab - f(1.0 / 3.0)).astype(np.float32)
    cc = (f(1) / np.sqrt(f(9) * d)).astype(np.float32)
    logg = np.log(d).astype(np.float32)          # fallback value log(d)
    done = np.zeros(T.shape, dtype=bool)
    boost_u = None
    for att in range(GAMMA_ATTEMPTS):
        r = philox4x32(T, C, np.uint32(inst), np.uint32(att), key[0], key[1])
        if att == 0:
            boost_u = bits_to_unit(r[3])
        u1 = bits_to_unit(r[0])
        u2 = bits_to_unit(r[1])
        x = (np.sqrt(f(-2) * np.log(u1)) * np.cos(f(2 * np.pi) * u2)).astype(np.float32)
        v = (f(1) + cc * x).astype(np.float32)
        ok = v > f(0)
        v3 = (v * v * v).astype(np.float32)
        u = bits_to_unit(r[2])
        with np.errstate(invalid="ignore", divide="ignore"):
            lv3 = np.log(np.where(ok, v3, f(1))).astype(np.float32)
            acc = ok & (np.log(u) < f(0.5) * x * x + d - d * v3 + d * lv3)
        new = acc & ~done
        logg = np.where(new, (np.log(d) + lv3).astype(np.float32), logg)
        done |= acc
        if done.all():
            break
    logg = np.where(small, logg + np.log(boost_u) / a, logg).astype(np.float32)
    return logg


def unit_vectors(seed: int, count: int, k: int) -> np.ndarray:
    """count x k random unit vectors (float32), e.g. the sketch directions."""
    g = rng(seed).standard_normal((count, k))
    return (g / np.linalg.norm(g, axis=1, keepdims=True)).astype(np.float32)


def whitened_lda_instances(seed: int, nb: int, k: int, alpha0_range=(0.5, 2.0),
                           concentration: float = 4.0) -> dict:
    """Parameters of nb exact-mixture LDA instances in whitened coordinates.

    Per instance: alpha0 ~ U[alpha0_range], alpha = alpha0 * pi with
    pi ~ Dir(concentration * 1_k), U* Haar-random orthonormal, and the whitened
    topic vectors m_i = sqrt(alpha0 / alpha_i) u*_i (columns of m).  A sample
    is y = m h with h ~ Dir(alpha); the Dirichlet moment identities then give
    (alpha0 + 1) E[y y^T] - alpha0 ybar ybar^T = I and a whitened third moment
    sum_i lam_i u*_i^(x)3 with lam_i = sqrt(alpha0 / alpha_i).
    """
    g = rng(seed)
    a0 = g.uniform(alpha0_range[0], alpha0_range[1], size=nb)
    pi = g.dirichlet(np.full(k, concentration), size=nb)
    alpha = a0[:, None] * pi
    U = np.stack([_haar(g, k) for _ in range(nb)])
    lam = np.sqrt(a0[:, None] / alpha)
    m = U * lam[:, None, :]
    return {"alpha0": a0, "alpha": alpha, "U": U, "lam": lam,
            "m": m.astype(np.float32), "alpha32": alpha.astype(np.float32)}


def whitened_lda_samples(inst: dict, n: int, seed: int, first: int = 0,
                         count: int | None = None) -> np.ndarray:
    """Samples y_t = m h_t, h_t ~ Dir(alpha) of instances first .. first+count-1
    (count x n x k float32) from the counter-based generator: counter (t, c,
    instance, attempt), key (seed lo, seed hi); h = exp(L - max L) / sum exp(L
    - max L) with L the log-gamma draws; y accumulated in float32 in component
    order."""
    nb = inst["m"].shape[0] if count is None else count
    k = inst["m"].shape[1]
    key = (np.uint32(seed & 0xFFFFFFFF), np.uint32((seed >> 32) & 0xFFFFFFFF))
    out = np.empty((nb, n, k), dtype=np.float32)
    t = np.arange(n, dtype=np.uint32)
    c = np.arange(k, dtype=np.uint32)
    for j in range(nb):
        i = first + j
        L = _log_gamma_draws(inst["alpha32"][i], t, c, i, key)
        e = np.exp(L - L.max(axis=1, keepdims=True)).astype(np.float32)
        h = (e / e.sum(axis=1, keepdims=True, dtype=np.float32)).astype(np.float32)
        y = np.zeros((n, k), dtype=np.float32)
        for cc in range(k):
            y = (y + h[:, cc:cc + 1] * inst["m"][i][:, cc][None, :]).astype(np.float32)
        out[j] = y
    return out
