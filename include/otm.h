/*
 * otm.h -- C ABI of the GB300 (sm_103a) library for the online tensor method of
 * Huang, Niranjan, Hakeem and Anandkumar, "Online Tensor Methods for Learning
 * Latent Variable Models" (the paper).
 *
 * The library computes the paper's data-parallel hot path on one GPU:
 *   moments of sparse count data        (Section 2, Eqs. (1)-(2), (9)-(10))
 *   whitening W with W^T M2 W = I       (Section 3.1; randomised, Section 4.2)
 *   projection of samples y_t = W^T c_t (Section 3.1, Section 4.1)
 *   stochastic tensor gradient descent  (Section 3.2, Lemma 3 / Eq. (16))
 *   unwhitening / post-processing       (Section 3.3, Lemma 4)
 *   community membership and its p-value validation (Lemma 4, community case;
 *                                        Section "Validation methods")
 *
 * Conventions that hold for every entry point:
 *   - Every pointer argument is a DEVICE pointer owned by the caller, unless the
 *     argument's comment says "host".  The library never frees caller memory.
 *   - Dense matrices are row-major unless stated.  "rows x cols, row-major" means
 *     element (r, c) is at ptr[r * cols + c].  The k x k component matrix V is
 *     column-major: component v_i is the contiguous run V[i * k .. i * k + k).
 *   - Sparse count data use CSR with int32 row_ptr (rows + 1 entries, row_ptr[0]
 *     = 0, non-decreasing), int32 column indices in [0, cols) and float32 values.
 *   - Calls are asynchronous on the CUDA stream passed as `stream` (a
 *     cudaStream_t; NULL = legacy default stream).  Outputs are valid once the
 *     stream reaches the point of the call.  Calls that return a value to the
 *     host (documented) synchronise the stream.
 *   - Scratch memory: calls that need it take `ws` (device) and `ws_bytes`;
 *     the matching *_workspace() function returns the bytes required.  The
 *     library itself allocates no device memory.
 *   - Errors: each call returns an otm_status.  Argument errors are detected on
 *     the host before any launch (OTM_EINVAL) and leave outputs untouched.
 *     otm_last_error() returns a message for the calling thread's last error.
 *     There is no CPU fallback: without a usable GPU the calls fail with
 *     OTM_ECUDA.
 */
#ifndef OTM_H
#define OTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum otm_status {
  OTM_OK = 0,
  OTM_EINVAL = 1,          /* invalid argument (sizes, null pointers, workspace too small) */
  OTM_ENOTPSD = 2,         /* fewer than k positive eigenvalues: no whitening (Section 3.1) */
  OTM_ENOMEM = 3,          /* reserved (the library does not allocate) */
  OTM_ECUDA = 4,           /* a CUDA runtime call or kernel launch failed */
  OTM_ETIMEOUT = 5,        /* a bounded device-side wait expired */
  OTM_ENOTCONVERGED = 6    /* an iterative kernel hit its iteration limit */
} otm_status;

/* CSR sparse matrix (device arrays). */
typedef struct otm_csr {
  int64_t rows;
  int64_t cols;
  int64_t nnz;
  const int32_t* row_ptr;  /* rows + 1 */
  const int32_t* col;      /* nnz */
  const float* val;        /* nnz */
} otm_csr;

/* Library version (major * 10000 + minor * 100 + patch); no paper counterpart. */
int otm_version(void);

/* Message describing the calling thread's last error ("" if none). */
const char* otm_last_error(void);

/* Number of kernels this library has launched in this process so far (all
 * threads, all devices).  A diagnostic for profiling and launch accounting. */
uint64_t otm_launch_count(void);

/* ------------------------------------------------------------------------ */
/* Moments (Section 2.1 Eqs. (1)-(2); length normalisation as read for Lemma 1) */
/* ------------------------------------------------------------------------ */

/*
 * otm_topic_moments -- per-document statistics and first moments of a corpus.
 * X: n x d word counts (documents x vocabulary).
 * Outputs: row_invlen[n] = 1/l_t (0 if l_t = 0), row_w[n] = 1/(l_t (l_t - 1))
 * (0 if l_t < 2), M1[d] = (1/n) sum_t c_t / l_t (Eq. (1)), delta[d] =
 * (1/n) sum_t row_w[t] c_t (the diagonal term of Eq. (2)).  FP64 sums.
 */
otm_status otm_topic_moments(const otm_csr* X, float* row_invlen, float* row_w,
                             double* M1, double* delta, void* stream);

/*
 * otm_csr_transpose -- the CSR of X^T (d x n): colptr[d + 1], rowT[nnz] (the
 * document of each entry), valT[nnz], all caller-owned device arrays.  X must
 * have distinct columns within each row (a word counted once per document).
 * A counting sort by word over blocks of rows (per-block counts in shared
 * memory) where d fits, else one atomic position per entry; within a word the
 * documents come in no fixed order, colptr is exact.  Scratch:
 * otm_csr_transpose_workspace(n, d) bytes.  Used by the topic M2 products
 * (Eq. (2)): X^T P becomes a gather over the transpose.
 */
size_t otm_csr_transpose_workspace(int64_t n, int64_t d);
otm_status otm_csr_transpose(const otm_csr* X, int32_t* colptr, int32_t* rowT, float* valT,
                             void* ws, size_t ws_bytes, void* stream);

/*
 * otm_topic_m2_apply -- O = M2 S for Eq. (2) without forming M2:
 *   M2 S = (alpha0+1) [ (1/n) X^T diag(row_w) (X S) - diag(delta) S ]
 *          - alpha0 M1 (M1^T S).
 * S: d x m, O: d x m (float32, row-major; O must not alias S).  Xt: the
 * transpose of X from otm_csr_transpose, or NULL.  With Xt, X^T P is a gather
 * over it (m at most 384); without, a scatter with one atomic per nonzero and
 * column.
 * Scratch: otm_topic_m2_workspace(n, m) bytes.
 */
size_t otm_topic_m2_workspace(int64_t n, int64_t m);
otm_status otm_topic_m2_apply(const otm_csr* X, const otm_csr* Xt, const float* row_w,
                              const double* M1, const double* delta, double alpha0,
                              const float* S, int64_t m, float* O, void* ws, size_t ws_bytes,
                              void* stream);

/*
 * otm_pairs_apply -- O = Pairs(Y1, Y2) S = (1/n_X) G_{X,Y1}^T (G_{X,Y2} S)
 * (Section 2.2; the sparse core of Eqs. (7)-(8) and (10)).
 * G1: n_X x n_1, G2: n_X x n_2 (same n_X), S: n_2 x m, O: n_1 x m (float32).
 * Scratch: otm_pairs_workspace(n_X, m) bytes.
 */
size_t otm_pairs_workspace(int64_t n_x, int64_t m);
otm_status otm_pairs_apply(const otm_csr* G1, const otm_csr* G2, const float* S, int64_t m,
                           float* O, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Dense kernels of the whitening (Section 4.2: tall-thin QR, short-thin SVD) */
/* ------------------------------------------------------------------------ */

/*
 * otm_orthonormalize -- in-place tall-thin QR (Section 4.2 "Tall-thin QR"):
 * A (rows x m, float32, row-major, rows >= m, m <= 160) is replaced by an
 * orthonormal basis Q of a space containing its column space (exactly its
 * column space when A has full rank).  Cholesky-QR, two shifted passes then
 * two plain ones (Gram matrices accumulated in FP64); numerically
 * rank-deficient directions are completed with orthonormalised rounding
 * noise.  Scratch: otm_orth_workspace(m).  OTM_ENOTCONVERGED if the Gram
 * matrix is not finite.  Synchronises the stream.
 */
size_t otm_orth_workspace(int64_t m);
otm_status otm_orthonormalize(float* A, int64_t rows, int64_t m, void* ws, size_t ws_bytes,
                              void* stream);

/*
 * otm_syev -- FP64 symmetric eigendecomposition of a small matrix (the
 * "short-thin SVD" of Section 4.2, Table 3): A (n x n, FP64, row-major, n <= 160,
 * symmetrised as (A + A^T)/2) -> evals[n] descending, evecs (n x n, row-major,
 * column j = eigenvector j, sign fixed so its largest-magnitude entry is
 * positive).  A float32 start (Householder tridiagonalisation, multisection
 * bisection, eigenvectors from twisted factorisations) is refined in FP64
 * (Ogita-Aishima iteration, one cooperative launch over all SMs) until the
 * correction is below 1e-10 in every entry, at most 8 times: eigenvalues
 * separated from their neighbours by more than ~1e-5 ||A|| are FP64-accurate
 * (~1e-13 ||A||); closer groups get an FP64-exact invariant subspace and
 * eigenvalues to ~1e-9 ||A||.  Scratch: otm_syev_workspace(n).
 * OTM_ENOTCONVERGED on a non-finite eigenvalue, or if the refinement's grid
 * barrier timed out.  Synchronises the stream.
 */
size_t otm_syev_workspace(int64_t n);
otm_status otm_syev(const double* A, int64_t n, double* evals, double* evecs, void* ws,
                    size_t ws_bytes, void* stream);

/*
 * otm_syev_noalloc -- otm_syev without a caller workspace, for callers that
 * cannot allocate device memory (a host whose framework's memory pool owns the
 * GPU, an interface that passes only data pointers, or a loop that must not
 * call cudaMalloc / cudaFree because they synchronise the device).  The paper
 * has no counterpart: this is a packaging of the same eigendecomposition.
 * Arguments and results are those of otm_syev; n must be at most 160
 * (OTM_EINVAL with a message otherwise).
 * Scratch: a fixed 2 MiB array inside the library, present on every GPU on
 * which the library is loaded until the process exits.  The call allocates
 * nothing.  The first call on a device looks up the array's address on that
 * device (the current device; `stream` must belong to it).  All calls on one
 * device share the array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and give wrong results, so serialise them.
 * Every call copies a status flag to the host and synchronises the stream, so
 * no call can be captured in a CUDA graph: do not call it while its stream, or
 * any stream in global capture mode, is being captured.
 */
otm_status otm_syev_noalloc(const double* A, int64_t n, double* evals, double* evecs,
                            void* stream);

/* ------------------------------------------------------------------------ */
/* Whitening (Section 3.1, Section 4.2)                                     */
/* ------------------------------------------------------------------------ */

/*
 * otm_whiten_topic -- randomised whitening of the topic-model M2 (Eq. (2)):
 * range finder with the caller's random projection S (d x kt, kt = k + p,
 * k < kt <= 160, kt <= d), power_iters power iterations, tall-thin QR, FP64
 * eigendecomposition of Omega = Q^T M2 Q, truncation to the k largest.
 * Outputs: W (d x k, float32) with W^T M2 W = I; Q (d x kt, float32); Cw, Cp
 * (kt x k, FP64) with W = Q Cw and (W^T)^+ = Q Cp; eig[k] (descending); M1[d];
 * row_invlen[n], row_w[n] (as otm_topic_moments).  Returns OTM_ENOTPSD if the
 * k-th eigenvalue is not above 1e-5 times the largest (not positive, or not
 * resolvable at the float32 accuracy of the range finder).  Synchronises the
 * stream (the eigenvalue check).  Scratch: otm_whiten_topic_workspace(n, d,
 * nnz, k, kt); it holds, among the rest, the transpose of X (the CSR of X^T,
 * formed once per call, 8 nnz + 8 d bytes), through which X^T P and the
 * first moments are gathered.  The order of a word's documents in that
 * transpose comes from atomic positions, so FP32 sums over them (X^T P) vary
 * in the last bits from call to call; M1 and the other FP64 outputs of the
 * moments do not depend on it beyond FP64 rounding.
 */
size_t otm_whiten_topic_workspace(int64_t n, int64_t d, int64_t nnz, int64_t k, int64_t kt);
otm_status otm_whiten_topic(const otm_csr* X, const float* S, int64_t k, int64_t kt,
                            int power_iters, double alpha0, float* W, float* Q, double* Cw,
                            double* Cp, double* eig, double* M1, float* row_invlen,
                            float* row_w, void* ws, size_t ws_bytes, void* stream);

/*
 * otm_whiten_topic_nystrom -- the paper's own randomised whitening of the
 * topic-model M2 (Section 4.2, Algorithm 2 "Randomized Tall-thin SVD"): for a
 * random S (d x kt; the paper's choice for a sparse M2 is a column selection
 * with random signs, kt = 2k), O = M2 S, Omega = S^T O, and
 *   W = U_O L_O^{-1} V_O^T V_Omega L_Omega^{1/2}   (d x k),
 * with the SVD of O and the symmetric eigendecomposition of Omega both
 * truncated to rank k (the printed formula's trailing U_Omega^T is dropped so
 * that W has k columns; W^T M2 W = I_k exactly when M2 has rank k).  The SVD
 * of O comes from the FP64 eigendecomposition of O^T O.  k < kt <= 160, kt <= d.
 * Outputs, in the layout of otm_whiten_topic so that otm_project and
 * otm_unwhiten take them unchanged: W (d x k, float32); O (d x kt, float32,
 * in the Q slot: not orthonormal); Cw, Cp (kt x k, FP64) with W = O Cw and
 * (W^T)^+ = W (W^T W)^{-1} = O Cp; eig[k] = the k largest eigenvalues of
 * Omega (descending); M1, row_invlen, row_w as otm_topic_moments.
 * OTM_ENOTPSD if the k-th eigenvalue of Omega is not above 1e-5 times the
 * largest or O has rank < k.  Synchronises the stream.
 * Scratch: otm_whiten_topic_nystrom_workspace(n, d, k, kt).
 */
size_t otm_whiten_topic_nystrom_workspace(int64_t n, int64_t d, int64_t k, int64_t kt);
otm_status otm_whiten_topic_nystrom(const otm_csr* X, const float* S, int64_t k, int64_t kt,
                                    double alpha0, float* W, float* O, double* Cw, double* Cp,
                                    double* eig, double* M1, float* row_invlen, float* row_w,
                                    void* ws, size_t ws_bytes, void* stream);

/*
 * otm_whiten_community -- randomised whitening of the community-model M2
 * (Eq. (10), Sections 4.1-4.2).  G_XA, G_XB, G_XC: n_X x n_A, n_X x n_B,
 * n_X x n_C adjacency blocks.  S_pairs (n_B x kt) and S_w (n_A x kt) are the
 * random projections for the rank-k SVD of Pairs(C,B) and for the range
 * finder of M2.  Steps: Pairs(C,B) ~ U_C diag(sigma) V_B^T; Z_B = L_B V_B^T,
 * Z_C = L_C U_C^T (Eqs. (7)-(8) at rank k); the symmetric part of
 * (alpha0+1) Z_C Pairs(C,B) Z_B^T - alpha0 M1 M1^T applied in factored form;
 * range finder + QR + FP64 eig as in otm_whiten_topic.  OTM_ENOTPSD also when
 * sigma_k^2 <= 1e-5 sigma_1^2 (Pairs(C,B) numerically of rank < k).
 * Outputs: W (n_A x k), W_B = Z_B^T W (n_B x k), W_C = Z_C^T W (n_C x k)
 * (float32), Q (n_A x kt), Cw, Cp (kt x k FP64), eig[k], sigma[k] (singular
 * values of Pairs(C,B)), M1[n_A] (FP64).  OTM_ENOTPSD as above.  Synchronises
 * the stream.  Scratch: otm_whiten_community_workspace(n_X, n_A, n_B, n_C, k, kt).
 */
size_t otm_whiten_community_workspace(int64_t n_x, int64_t n_a, int64_t n_b, int64_t n_c,
                                      int64_t k, int64_t kt);
otm_status otm_whiten_community(const otm_csr* G_XA, const otm_csr* G_XB, const otm_csr* G_XC,
                                const float* S_pairs, const float* S_w, int64_t k, int64_t kt,
                                int power_iters, double alpha0, float* W, float* W_B,
                                float* W_C, float* Q, double* Cw, double* Cp, double* eig,
                                double* sigma, double* M1, void* ws, size_t ws_bytes,
                                void* stream);

/* ------------------------------------------------------------------------ */
/* Projection and means (Section 3.1 "whitened data", Section 4.1)          */
/* ------------------------------------------------------------------------ */

/*
 * otm_project -- Y = diag(row_scale) X W: y_t = W^T c_t (times row_scale[t]).
 * X: n x d CSR, W: d x k (float32), row_scale: n floats or NULL (= 1),
 * Y: n x k (float32).  For topics row_scale = row_invlen (y_t = W^T c_t / l_t).
 */
otm_status otm_project(const otm_csr* X, const float* W, int64_t k, const float* row_scale,
                       float* Y, void* stream);

/*
 * otm_column_mean -- ybar = (1/n) sum_t Y[t, :] (the means y-bar of Section
 * 3.2), to FP64-class accuracy: compensated float32 sums over blocks of 512
 * rows (the rounding error of every addition kept), added in FP64.  Y: n x k
 * float32; ybar: k doubles.
 */
otm_status otm_column_mean(const float* Y, int64_t n, int64_t k, double* ybar, void* stream);

/* ------------------------------------------------------------------------ */
/* Stochastic tensor gradient descent (Section 3.2, Lemma 3, Appendix A)     */
/* ------------------------------------------------------------------------ */

/*
 * otm_sgd_step -- one STGD update over a minibatch (Lemma 3, Eq. (16)):
 *   G = kappa V ((V^T V) o (V^T V)) - T_b(V, V, I),   V <- V - beta G,
 * kappa = (1 + theta)/2, where column i of T_b(V, V, I) is the minibatch mean of
 * the implicit tensor contraction
 *   c1 <v_i,yA><v_i,yB> yC - c2 [<v_i,yA><v_i,yB> ybC + <v_i,yA><v_i,ybB> yC
 *   + <v_i,ybA><v_i,yB> yC] + c3 <v_i,ybA><v_i,ybB> ybC,
 * c1 = (a0+1)(a0+2)/2, c2 = a0(a0+1)/2, c3 = a0^2.  The tensor is never formed.
 * V: k x k column-major float32, updated in place.  YA, YB, YC: b x k float32
 * (may alias each other; equal pointers select the symmetric fast path).
 * ybar3: 3 x k doubles (ybA, ybB, ybC).  1 <= k <= 128, b >= 1.
 * ws: otm_sgd_workspace(k, b) bytes of scratch for the grid form of the
 * kernel (see otm_sgd_set_form), or NULL / too small, in which case the
 * cluster form runs (forcing the grid form then returns OTM_EINVAL).
 */
size_t otm_sgd_workspace(int64_t k, int64_t b);
otm_status otm_sgd_step(float* V, const float* YA, const float* YB, const float* YC,
                        int64_t b, int64_t k, const double* ybar3, double theta, double beta,
                        double alpha0, void* ws, size_t ws_bytes, void* stream);

/*
 * otm_sgd_run -- the whole STGD loop in ONE persistent launch (V stays
 * on-chip between steps, Section 4.3 "device interface").  For epoch e the
 * samples are visited in the order perm[e * n .. e * n + n) in minibatches of b
 * (the last one partial), step t = 1, 2, ... uses beta_t = beta0 / sqrt(t).
 * YA, YB, YC: n x k (may alias); perm: epochs x n int32 (NULL = identity order
 * every epoch).  If snapshot_every > 0, V after every snapshot_every-th step
 * is written to V_snap[(t / snapshot_every - 1) * k * k ...] (caller sizes it
 * for floor(total_steps / snapshot_every) matrices).  ws / ws_bytes: as for
 * otm_sgd_step (otm_sgd_workspace(k, b) bytes).
 */
otm_status otm_sgd_run(float* V, const float* YA, const float* YB, const float* YC, int64_t n,
                       int64_t k, const double* ybar3, const int32_t* perm, int64_t epochs,
                       int64_t b, double beta0, double theta, double alpha0,
                       int64_t snapshot_every, float* V_snap, void* ws, size_t ws_bytes,
                       void* stream);

/*
 * otm_sgd_set_form -- which FP32 kernel otm_sgd_step / otm_sgd_run use, for
 * the whole process (no paper counterpart; a performance choice with the same
 * results up to FP32 summation order):
 *   0 (default)  chosen by size: with a caller workspace, the grid form for
 *                k <= 128 and 256 <= b <= 32 x (SM count), the split form for
 *                larger minibatches where it applies; the cluster form otherwise;
 *   1            the cluster form: one thread-block cluster of up to 16 CTAs
 *                keeps V in shared memory, the minibatch split over its CTAs,
 *                partial products reduced through distributed shared memory;
 *   2            the grid form: one cooperative launch of up to one CTA per SM,
 *                the minibatch split over all of them, partial products
 *                reduced through L2 by the owners of the columns, two grid
 *                barriers per step (k <= 128, 16 <= b <= 32 x SMs and a
 *                workspace of otm_sgd_workspace(k, b) bytes, else OTM_EINVAL
 *                from the run).  On a barrier time-out the affected columns
 *                of V are NaN;
 *   3            the split form: one launch of C thread-block clusters; the
 *                components are cut into C blocks (one per cluster) and every
 *                minibatch into slices (one per CTA of a cluster); each CTA
 *                forms its slice's products for its cluster's block, the
 *                partial columns are summed by their owners through
 *                distributed shared memory, and one grid barrier per step
 *                publishes the new V (k <= 128, all clusters resident at once,
 *                a workspace of otm_sgd_workspace(k, b) bytes, else OTM_EINVAL
 *                from the run).  On a barrier time-out the owners' columns of
 *                V are NaN.
 * OTM_EINVAL for another value.
 */
otm_status otm_sgd_set_form(int form);

/*
 * otm_sgd_split_shape -- the launch shape the split form (form 3) takes for
 * k components, minibatch b and symmetric (sym != 0) or three distinct views:
 * *clusters thread-block clusters of *cluster_size CTAs, or 0 and 0 where the
 * split form does not apply on the current device.  No paper counterpart (a
 * diagnostic of the performance choice above).  OTM_EINVAL on a null pointer.
 */
otm_status otm_sgd_split_shape(int64_t k, int64_t b, int sym, int* clusters, int* cluster_size);

/*
 * otm_sgd_run_topic_exact -- STGD for the topic model on the whole third
 * moment of Section 2.1, Eq. (3) (its self-token terms kept), whitened by W,
 * instead of the sample tensor of Section 3.2; the implicit form of Lemma 3:
 *   G = kappa V ((V^T V) o (V^T V)) - T(V, V, I),   V <- V - beta_t G,
 * where column i of T(V, V, I) is the minibatch mean over documents t of
 *   c1 [s^2 y' - q y' - 2 s r + 2 z] / (l (l-1) (l-2))
 *   - c2 ([s^2 - q] m + 2 mu [s y' - r]) / (l (l-1))
 * plus c3 mu^2 m, with y' = W^T c_t, u = W v_i, s = <c_t, u>, q = sum_j c_j u_j^2,
 * r = W^T (c_t o u), z = W^T (c_t o u o u), m = W^T M1, mu = <m, v_i>, l the
 * document's length (a term is dropped for documents shorter than its
 * order).  The tensor is never formed: per minibatch the rows of W of its word
 * occurrences are gathered, U = W_g V^T, the per-document sums and
 * coefficients are formed, and the data term is W_g^T Coef + Y'^T A.
 * precision 0: the products in FP32 tiles with FP64 accumulation; precision 1
 * (OTM_PREC_BF16): U = W_g V^T and W_g^T Coef on the tensor cores (tcgen05,
 * BF16 operands, FP32 accumulation; W_g^T Coef as slices of 1,536 occurrences
 * whose partials are added in FP64), the per-document sums and coefficients
 * as in FP32; about 3e-3 relative error in the gradient.
 * X: the corpus (n documents x d words, CSR counts); W: d x k float32
 * row-major; M1: d doubles (the first moment of Eq. (1)); V: k x k float32,
 * component i contiguous, updated in place; perm: epochs x n int32 (NULL =
 * identity order); minibatches of b documents, beta_t = beta0 / sqrt(t).
 * nnz_b_max: the most word occurrences (CSR entries) any minibatch holds; a
 * larger minibatch is not processed and makes the call return OTM_EINVAL.
 * Snapshots as for otm_sgd_run.  1 <= k <= 128.
 * Scratch: otm_sgd_topic_exact_workspace(k, b, nnz_b_max, precision) bytes (0
 * for arguments out of range).  The host drives the steps (about ten launches
 * each); synchronises the stream at the end.  OTM_ETIMEOUT if a tensor-core
 * product's bounded wait expired.
 */
size_t otm_sgd_topic_exact_workspace(int64_t k, int64_t b, int64_t nnz_b_max, int precision);
otm_status otm_sgd_run_topic_exact(float* V, const otm_csr* X, const float* W, const double* M1,
                                   int64_t k, const int32_t* perm, int64_t epochs, int64_t b,
                                   int64_t nnz_b_max, double beta0, double theta, double alpha0,
                                   int precision, float* V_snap, int64_t snapshot_every, void* ws,
                                   size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Precision form of the STGD (not in the paper: BF16 / FP8 tensor cores)     */
/* ------------------------------------------------------------------------ */

#define OTM_PREC_BF16 1
#define OTM_PREC_FP8 2 /* e4m3 */
#define OTM_PREC_FP8X2 3 /* e4m3, samples and B as two terms (otm_sgd_run_lp only) */

/*
 * otm_quantize_samples -- store whitened samples for the low-precision STGD.
 * Y: n x k float32 (row-major), 1 <= k <= 256.  Yq: n x ldq elements with
 * ldq = k rounded up to a multiple of 16, zero padded; BF16 (2 bytes each) or
 * FP8 e4m3 (1 byte each) per `precision`.  FP8 rows are scaled by one factor
 * per sample, scales[t] = max_r |Y[t][r]| / 448 (1 for an all-zero row), so
 * Y[t] ~ scales[t] * Yq[t]; BF16 writes scales[t] = 1 when scales != NULL.
 * OTM_PREC_FP8X2: Yq holds 2 n rows, the e4m3 rows above and then the e4m3
 * rounding of their residuals at the same scales, Y[t] ~ scales[t] (Yq[t] +
 * Yq[n + t]).
 */
otm_status otm_quantize_samples(const float* Y, int64_t n, int64_t k, int precision, void* Yq,
                                float* scales, void* stream);

/*
 * otm_sgd_run_lp -- otm_sgd_run (the Lemma 3 update, same schedule and
 * arguments) with the two sample products on the tensor cores: A = Y V in
 * BF16 or FP8 from samples stored by otm_quantize_samples (YA, YB, YC with
 * their per-sample scales sA, sB, sC, NULL = 1; equal pointers select the
 * symmetric path), V re-quantised every step with one scale per component,
 * B = c1 A_A o A_B - c2 (...) quantised with one scale per component per 128
 * samples, FP32 accumulation in tensor memory; the Gram term V((V^T V) o 2)
 * runs as BF16 tensor-core products of the BF16 image of V, and so do
 * a_A = V^T ybar_A, a_B = V^T ybar_B for k <= 128 (k > 128: FP32 sums of the
 * BF16 rows on the CUDA cores); the master V, the mean terms and the update
 * stay FP32.  ybar3 are the FP64 means of the unquantised samples.
 * OTM_PREC_FP8X2 (samples stored as two e4m3 terms; B split the same way at
 * its per-tile scales): the first product takes Y_hi V_hi + Y_hi V_lo +
 * Y_lo V_hi and the second Y_hi^T B_hi + Y_lo^T B_hi + Y_hi^T B_lo, which
 * brings long whitened samples (those of a 300-word LDA corpus) within 2e-2.
 * 1 <= k <= 256; for k > 128 every CTA of the cluster keeps only its own rows
 * of the BF16 image on chip and the whole image is exchanged through two
 * buffers in the workspace (three distinct views: 16-CTA clusters).
 * Scratch: otm_sgd_run_lp_workspace() bytes.  Synchronises the stream;
 * returns OTM_ETIMEOUT if a bounded wait on the tensor cores expired.
 */
size_t otm_sgd_run_lp_workspace(void);
otm_status otm_sgd_run_lp(float* V, const void* YA, const void* YB, const void* YC,
                          const float* sA, const float* sB, const float* sC, int64_t n, int64_t k,
                          const double* ybar3, const int32_t* perm, int64_t epochs, int64_t b,
                          double beta0, double theta, double alpha0, int precision,
                          int64_t snapshot_every, float* V_snap, void* ws, size_t ws_bytes,
                          void* stream);

/* ------------------------------------------------------------------------ */
/* Batched form: many independent decompositions in one persistent launch   */
/* (not in the paper)                                                        */
/* ------------------------------------------------------------------------ */

/* One decomposition problem (symmetric views); all pointers are device
 * pointers.  Its `restarts` independent chains start from V[r * k * k ...]
 * (restart r, k x k, component-contiguous) and are updated in place.
 * k <= 256. */
typedef struct otm_problem {
  int64_t n, k, b, epochs;   /* samples, components (1..256), minibatch, epochs */
  const void* Yq;            /* n x ldq samples from otm_quantize_samples */
  const float* scales;       /* per-sample scales or NULL */
  const int32_t* perm;       /* epochs x n sample orders or NULL */
  const double* ybar3;       /* 3 x k means (the same mean three times) */
  float* V;                  /* restarts x k x k, in/out */
  int64_t restarts;
  double beta0, theta, alpha0;
} otm_problem;

/* A prepared batch: filled by otm_sgd_batched_prepare, read by the launch. */
typedef struct otm_batch_plan {
  int32_t nitems;         /* work items: restarts, with those of a problem with k <= 64
                             stacked floor(128 / k) to an item */
  int32_t cluster;        /* CTAs per chain (k <= 128), chosen by the autotuner or given */
  int32_t precision;
  int32_t max_k;          /* most components of an item with k <= 128 (stacked: R k) */
  int32_t grid_clusters;  /* clusters in the persistent grid (k <= 128) */
  int32_t nitems_wide;    /* chains with 128 < k <= 256 (second launch) */
  int32_t grid_clusters_wide;
  int32_t max_k_wide;
  int32_t cluster_wide;   /* CTAs per chain with k > 128: 4, 8 or 16, by the same trial */
  int32_t stages;         /* sample stages (1-4) of the k <= 128 group's schedule */
  int32_t vimg2;          /* its V image double-buffered (1) or single (0) */
  int32_t stages_wide;    /* the same for the k > 128 group */
  int32_t vimg2_wide;
  int64_t smem_bytes;
  void* ws;
  size_t ws_bytes;
} otm_batch_plan;

/*
 * otm_sgd_batched_prepare -- expands the problems into work items, orders them
 * by cost (steps x (b c k + c^2 k) for c components, longest first) and
 * uploads the work list to the workspace (otm_sgd_batched_workspace(chains)
 * bytes, chains = the sum of restarts, kept alive until the last launch).  An
 * item is one restart, or for k <= 64 up to floor(128 / k) restarts of one
 * problem run together as one chain of R k components: every sample tile is
 * loaded and multiplied once for all of them, each keeps its own Gram term
 * (H = V^T V is masked to the restart's block), and the results equal R
 * separate runs up to FP32 summation order.  cluster = 0 runs the autotuner
 * for each group (k <= 128, 128 < k <= 256): a short trial launch (at most 4
 * steps per chain, on scratch V) for every schedule that fits the group's
 * largest k -- the cluster size (CTAs per chain, i.e. the width of a CTA's tile
 * of components), the number of sample stages (1 to 4) and a single or double
 * V image; the fastest is kept (cached per group, precision, largest k and
 * chain count) and recorded in the plan.  A given cluster size (k <= 128 group)
 * takes its first fitting schedule.  Synchronises the stream.  Each chain runs
 * the Lemma 3 schedule of otm_sgd_run_lp.
 *
 * otm_sgd_batched_launch -- one persistent launch running every chain with
 * k <= 128 (and, if the plan has any, a second one for 128 < k <= 256, whose
 * chains use 4- to 16-CTA clusters, chosen by the same trial, keep their FP32
 * master rows in tensor memory and exchange the BF16 image of V through two
 * buffers per cluster in the workspace): as many clusters as fit on the GPU take chains
 * from the work list until it is empty.  Asynchronous and free of host synchronisation, so it can
 * be captured in a CUDA graph.  otm_sgd_batched_check reads the plan's
 * timeout flag (synchronises; OTM_ETIMEOUT if a tensor-core wait expired).
 */
size_t otm_sgd_batched_workspace(int64_t nitems);
otm_status otm_sgd_batched_prepare(const otm_problem* probs, int nprob, int precision,
                                   int cluster, void* ws, size_t ws_bytes, otm_batch_plan* plan,
                                   void* stream);
otm_status otm_sgd_batched_launch(const otm_batch_plan* plan, void* stream);
otm_status otm_sgd_batched_check(const otm_batch_plan* plan, void* stream);

/* ------------------------------------------------------------------------ */
/* Learned warm start (not in the paper)                                     */
/* ------------------------------------------------------------------------ */
/*
 * A small MLP maps J <= 4 sketches of the whitened tensor of Section 3.2,
 * S_j = T(I, I, theta_j) (k x k each, k <= 64), to an initial component
 * matrix.  The network is x -> GELU(W1 x + b1) -> GELU(W2 h1 + b2) -> W3 h2 + b3
 * (exact GELU z Phi(z)), x = vec(S_1..S_J) scaled to unit root-mean-square;
 * its output (k^2) is read row-major as a k x k matrix M whose columns are
 * orthonormalised by Gram-Schmidt (U0 = GS(M)); v_i = sign(t_i) (|t_i| /
 * kappa)^(1/3) u_i with t_i = T(u_i, u_i, u_i) (the stationary scaling of
 * Lemma 3).  Training minimises the batch mean of
 *   L(U) = - sum_i T*(u_i, u_i, u_i)^2 / sum_j lam_j^2,
 * T* = sum_j lam_j u*_j^(x)3 the instance's known decomposition, with Adam
 * (Kingma & Ba 2015).  Weights are FP32 masters with BF16 copies; the dense
 * products run on tcgen05 tensor cores with FP32 accumulation.
 * Matrices of one instance are k x k row-major (U[a * k + i] = entry a of
 * column u_i) unless stated; batches are contiguous.
 */

/* Network descriptor; every buffer is caller-owned device memory.
 * d_in, width, d_out: multiples of 8 (d_in = J k^2, d_out = k^2).
 * Parameter order (otm_mlp_param_count elements): W1 (width x d_in, row-major),
 * b1 (width), W2 (width x width), b2, W3 (d_out x width), b3 (d_out). */
typedef struct otm_mlp {
  int64_t d_in, width, d_out;
  float* p;        /* FP32 master parameters */
  void* p16;       /* BF16 copy of p (same order) */
  void* w2t16;     /* BF16 W2^T (width x width) */
  void* w3t16;     /* BF16 W3^T (width x d_out) */
  float* grad;     /* FP32 gradient (same order as p), written by the backward pass */
  float* adam_m;   /* Adam first and second moments (same order; zero before step 1) */
  float* adam_v;
} otm_mlp;

int64_t otm_mlp_param_count(int64_t d_in, int64_t width, int64_t d_out);

/* Refresh p16, w2t16 and w3t16 from p (after the caller writes p). */
otm_status otm_mlp_sync_weights(const otm_mlp* net, void* stream);

/*
 * otm_mlp_forward -- out (batch x d_out, FP32) for BF16 inputs x16 (batch x
 * d_in); batch a multiple of 8.  Leaves the activations in ws for
 * otm_mlp_backward.  otm_mlp_backward -- net->grad from dL/d(out) (batch x
 * d_out, FP32) and the cache of the preceding forward call on the same ws.
 * Scratch: otm_mlp_workspace(net, batch) bytes.
 */
size_t otm_mlp_workspace(const otm_mlp* net, int64_t batch);
otm_status otm_mlp_forward(const otm_mlp* net, const void* x16, int64_t batch, float* out,
                           void* ws, size_t ws_bytes, void* stream);
otm_status otm_mlp_backward(const otm_mlp* net, const void* x16, int64_t batch, const float* dout,
                            void* ws, size_t ws_bytes, void* stream);

/* One Adam update of p from grad (step t >= 1), then the BF16 copies. */
otm_status otm_adam_step(const otm_mlp* net, double lr, double b1, double b2, double eps, int64_t t,
                         void* stream);

/*
 * otm_gram_schmidt -- M (nb x k x k) = U R column by column (classical
 * Gram-Schmidt applied twice per column, FP32); R upper triangular with
 * positive diagonal.  otm_gram_schmidt_backward -- dL/dM = (dU + U
 * copyltu(-dU^T U)) R^{-T}, copyltu(A) = tril(A) + tril(A, -1)^T.
 * otm_ws_loss_grad -- loss[b] = L(U_b) and dU = scale * dL/dU
 * (column i = -6 T*(u_i,u_i,u_i) T*(u_i,u_i,I) / sum lam^2); Ustar nb x k x k
 * (columns u*_j), lam nb x k.  k <= 64.
 */
otm_status otm_gram_schmidt(const float* M, int64_t nb, int64_t k, float* U, float* R,
                            void* stream);
otm_status otm_gram_schmidt_backward(const float* U, const float* R, const float* dU, int64_t nb,
                                     int64_t k, float* dM, void* stream);
otm_status otm_ws_loss_grad(const float* U, const float* Ustar, const float* lam, int64_t nb,
                            int64_t k, double scale, float* loss, float* dU, void* stream);

/*
 * otm_ws_train_step -- forward, Gram-Schmidt, loss (loss[b] per instance,
 * FP32), backward through Gram-Schmidt and the MLP (dL/dout scaled by
 * 1/batch: the gradient of the batch mean), then Adam step t with learning
 * rate lr (b1 = 0.9, b2 = 0.999, eps = 1e-8).  otm_ws_infer -- U0 (batch x k x k)
 * = GS(MLP(x16)).  Scratch of both: otm_ws_train_workspace(net, batch).
 * Asynchronous; otm_ws_check(ws) reports a timed-out tensor-core wait.
 */
size_t otm_ws_train_workspace(const otm_mlp* net, int64_t batch);
otm_status otm_ws_train_step(const otm_mlp* net, const void* x16, const float* Ustar,
                             const float* lam, int64_t batch, int64_t k, double lr, int64_t t,
                             float* loss, void* ws, size_t ws_bytes, void* stream);
otm_status otm_ws_infer(const otm_mlp* net, const void* x16, int64_t batch, int64_t k, float* U0,
                        void* ws, size_t ws_bytes, void* stream);
otm_status otm_ws_check(const void* ws, void* stream);

/*
 * otm_ws_sketch -- J sketches S_j = T(I, I, theta_j) of the symmetric whitened
 * tensor of Section 3.2 per instance, from samples Y (nb x n x k) with the
 * instance's alpha0 (nb, host-order device array):
 *   S = c1 P - c2 <theta,ybar> Q - c2 (m ybar^T + ybar m^T) + c3 <theta,ybar> ybar ybar^T,
 *   Q = Y^T Y / n, P = Y^T diag(Y theta) Y / n, m = Q theta.
 * Q and P_j are BF16 tensor-core products with FP32 accumulation.
 * thetas: J x k; S (optional): nb x J x k x k FP32; x16: nb x J k^2 BF16
 * network inputs (unit root-mean-square).  Scratch: otm_ws_sketch_workspace.
 */
size_t otm_ws_sketch_workspace(int64_t nb, int64_t n, int64_t k, int J);
otm_status otm_ws_sketch(const float* Y, int64_t nb, int64_t n, int64_t k, const double* alpha0,
                         const float* thetas, int J, float* S, void* x16, void* ws,
                         size_t ws_bytes, void* stream);

/*
 * otm_ws_canonicalize -- the canonical frame of each instance: E (nb x k x k,
 * columns) = eigenvectors of the symmetric part of S_1 (cyclic Jacobi, FP32),
 * ordered by descending eigenvalue (evals, nb x k, optional) with each
 * vector's largest-magnitude entry positive; x16 (nb x J k^2, BF16) =
 * vec(E^T S_j E) scaled to unit root-mean-square.  S: nb x J x k x k.
 * otm_ws_rotate -- out = E U (transpose = 0) or E^T U (transpose = 1) per
 * instance (out must not alias U).  k <= 64.
 */
otm_status otm_ws_canonicalize(const float* S, int64_t nb, int64_t k, int J, float* E,
                               float* evals, void* x16, void* stream);
otm_status otm_ws_rotate(const float* E, const float* U, int64_t nb, int64_t k, int transpose,
                         float* out, void* stream);

/*
 * otm_ws_init_components -- V0 (nb x k x k, component i contiguous, the STGD
 * layout) from orthonormal directions U0 (nb x k x k, columns) and samples Y:
 * v_i = sign(t_i) (|t_i| / kappa)^(1/3) u_i, kappa = (1 + theta) / 2,
 * t_i = c1 E[(y.u_i)^3] - 3 c2 E[(y.u_i)^2] (ybar.u_i) + c3 (ybar.u_i)^3.
 * Scratch: otm_ws_init_workspace(nb, n, k).
 */
size_t otm_ws_init_workspace(int64_t nb, int64_t n, int64_t k);
otm_status otm_ws_init_components(const float* U0, const float* Y, int64_t nb, int64_t n,
                                  int64_t k, const double* alpha0, double theta, float* V0,
                                  void* ws, size_t ws_bytes, void* stream);

/*
 * otm_ws_generate -- samples of exact-mixture LDA instances in whitened
 * coordinates (training and evaluation data): y_t = m h_t, h_t ~ Dir(alpha)
 * for instances first .. first + nb - 1.  m: nb x k x k (row-major, column i
 * the whitened topic vector sqrt(alpha0/alpha_i) u*_i), alpha: nb x k, Y: nb x
 * n x k.  Gamma draws by Marsaglia & Tsang (ACM TOMS 2000) on Philox4x32-10
 * counters (t, c, instance, attempt) with key seed (Salmon et al., SC 2011);
 * h = exp(L - max L) / sum exp(L - max L) from the log-gamma draws L.
 */
otm_status otm_ws_generate(const float* m, const float* alpha, int64_t nb, int64_t n, int64_t k,
                           uint64_t seed, int64_t first, float* Y, void* stream);

/*
 * otm_gemm_bf16 -- C[z] = alpha A[z] B[z]^T for z < batch on the tensor cores
 * (tcgen05, TMA-fed, FP32 accumulation).  A: M x K, B: N x K, BF16 row-major
 * with leading dimensions lda, ldb and batch strides (elements); K, lda, ldb
 * and the strides multiples of 8, A and B 16-byte aligned.  epilogue 0: C
 * (FP32, ldc, strideC; optional) and H (BF16, ldh, strideH; optional) =
 * result; 1: result + bias[col]; 2: C = result + bias, H = GELU(C).  Scratch:
 * otm_gemm_bf16_workspace() bytes (its first int is set if a wait timed out).
 */
size_t otm_gemm_bf16_workspace(void);
otm_status otm_gemm_bf16(const void* A, const void* B, int64_t M, int64_t N, int64_t K,
                         int64_t batch, int64_t lda, int64_t ldb, int64_t strideA, int64_t strideB,
                         int epilogue, float alpha, const float* bias, float* C, int64_t ldc,
                         int64_t strideC, void* H, int64_t ldh, int64_t strideH, void* ws,
                         size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Post-processing (Section 3.3, Lemma 4) and error evaluation               */
/* ------------------------------------------------------------------------ */

/*
 * otm_unwhiten -- lambda_i = kappa ||v_i||^3; u_i = v_i / ||v_i||;
 * comps[:, i] = lambda_i (W^T)^+ u_i with (W^T)^+ = Q Cp (Lemma 4).  With
 * normalize != 0 each column is sign-flipped to a non-negative sum and divided
 * by its sum (topic-word distributions).  alpha_hat_i = lambda_i^-2 / sum_j
 * lambda_j^-2.  V: k x k column-major float32; Q: d x kt float32; Cp: kt x k
 * FP64; comps: d x k FP64 row-major; lambda, alpha_hat: k doubles.  The k x k
 * factors, the normalisation and alpha_hat are FP64; the d x kt by kt x k
 * product runs in double-float arithmetic on the FP32 units (every entry
 * within about 2^-48 of the sum of its absolute terms).
 * Scratch: otm_unwhiten_workspace(d, k, kt).
 */
size_t otm_unwhiten_workspace(int64_t d, int64_t k, int64_t kt);
otm_status otm_unwhiten(const float* V, int64_t k, const float* Q, int64_t d, int64_t kt,
                        const double* Cp, double theta, int normalize, double* comps,
                        double* lambda, double* alpha_hat, void* ws, size_t ws_bytes,
                        void* stream);

/*
 * otm_recon_error -- (not in the paper: the convergence measure of the
 * benchmark) relative reconstruction error of the components in V
 * against reference components (lam_true[k], U_true: k x k column-major FP64,
 * unit columns):
 *   err = || kappa sum_i v_i^(x)3 - sum_j lam_j u_j^(x)3 ||_F / || sum_j lam_j u_j^(x)3 ||_F,
 * evaluated in closed form from Gram matrices (<x^(x)3, y^(x)3> = <x,y>^3), FP64.
 * Writes one double to err (device): NaN if V holds a non-finite value (a
 * diverged run), never a clamped zero.  Scratch: otm_recon_error_workspace(k).
 */
size_t otm_recon_error_workspace(int64_t k);
otm_status otm_recon_error(const float* V, int64_t k, double theta, const double* U_true,
                           const double* lam_true, double* err, void* ws, size_t ws_bytes,
                           void* stream);

/*
 * otm_membership -- community membership estimate (Section 3.3 Lemma 4,
 * community case): Pi_hat = diag(gamma)^{1/3} diag(Lambda)^{-1} Phi^T W^T G_{A,X}
 * for the n nodes X whose whitened view-A rows y_x = W^T G_{A,x} are the rows
 * of Y.  Phi holds the unit components u_i = v_i / ||v_i||, Lambda the
 * eigenvalues lambda_i = kappa ||v_i||^3 (kappa = (1 + theta) / 2), and gamma
 * the scalar of the Dirichlet normalisation, gamma = (sum_i lambda_i^-2)^{-1/2}.
 * With population moments and exact components the result is the true
 * membership.  Entries below tau are set to 0 (thresholding; pass -INFINITY
 * to keep all).
 *   Y: n x k float32 row-major (the view-A samples, as otm_project writes them);
 *   V: k x k float32 column-major (the STGD components);
 *   Pi_hat: k x n float32 row-major, row i = community i over the nodes.
 * FP32 dot products, FP64 scale.  1 <= k <= 1024; n = 0 is a no-op.
 * Scratch: otm_membership_workspace(k).  OTM_EINVAL on bad sizes or pointers.
 */
size_t otm_membership_workspace(int64_t k);
otm_status otm_membership(const float* Y, int64_t n, int64_t k, const float* V, double theta,
                          double tau, float* Pi_hat, void* ws, size_t ws_bytes, void* stream);

/*
 * otm_pvalue_match -- validation of an estimated membership against the
 * ground truth by p-value testing (Section "Validation methods": p-value
 * testing, recovery ratio, error function).  For each estimated row i
 * (k_hat rows) and ground-truth row j (k rows) over n nodes:
 *   rho(i,j) = Pearson correlation (0 when either row is constant),
 *   T = rho sqrt(n-2) / sqrt(1 - rho^2),  pvals[i*k + j] = P(t_{n-2} > T),
 *   l1[i*k + j] = (1/n) sum_x |Pi_hat[i,x] - Pi[j,x]|.
 * A pair is significant when its p-value is <= threshold (the paper uses
 * 0.01).  scores[0] = recovery ratio R = fraction of ground-truth rows with at
 * least one significant pair; scores[1] = average error E = (1/k) * sum of
 * l1 over the significant pairs.
 *   Pi_hat: k_hat x n, Pi: k x n, float32 row-major; pvals, l1: k_hat x k FP64
 *   row-major; scores: 2 doubles (device).  All statistics in FP64; the
 *   t tail from the continued fraction of the regularised incomplete beta.
 * Needs n >= 3, 1 <= k <= 1024.  Scratch: otm_pvalue_match_workspace(k_hat, k).
 */
size_t otm_pvalue_match_workspace(int64_t k_hat, int64_t k);
otm_status otm_pvalue_match(const float* Pi_hat, int64_t k_hat, const float* Pi, int64_t k,
                            int64_t n, double threshold, double* pvals, double* l1,
                            double* scores, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OTM_H */
