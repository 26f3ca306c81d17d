// Whitening (Section 3.1) by the randomised low-rank method of Section 4.2.
//
// Topic model: M2 of Eq. (2) is applied implicitly, M2 S = (a0+1)[(1/n) X^T
// diag(w) (X S) - diag(delta) S] - a0 M1 (M1^T S), i.e. one gather SpMM over
// the counts, one over their transpose (formed once per call; the scatter
// SpMM where no transpose is given) and a fused diagonal/rank-one epilogue;
// the d x d matrix is never formed.
//
// Community model: Pairs(C,B) = (1/n_X) G_XC^T G_XB gets a rank-k randomised
// SVD (the pseudo-inverses of Eqs. (7)-(8)); Z_B, Z_C and M2 of Eq. (10) are
// then kept in factored form (Section 4.1, "we avoid products of sizes
// O(n) x O(n)"): with L = [L_C | L_B] (n_A x 2k) and K = U_C^T Pairs(C,B) V_B,
//   sym(M2) X = L [ (a0+1)/2 K (L_B^T X) ; (a0+1)/2 K^T (L_C^T X) ] - a0 M1 (M1^T X).
//
// Both then run the same range finder: Q = orth(M2 S); q times Q = orth(M2 Q);
// Omega = Q^T M2 Q; FP64 eigendecomposition; W = Q U_k Lambda_k^{-1/2}.  For the
// topic model Omega is formed as a Gram matrix, without the scatter product:
//   Omega = (a0+1)[(1/n) R^T R - D^T D] - a0 (Q^T M1)(M1^T Q),
//   R = diag(sqrt(w)) X Q (n x m, one gather SpMM),  D = diag(sqrt(delta)) Q,
// symmetric by construction (w and delta are non-negative).
//
// The topic model also has the paper's own Nystrom form (Algorithm 2): O = M2 S
// for a signed column selection S, Omega = S^T O, both decomposed at rank k,
// W = U_O L_O^{-1} V_O^T V_Omega L_Omega^{1/2} (d x k).
#include "otm_internal.cuh"

namespace otm {
namespace {

// O <- (a0 + 1)(O - diag(delta) S) - a0 M1 u^T (d x m), one warp per row in
// FP32 (FP64 issues at 1/64 of the FP32 rate on this part): the row's FP64
// values are converted once, delta_r = dh + dl as two floats so that
// delta_r S = dh S + dl S with dh S formed exactly (Dekker's product, FMA form);
// O - delta_r S then carries one float32 rounding, as the FP64 form does before
// its final rounding.  u (m values) is converted once per block (shared memory).
__global__ void __launch_bounds__(256) topic_m2_epilogue_kernel(
    float* __restrict__ O, const float* __restrict__ S, const double* __restrict__ delta,
    const double* __restrict__ M1, const double* __restrict__ u, int64_t d, int64_t m,
    double a0) {
  extern __shared__ float uf[];
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) uf[j] = (float)u[j];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const float c1 = (float)(a0 + 1.0);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < d; r += nw) {
    float dh = 0.f, dl = 0.f, am = 0.f;
    if (lane == 0) {
      const double dr = delta[r];
      dh = (float)dr;
      dl = (float)(dr - (double)dh);
      am = (float)(a0 * M1[r]);
    }
    dh = __shfl_sync(0xffffffffu, dh, 0);
    dl = __shfl_sync(0xffffffffu, dl, 0);
    am = __shfl_sync(0xffffffffu, am, 0);
    for (int64_t j = lane; j < m; j += 32) {
      const int64_t idx = r * m + j;
      const float sv = S[idx];
      const float p = __fmul_rn(dh, sv);
      const float e = fmaf(dh, sv, -p);  // dh sv = p + e exactly
      const float t = __fsub_rn(__fsub_rn(O[idx], p), fmaf(dl, sv, e));
      O[idx] = fmaf(c1, t, -am * uf[j]);
    }
  }
}

// out = diag(sqrt(delta)) Q (d x m): one warp per row, the square root once per row.
__global__ void __launch_bounds__(256) scale_rows_sqrt_kernel(const float* __restrict__ Q,
                                                              const double* __restrict__ delta,
                                                              int64_t d, int64_t m,
                                                              float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < d; r += nw) {
    float sr = 0.f;
    if (lane == 0) {
      const double w = delta[r];
      sr = (float)sqrt(w > 0.0 ? w : 0.0);
    }
    sr = __shfl_sync(0xffffffffu, sr, 0);
    for (int64_t j = lane; j < m; j += 32) out[r * m + j] = sr * Q[r * m + j];
  }
}

// Grid of the one-warp-per-row kernels: up to eight resident blocks per SM.
inline unsigned row_warp_blocks(int64_t rows) {
  const int64_t want = (rows + 7) / 8;
  return (unsigned)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
}

__global__ void sqrt_f32_kernel(const float* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = sqrtf(a[i] > 0.f ? a[i] : 0.f);
}

// Om (m x m) -= a0 u u^T.
__global__ void rank1_sub_kernel(double* __restrict__ Om, const double* __restrict__ u, int64_t m,
                                 double a0) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  Om[idx] -= a0 * u[idx / m] * u[idx % m];
}

__global__ void concat2_kernel(const float* __restrict__ A, const float* __restrict__ B,
                               int64_t rows, int64_t k, float* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * 2 * k) return;
  const int64_t r = idx / (2 * k), c = idx % (2 * k);
  out[idx] = c < k ? A[r * k + c] : B[r * k + c - k];
}

__global__ void scale_cols_mod_kernel(float* __restrict__ L, int64_t rows, int64_t k,
                                      const double* __restrict__ ev) {
  // L is rows x 2k; column c is divided by sigma_{c mod k} = sqrt(ev[c mod k]).
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * 2 * k) return;
  const int64_t c = idx % (2 * k);
  L[idx] = (float)((double)L[idx] / sqrt(ev[c % k]));
}

__global__ void sqrt_vec_kernel(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = sqrt(a[i] > 0.0 ? a[i] : 0.0);
}

// First k columns of an n x n row-major matrix -> n x k.
__global__ void take_cols_kernel(const double* __restrict__ a, int64_t n, int64_t k,
                                 float* __restrict__ b) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * k) return;
  b[idx] = (float)a[(idx / k) * n + idx % k];
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Nystrom whitening (Algorithm 2), k x k middle factors.  T1 = V_G,k^T V_Om,k;
// T2 = diag(1/ev_G) T1 diag(sqrt(ev_Om)); D = diag(ev_G) T2 = T1 diag(sqrt(ev_Om));
// eig = ev_Om[:k].  Flags the k-th eigenvalue of Omega (relative to the first,
// as for the range finder) and of G = O^T O not being positive.
__global__ void nystrom_scale_kernel(const double* __restrict__ T1, const double* __restrict__ evG,
                                     const double* __restrict__ evO, int64_t k,
                                     double* __restrict__ T2, double* __restrict__ D,
                                     double* __restrict__ eig, int* __restrict__ flag) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx == 0 && (!(evO[k - 1] > 1e-5 * fabs(evO[0])) || !(evG[k - 1] > 0.0))) *flag = 1;
  if (idx < k) eig[idx] = evO[idx];
  if (idx >= k * k) return;
  const int64_t a = idx / k, b = idx % k;
  const double so = evO[b] > 0.0 ? sqrt(evO[b]) : 0.0;
  const double g = evG[a] > 0.0 ? evG[a] : 1.0;
  D[idx] = T1[idx] * so;
  T2[idx] = T1[idx] * so / g;
}

// E = V diag(1/ev) (k x k, column scaling); flags a non-positive eigenvalue.
__global__ void inv_scale_cols_kernel(const double* __restrict__ V, const double* __restrict__ ev,
                                      int64_t k, double* __restrict__ E, int* __restrict__ flag) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx == 0 && !(ev[k - 1] > 0.0)) *flag = 1;
  if (idx >= k * k) return;
  const double e = ev[idx % k];
  E[idx] = e > 0.0 ? V[idx] / e : 0.0;
}

struct TopicOp {
  const otm_csr* X;
  const float* row_w;
  const double* M1;
  const double* delta;
  double a0;
  float* P;    // n x m scratch
  double* u;   // m scratch
  float* sqw;  // n: sqrt(row_w), for rayleigh (may be null if rayleigh is not used)
  // the transpose of X (CSR of X^T), or null: X^T P by the scatter SpMM
  const int32_t* colptr;
  const int32_t* rowT;
  const float* valT;
  otm_status apply(const float* S, int64_t m, float* O, cudaStream_t st) const {
    const int64_t n = X->rows, d = X->cols;
    const float inv_n = (float)(1.0 / (double)(n > 0 ? n : 1));
    OTM_TRY(spmm_gather(X, S, m, row_w, P, st));
    OTM_CHECK_CUDA(cudaMemsetAsync(O, 0, sizeof(float) * d * m, st));
    if (colptr)
      OTM_TRY(spmm_csc(colptr, rowT, valT, d, X->nnz, P, m, inv_n, O, st));
    else
      OTM_TRY(spmm_scatter(X, P, m, nullptr, inv_n, O, st));
    OTM_TRY(vec_tn(M1, S, d, m, u, st));
    topic_m2_epilogue_kernel<<<row_warp_blocks(d), 256, sizeof(float) * m, st>>>(O, S, delta, M1,
                                                                                 u, d, m, a0);
    OTM_CHECK_LAUNCH();
    return OTM_OK;
  }
  // Om = Q^T M2 Q (m x m, FP64) in the Gram form; D (d x m) is scratch.
  otm_status rayleigh(const float* Q, int64_t m, double* Om, float* D, cudaStream_t st) const {
    const int64_t n = X->rows, d = X->cols;
    OTM_TRY(spmm_gather(X, Q, m, sqw, P, st));
    OTM_TRY(gemm_tn_f64acc(P, P, n, m, m, (a0 + 1.0) / (double)(n > 0 ? n : 1), Om, 0, st));
    scale_rows_sqrt_kernel<<<row_warp_blocks(d), 256, 0, st>>>(Q, delta, d, m, D);
    OTM_CHECK_LAUNCH();
    OTM_TRY(gemm_tn_f64acc(D, D, d, m, m, -(a0 + 1.0), Om, 1, st));
    OTM_TRY(vec_tn(M1, Q, d, m, u, st));
    rank1_sub_kernel<<<blocks_for(m * m), 256, 0, st>>>(Om, u, m, a0);
    OTM_CHECK_LAUNCH();
    return OTM_OK;
  }
};

struct CommunityOp {
  const float* L;   // n_A x 2k  ([L_C | L_B])
  const double* K;  // k x k
  const double* M1; // n_A
  int64_t n_a, k;
  double a0;
  double* ab;    // 2k x m scratch
  double* coef;  // 2k x m scratch
  double* u;     // m scratch
  float* coef32; // 2k x m scratch
  otm_status apply(const float* X, int64_t m, float* O, cudaStream_t st) const {
    OTM_TRY(gemm_tn_f64acc(L, X, n_a, 2 * k, m, 1.0, ab, 0, st));  // [L_C^T X ; L_B^T X]
    OTM_TRY(vec_tn(M1, X, n_a, m, u, st));
    const double s = 0.5 * (a0 + 1.0);
    // top rows multiply L_C: s K (L_B^T X); bottom rows multiply L_B: s K^T (L_C^T X)
    OTM_TRY(dgemm_small(0, 0, k, m, k, s, K, k, ab + k * m, m, 0.0, coef, m, st));
    OTM_TRY(dgemm_small(1, 0, k, m, k, s, K, k, ab, m, 0.0, coef + k * m, m, st));
    OTM_TRY(f64_to_f32(coef, coef32, 2 * k * m, st));
    OTM_TRY(gemm_nn_small(L, n_a, 2 * k, coef32, m, O, M1, u, a0, st));
    return OTM_OK;
  }
  // Om = Q^T (M2 Q); O (n_A x m) is scratch.
  otm_status rayleigh(const float* Q, int64_t m, double* Om, float* O, cudaStream_t st) const {
    OTM_TRY(apply(Q, m, O, st));
    return gemm_tn_f64acc(Q, O, n_a, m, m, 1.0, Om, 0, st);
  }
};

// Range finder + QR + eig + whitening factors, shared by both models.
template <class Op>
otm_status range_finder(const Op& op, int64_t d, const float* S, int64_t k, int64_t kt,
                        int power_iters, float* W, float* Q, double* Cw, double* Cp, double* eig,
                        Workspace& ws, cudaStream_t st, int* flags) {
  float* O = ws.take<float>(d * kt);
  double* Om = ws.take<double>(kt * kt);
  double* ev = ws.take<double>(kt);
  double* evec = ws.take<double>(kt * kt);
  float* Cw32 = ws.take<float>(kt * k);
  if (!O || !Om || !ev || !evec || !Cw32)
    return set_error(OTM_EINVAL, "whiten: workspace too small");
  const size_t mark = ws.used;
  // intermediate bases need only be well conditioned -- the next product
  // depends on their span alone -- so one shifted Cholesky-QR pass; the last
  // one is orthonormalised fully
  OTM_TRY(op.apply(S, kt, Q, st));
  OTM_TRY(orthonormalize(Q, d, kt, ws, st, flags + 2, power_iters > 0 ? 1 : 4));
  ws.used = mark;
  for (int it = 0; it < power_iters; ++it) {
    OTM_TRY(op.apply(Q, kt, O, st));
    OTM_CHECK_CUDA(cudaMemcpyAsync(Q, O, sizeof(float) * d * kt, cudaMemcpyDeviceToDevice, st));
    OTM_TRY(orthonormalize(Q, d, kt, ws, st, flags + 2, it + 1 < power_iters ? 1 : 4));
    ws.used = mark;
  }
  OTM_TRY(op.rayleigh(Q, kt, Om, O, st));
  OTM_TRY(syev(Om, kt, ev, evec, ws, st, flags + 2));
  ws.used = mark;
  OTM_TRY(whitening_factors(ev, evec, kt, k, Cw, Cp, eig, flags, st, Cw32));
  OTM_TRY(gemm_nn_small(Q, d, kt, Cw32, k, W, nullptr, nullptr, 0.0, st));
  return OTM_OK;
}

// Flag slots written by the device: [0] k-th eigenvalue of M2 not resolvable,
// [1] Pairs(C,B) of numerical rank < k, [2] QR / eigensolver failure.
constexpr int kFlags = 4;

otm_status check_flags(int* flags, cudaStream_t st, const char* who) {
  int h[kFlags] = {0, 0, 0, 0};
  OTM_CHECK_CUDA(cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h[2]) return set_error(OTM_ENOTCONVERGED, "%s: QR or eigensolver failed (non-finite data or "
                             "Jacobi sweep limit)", who);
  if (h[1]) return set_error(OTM_ENOTPSD, "%s: Pairs(C,B) has numerical rank < k", who);
  if (h[0]) return set_error(OTM_ENOTPSD, "%s: fewer than k resolvable positive eigenvalues", who);
  return OTM_OK;
}

size_t range_finder_ws(int64_t d, int64_t kt) {
  WorkspaceSize w;
  w.add<float>(d * kt).add<double>(kt * kt).add<double>(kt).add<double>(kt * kt);
  w.add<float>(kt * 160);
  const size_t inner = orth_workspace(kt) > syev_workspace(kt) ? orth_workspace(kt)
                                                                  : syev_workspace(kt);
  return w.bytes() + inner;
}

otm_status pairs_apply_ws(const otm_csr* G1, const otm_csr* G2, const float* S, int64_t m,
                          float* O, float* tmp, cudaStream_t st) {
  const int64_t nx = G1->rows;
  OTM_TRY(spmm_gather(G2, S, m, nullptr, tmp, st));
  OTM_CHECK_CUDA(cudaMemsetAsync(O, 0, sizeof(float) * G1->cols * m, st));
  OTM_TRY(spmm_scatter(G1, tmp, m, nullptr, (float)(1.0 / (double)(nx > 0 ? nx : 1)), O, st));
  return OTM_OK;
}

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

size_t otm_topic_m2_workspace(int64_t n, int64_t m) {
  WorkspaceSize w;
  w.add<float>(n * m).add<double>(m);
  return w.bytes();
}

size_t otm_csr_transpose_workspace(int64_t n, int64_t d) {
  return csr_transpose_workspace(n, d) + 256;
}

otm_status otm_csr_transpose(const otm_csr* X, int32_t* colptr, int32_t* rowT, float* valT,
                             void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_TRY(check_csr(X, "otm_csr_transpose"));
  OTM_REQUIRE(colptr && (X->nnz == 0 || (rowT && valT)), "otm_csr_transpose: null output");
  Workspace w(ws, ws_bytes);
  uint8_t* scratch = w.take<uint8_t>(csr_transpose_workspace(X->rows, X->cols));
  OTM_REQUIRE(scratch, "otm_csr_transpose: workspace too small (need %zu bytes)",
              otm_csr_transpose_workspace(X->rows, X->cols));
  return csr_transpose(X, colptr, rowT, valT, scratch, as_stream(stream));
}

otm_status otm_topic_m2_apply(const otm_csr* X, const otm_csr* Xt, const float* row_w,
                              const double* M1, const double* delta, double alpha0,
                              const float* S, int64_t m, float* O, void* ws, size_t ws_bytes,
                              void* stream) {
  clear_error();
  OTM_TRY(check_csr(X, "otm_topic_m2_apply"));
  OTM_REQUIRE(m >= 1 && row_w && M1 && delta && S && O, "otm_topic_m2_apply: bad arguments");
  OTM_REQUIRE(S != O, "otm_topic_m2_apply: O must not alias S");
  if (Xt) {
    OTM_TRY(check_csr(Xt, "otm_topic_m2_apply (Xt)"));
    OTM_REQUIRE(Xt->rows == X->cols && Xt->cols == X->rows && Xt->nnz == X->nnz,
                "otm_topic_m2_apply: Xt is not the transpose of X (shape or nnz)");
    OTM_REQUIRE(m <= 384, "otm_topic_m2_apply: with Xt, m must be at most 384");
  }
  Workspace w(ws, ws_bytes);
  TopicOp op{X, row_w, M1, delta, alpha0, w.take<float>(X->rows * m), w.take<double>(m), nullptr,
             Xt ? Xt->row_ptr : nullptr, Xt ? Xt->col : nullptr, Xt ? Xt->val : nullptr};
  OTM_REQUIRE(op.P && op.u, "otm_topic_m2_apply: workspace too small (need %zu bytes)",
              otm_topic_m2_workspace(X->rows, m));
  return op.apply(S, m, O, as_stream(stream));
}

size_t otm_pairs_workspace(int64_t n_x, int64_t m) {
  WorkspaceSize w;
  w.add<float>(n_x * m);
  return w.bytes();
}

otm_status otm_pairs_apply(const otm_csr* G1, const otm_csr* G2, const float* S, int64_t m,
                           float* O, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_TRY(check_csr(G1, "otm_pairs_apply G1"));
  OTM_TRY(check_csr(G2, "otm_pairs_apply G2"));
  OTM_REQUIRE(G1->rows == G2->rows, "otm_pairs_apply: G1 and G2 need the same rows (n_X)");
  OTM_REQUIRE(m >= 1 && S && O, "otm_pairs_apply: bad arguments");
  Workspace w(ws, ws_bytes);
  float* tmp = w.take<float>(G2->rows * m);
  OTM_REQUIRE(tmp, "otm_pairs_apply: workspace too small");
  return pairs_apply_ws(G1, G2, S, m, O, tmp, as_stream(stream));
}

size_t otm_whiten_topic_workspace(int64_t n, int64_t d, int64_t nnz, int64_t k, int64_t kt) {
  (void)k;
  WorkspaceSize w;
  w.add<double>(d).add<float>(n * kt).add<double>(kt).add<int>(kFlags).add<float>(n);
  w.add<int32_t>(d + 1).add<int32_t>(nnz).add<float>(nnz);                  // transpose
  w.add<uint8_t>(csr_transpose_workspace(n, d)).add<double>(n).add<double>(n);  // its scratch, wa, wb
  return w.bytes() + range_finder_ws(d, kt);
}

otm_status otm_whiten_topic(const otm_csr* X, const float* S, int64_t k, int64_t kt,
                            int power_iters, double alpha0, float* W, float* Q, double* Cw,
                            double* Cp, double* eig, double* M1, float* row_invlen,
                            float* row_w, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_TRY(check_csr(X, "otm_whiten_topic"));
  OTM_REQUIRE(k >= 1 && kt > k && kt <= 160 && kt <= X->cols,
              "otm_whiten_topic: need 1 <= k < kt <= min(160, d) (k=%lld kt=%lld d=%lld)",
              (long long)k, (long long)kt, (long long)X->cols);
  OTM_REQUIRE(X->rows >= 1, "otm_whiten_topic: empty corpus");
  OTM_REQUIRE(power_iters >= 0 && power_iters <= 16, "otm_whiten_topic: power_iters in [0,16]");
  OTM_REQUIRE(alpha0 >= 0.0, "otm_whiten_topic: alpha0 must be >= 0");
  OTM_REQUIRE(S && W && Q && Cw && Cp && eig && M1 && row_invlen && row_w,
              "otm_whiten_topic: null output");
  OTM_REQUIRE(ws_bytes >= otm_whiten_topic_workspace(X->rows, X->cols, X->nnz, k, kt),
              "otm_whiten_topic: workspace too small (need %zu bytes)",
              otm_whiten_topic_workspace(X->rows, X->cols, X->nnz, k, kt));
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  double* delta = w.take<double>(X->cols);
  float* P = w.take<float>(X->rows * kt);
  double* u = w.take<double>(kt);
  int* flags = w.take<int>(kFlags);
  float* sqw = w.take<float>(X->rows);
  int32_t* colptr = w.take<int32_t>(X->cols + 1);
  int32_t* rowT = w.take<int32_t>(X->nnz);
  float* valT = w.take<float>(X->nnz);
  uint8_t* tscratch = w.take<uint8_t>(csr_transpose_workspace(X->rows, X->cols));
  double* wa = w.take<double>(X->rows);
  double* wb = w.take<double>(X->rows);
  OTM_CHECK_CUDA(cudaMemsetAsync(flags, 0, kFlags * sizeof(int), st));
  OTM_TRY(csr_transpose(X, colptr, rowT, valT, tscratch, st));
  OTM_TRY(topic_moments_csc(X, colptr, rowT, valT, wa, wb, row_invlen, row_w, M1, delta, st));
  sqrt_f32_kernel<<<blocks_for(X->rows), 256, 0, st>>>(row_w, sqw, X->rows);
  OTM_CHECK_LAUNCH();
  TopicOp op{X, row_w, M1, delta, alpha0, P, u, sqw, colptr, rowT, valT};
  OTM_TRY(range_finder(op, X->cols, S, k, kt, power_iters, W, Q, Cw, Cp, eig, w, st, flags));
  return check_flags(flags, st, "otm_whiten_topic");
}

size_t otm_whiten_community_workspace(int64_t n_x, int64_t n_a, int64_t n_b, int64_t n_c,
                                      int64_t k, int64_t kt) {
  WorkspaceSize w;
  w.add<float>(n_c * kt).add<float>(n_b * kt).add<float>(n_x * (kt > 2 * k ? kt : 2 * k));
  w.add<double>(kt * kt).add<double>(kt).add<double>(kt * kt);  // BB, ev, evec
  w.add<float>(kt * k).add<double>(kt * k).add<double>(kt * k).add<double>(k);  // Ub, Cv, Cu, s2
  w.add<float>(kt * k).add<float>(2 * k * kt).add<float>(2 * k * k);  // Cv32, coef32, LW32
  w.add<float>(n_c * k).add<float>(n_b * k);                      // U_C, V_B
  w.add<float>(n_x * k).add<float>(n_x * k).add<float>(n_a * 2 * k);  // CU, BV, L
  w.add<double>(k * k);                                           // K
  w.add<double>(2 * k * kt).add<double>(2 * k * kt).add<double>(kt);  // ab, coef, u
  w.add<double>(2 * k * k).add<int>(kFlags);                       // LW, flags
  const size_t a = w.bytes();
  const size_t inner = orth_workspace(kt) > syev_workspace(kt) ? orth_workspace(kt)
                                                                  : syev_workspace(kt);
  const size_t b = range_finder_ws(n_a, kt);
  return a + (b > inner ? b : inner);
}

otm_status otm_whiten_community(const otm_csr* G_XA, const otm_csr* G_XB, const otm_csr* G_XC,
                                const float* S_pairs, const float* S_w, int64_t k, int64_t kt,
                                int power_iters, double alpha0, float* W, float* W_B,
                                float* W_C, float* Q, double* Cw, double* Cp, double* eig,
                                double* sigma, double* M1, void* ws, size_t ws_bytes,
                                void* stream) {
  clear_error();
  OTM_TRY(check_csr(G_XA, "otm_whiten_community G_XA"));
  OTM_TRY(check_csr(G_XB, "otm_whiten_community G_XB"));
  OTM_TRY(check_csr(G_XC, "otm_whiten_community G_XC"));
  const int64_t nx = G_XA->rows, na = G_XA->cols, nb = G_XB->cols, nc = G_XC->cols;
  OTM_REQUIRE(G_XB->rows == nx && G_XC->rows == nx && nx >= 1,
              "otm_whiten_community: blocks must share the same (non-empty) X rows");
  OTM_REQUIRE(k >= 1 && kt > k && kt <= 160 && kt <= na && kt <= nb && kt <= nc && 2 * k <= 256,
              "otm_whiten_community: need 1 <= k < kt <= min(160, n_A, n_B, n_C)");
  OTM_REQUIRE(power_iters >= 0 && power_iters <= 16,
              "otm_whiten_community: power_iters in [0,16]");
  OTM_REQUIRE(alpha0 >= 0.0, "otm_whiten_community: alpha0 must be >= 0");
  OTM_REQUIRE(S_pairs && S_w && W && W_B && W_C && Q && Cw && Cp && eig && sigma && M1,
              "otm_whiten_community: null argument");
  const size_t need = otm_whiten_community_workspace(nx, na, nb, nc, k, kt);
  OTM_REQUIRE(ws_bytes >= need, "otm_whiten_community: workspace too small (need %zu bytes)",
              need);
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  float* Yc = w.take<float>(nc * kt);
  float* Zb = w.take<float>(nb * kt);
  float* tmp = w.take<float>(nx * (kt > 2 * k ? kt : 2 * k));
  double* BB = w.take<double>(kt * kt);
  double* ev = w.take<double>(kt);
  double* evec = w.take<double>(kt * kt);
  float* Ub = w.take<float>(kt * k);
  double* Cv = w.take<double>(kt * k);
  double* Cu = w.take<double>(kt * k);
  double* s2 = w.take<double>(k);
  float* U_C = w.take<float>(nc * k);
  float* V_B = w.take<float>(nb * k);
  float* CU = w.take<float>(nx * k);
  float* BV = w.take<float>(nx * k);
  float* L = w.take<float>(na * 2 * k);
  double* K = w.take<double>(k * k);
  double* ab = w.take<double>(2 * k * kt);
  double* coef = w.take<double>(2 * k * kt);
  double* u = w.take<double>(kt);
  double* LW = w.take<double>(2 * k * k);
  float* Cv32 = w.take<float>(kt * k);
  float* coef32 = w.take<float>(2 * k * kt);
  float* LW32 = w.take<float>(2 * k * k);
  int* flags = w.take<int>(kFlags);
  OTM_CHECK_CUDA(cudaMemsetAsync(flags, 0, kFlags * sizeof(int), st));
  const size_t mark = w.used;

  // 1. rank-k randomised SVD of Pairs(C,B) ~ U_C diag(sigma) V_B^T
  OTM_TRY(pairs_apply_ws(G_XC, G_XB, S_pairs, kt, Yc, tmp, st));
  OTM_TRY(orthonormalize(Yc, nc, kt, w, st, flags + 2, power_iters > 0 ? 1 : 4));
  w.used = mark;
  for (int it = 0; it < power_iters; ++it) {
    OTM_TRY(pairs_apply_ws(G_XB, G_XC, Yc, kt, Zb, tmp, st));
    OTM_TRY(orthonormalize(Zb, nb, kt, w, st, flags + 2, 1));
    w.used = mark;
    OTM_TRY(pairs_apply_ws(G_XC, G_XB, Zb, kt, Yc, tmp, st));
    OTM_TRY(orthonormalize(Yc, nc, kt, w, st, flags + 2, it + 1 < power_iters ? 1 : 4));
    w.used = mark;
  }
  OTM_TRY(pairs_apply_ws(G_XB, G_XC, Yc, kt, Zb, tmp, st));  // B^T = Pairs(B,C) Q
  OTM_TRY(gemm_tn_f64acc(Zb, Zb, nb, kt, kt, 1.0, BB, 0, st));
  OTM_TRY(syev(BB, kt, ev, evec, w, st, flags + 2));
  w.used = mark;
  take_cols_kernel<<<blocks_for(kt * k), 256, 0, st>>>(evec, kt, k, Ub);
  OTM_CHECK_LAUNCH();
  OTM_TRY(whitening_factors(ev, evec, kt, k, Cv, Cu, s2, flags + 1, st, Cv32));  // Ub / sigma
  sqrt_vec_kernel<<<blocks_for(k), 256, 0, st>>>(s2, sigma, k);
  OTM_CHECK_LAUNCH();
  OTM_TRY(gemm_nn_small(Yc, nc, kt, Ub, k, U_C, nullptr, nullptr, 0.0, st));
  OTM_TRY(gemm_nn_small(Zb, nb, kt, Cv32, k, V_B, nullptr, nullptr, 0.0, st));

  // 2. factors of Z_B, Z_C and the middle matrix K
  OTM_TRY(spmm_gather(G_XC, U_C, k, nullptr, CU, st));
  OTM_TRY(spmm_gather(G_XB, V_B, k, nullptr, BV, st));
  concat2_kernel<<<blocks_for(nx * 2 * k), 256, 0, st>>>(BV, CU, nx, k, tmp);
  OTM_CHECK_LAUNCH();
  OTM_CHECK_CUDA(cudaMemsetAsync(L, 0, sizeof(float) * na * 2 * k, st));
  OTM_TRY(spmm_scatter(G_XA, tmp, 2 * k, nullptr, (float)(1.0 / (double)nx), L, st));
  scale_cols_mod_kernel<<<blocks_for(na * 2 * k), 256, 0, st>>>(L, na, k, s2);
  OTM_CHECK_LAUNCH();
  OTM_TRY(gemm_tn_f64acc(CU, BV, nx, k, k, 1.0 / (double)nx, K, 0, st));
  OTM_TRY(column_sums_scaled(G_XA, 1.0 / (double)nx, M1, st));

  // 3. range-finder whitening of sym(M2)
  CommunityOp op{L, K, M1, na, k, alpha0, ab, coef, u, coef32};
  OTM_TRY(range_finder(op, na, S_w, k, kt, power_iters, W, Q, Cw, Cp, eig, w, st, flags));

  // 4. other views: W_B = Z_B^T W = V_B (L_B^T W), W_C = Z_C^T W = U_C (L_C^T W)
  OTM_TRY(gemm_tn_f64acc(L, W, na, 2 * k, k, 1.0, LW, 0, st));
  OTM_TRY(f64_to_f32(LW, LW32, 2 * k * k, st));
  OTM_TRY(gemm_nn_small(V_B, nb, k, LW32 + k * k, k, W_B, nullptr, nullptr, 0.0, st));
  OTM_TRY(gemm_nn_small(U_C, nc, k, LW32, k, W_C, nullptr, nullptr, 0.0, st));

  return check_flags(flags, st, "otm_whiten_community");
}


size_t otm_whiten_topic_nystrom_workspace(int64_t n, int64_t d, int64_t k, int64_t kt) {
  WorkspaceSize w;
  w.add<double>(d).add<float>(n * kt).add<double>(kt).add<int>(kFlags);
  w.add<double>(kt * kt).add<double>(kt * kt);                  // G, Omega
  w.add<double>(kt).add<double>(kt * kt).add<double>(kt).add<double>(kt * kt);  // eigenpairs
  for (int i = 0; i < 6; ++i) w.add<double>(k * k);             // T1, T2, D, H, E, Hinv
  w.add<double>(k).add<double>(k * k).add<float>(kt * k);       // evH, vecH, Cw32
  return w.bytes() + syev_workspace(kt);
}

otm_status otm_whiten_topic_nystrom(const otm_csr* X, const float* S, int64_t k, int64_t kt,
                                    double alpha0, float* W, float* O, double* Cw, double* Cp,
                                    double* eig, double* M1, float* row_invlen, float* row_w,
                                    void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_TRY(check_csr(X, "otm_whiten_topic_nystrom"));
  OTM_REQUIRE(k >= 1 && kt > k && kt <= 160 && kt <= X->cols,
              "otm_whiten_topic_nystrom: need 1 <= k < kt <= min(160, d) (k=%lld kt=%lld "
              "d=%lld)", (long long)k, (long long)kt, (long long)X->cols);
  OTM_REQUIRE(X->rows >= 1, "otm_whiten_topic_nystrom: empty corpus");
  OTM_REQUIRE(alpha0 >= 0.0, "otm_whiten_topic_nystrom: alpha0 must be >= 0");
  OTM_REQUIRE(S && W && O && Cw && Cp && eig && M1 && row_invlen && row_w,
              "otm_whiten_topic_nystrom: null argument");
  OTM_REQUIRE(S != O, "otm_whiten_topic_nystrom: O must not alias S");
  const size_t need = otm_whiten_topic_nystrom_workspace(X->rows, X->cols, k, kt);
  OTM_REQUIRE(ws_bytes >= need, "otm_whiten_topic_nystrom: workspace too small (need %zu bytes)",
              need);
  cudaStream_t st = as_stream(stream);
  const int64_t d = X->cols;
  Workspace w(ws, ws_bytes);
  double* delta = w.take<double>(d);
  float* P = w.take<float>(X->rows * kt);
  double* u = w.take<double>(kt);
  int* flags = w.take<int>(kFlags);
  double* G = w.take<double>(kt * kt);
  double* Om = w.take<double>(kt * kt);
  double* evG = w.take<double>(kt);
  double* vecG = w.take<double>(kt * kt);
  double* evO = w.take<double>(kt);
  double* vecO = w.take<double>(kt * kt);
  double* T1 = w.take<double>(k * k);
  double* T2 = w.take<double>(k * k);
  double* D = w.take<double>(k * k);
  double* H = w.take<double>(k * k);
  double* E = w.take<double>(k * k);
  double* Hinv = w.take<double>(k * k);
  double* evH = w.take<double>(k);
  double* vecH = w.take<double>(k * k);
  float* Cw32 = w.take<float>(kt * k);
  const size_t mark = w.used;
  OTM_CHECK_CUDA(cudaMemsetAsync(flags, 0, kFlags * sizeof(int), st));
  OTM_TRY(topic_moments(X, row_invlen, row_w, M1, delta, st));
  TopicOp op{X, row_w, M1, delta, alpha0, P, u};
  // O = M2 S; G = O^T O (its eigenpairs give the SVD of O); Omega = S^T O
  OTM_TRY(op.apply(S, kt, O, st));
  OTM_TRY(gemm_tn_f64acc(O, O, d, kt, kt, 1.0, G, 0, st));
  OTM_TRY(gemm_tn_f64acc(S, O, d, kt, kt, 1.0, Om, 0, st));
  OTM_TRY(syev(G, kt, evG, vecG, w, st, flags + 2));
  w.used = mark;
  OTM_TRY(syev(Om, kt, evO, vecO, w, st, flags + 2));
  w.used = mark;
  // C = V_G,k diag(1/ev_G) V_G,k^T V_Om,k diag(sqrt(ev_Om)) = U_O L_O^-1 V_O^T V_Om L_Om^1/2
  // expressed on O (U_O = O V_O L_O^-1), so that W = O C
  OTM_TRY(dgemm_small(1, 0, k, k, kt, 1.0, vecG, kt, vecO, kt, 0.0, T1, k, st));
  nystrom_scale_kernel<<<blocks_for(k * k), 256, 0, st>>>(T1, evG, evO, k, T2, D, eig, flags);
  OTM_CHECK_LAUNCH();
  OTM_TRY(dgemm_small(0, 0, kt, k, k, 1.0, vecG, kt, T2, k, 0.0, Cw, k, st));
  // (W^T)^+ = W (W^T W)^-1 = O C H^-1 with H = C^T G C = T2^T diag(ev_G) T2
  OTM_TRY(dgemm_small(1, 0, k, k, k, 1.0, T2, k, D, k, 0.0, H, k, st));
  OTM_TRY(syev(H, k, evH, vecH, w, st, flags + 2));
  w.used = mark;
  inv_scale_cols_kernel<<<blocks_for(k * k), 256, 0, st>>>(vecH, evH, k, E, flags);
  OTM_CHECK_LAUNCH();
  OTM_TRY(dgemm_small(0, 1, k, k, k, 1.0, E, k, vecH, k, 0.0, Hinv, k, st));
  OTM_TRY(dgemm_small(0, 0, kt, k, k, 1.0, Cw, k, Hinv, k, 0.0, Cp, k, st));
  OTM_TRY(f64_to_f32(Cw, Cw32, kt * k, st));
  OTM_TRY(gemm_nn_small(O, d, kt, Cw32, k, W, nullptr, nullptr, 0.0, st));
  return check_flags(flags, st, "otm_whiten_topic_nystrom");
}

}  // extern "C"
