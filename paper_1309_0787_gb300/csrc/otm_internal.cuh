// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/otm.h"

namespace otm {

// Thread-local error message (otm_last_error).
otm_status set_error(otm_status st, const char* fmt, ...);
void clear_error();

#define OTM_CHECK_CUDA(expr)                                                       \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return ::otm::set_error(OTM_ECUDA, "%s failed: %s (%s:%d)", #expr,           \
                              cudaGetErrorString(e_), __FILE__, __LINE__);         \
  } while (0)

void count_launch();

#define OTM_CHECK_LAUNCH()      \
  do {                          \
    ::otm::count_launch();      \
    OTM_CHECK_CUDA(cudaGetLastError()); \
  } while (0)

#define OTM_TRY(expr)                  \
  do {                                 \
    otm_status s_ = (expr);            \
    if (s_ != OTM_OK) return s_;       \
  } while (0)

#define OTM_REQUIRE(cond, ...)                                  \
  do {                                                          \
    if (!(cond)) return ::otm::set_error(OTM_EINVAL, __VA_ARGS__); \
  } while (0)

// Bump allocator over a caller-provided workspace; 256-byte aligned slices.
struct Workspace {
  char* base;
  size_t size;
  size_t used;
  Workspace(void* p, size_t n) : base(static_cast<char*>(p)), size(n), used(0) {}
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    size_t bytes = count * sizeof(T);
    if (base == nullptr || off + bytes > size) return nullptr;
    used = off + bytes;
    return reinterpret_cast<T*>(base + off);
  }
};

// Size accounting that mirrors Workspace::take.
struct WorkspaceSize {
  size_t used = 0;
  template <typename T>
  WorkspaceSize& add(size_t count) {
    used = ((used + 255) & ~size_t(255)) + count * sizeof(T);
    return *this;
  }
  size_t bytes() const { return used + 256; }
};

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

otm_status check_csr(const otm_csr* X, const char* name);

// ---- sparse kernels (sparse.cu) ----
// out[r, :] = row_scale[r] * sum_e val[e] * B[col[e], :]   (gather SpMM)
otm_status spmm_gather(const otm_csr* X, const float* B, int64_t m, const float* row_scale,
                       float* out, cudaStream_t st);
// out[col[e], :] += alpha * row_scale[r] * val[e] * P[r, :]  (scatter SpMM, out pre-zeroed)
otm_status spmm_scatter(const otm_csr* X, const float* P, int64_t m, const float* row_scale,
                        float alpha, float* out, cudaStream_t st);
otm_status topic_moments(const otm_csr* X, float* row_invlen, float* row_w, double* M1,
                         double* delta, cudaStream_t st);
// The CSR of X^T: colptr (cols + 1), rowT, valT (nnz each); scratch of
// csr_transpose_workspace(rows, cols) bytes (256-byte aligned).  A counting sort
// by word over row blocks where a word's count per block fits shared memory,
// else one global atomic position per entry.  The order of the entries within
// a column is not fixed.  X must have distinct columns within each row.
size_t csr_transpose_workspace(int64_t n, int64_t d);
otm_status csr_transpose(const otm_csr* X, int32_t* colptr, int32_t* rowT, float* valT,
                         void* scratch, cudaStream_t st);
// topic_moments over the transpose; wa, wb (rows, FP64) are scratch.
otm_status topic_moments_csc(const otm_csr* X, const int32_t* colptr, const int32_t* rowT,
                             const float* valT, double* wa, double* wb, float* row_invlen,
                             float* row_w, double* M1, double* delta, cudaStream_t st);
// out (d x m) += alpha * X^T P over the transpose of X (out pre-zeroed; m <= 384).
otm_status spmm_csc(const int32_t* colptr, const int32_t* rowT, const float* valT, int64_t d,
                    int64_t nnz, const float* P, int64_t m, float alpha, float* out,
                    cudaStream_t st);
// M1[c] = (1/rows) sum_r X[r, c]  (community first moment, Eq. (9))
otm_status column_sums_scaled(const otm_csr* X, double scale, double* out, cudaStream_t st);

// ---- dense kernels (dense.cu) ----
// C (m x p, FP64) = alpha * A^T B, A: rows x m, B: rows x p, float32 row-major.
// If accumulate == 0 C is overwritten, else added to.
otm_status gemm_tn_f64acc(const float* A, const float* B, int64_t rows, int64_t m, int64_t p,
                          double alpha, double* C, int accumulate, cudaStream_t st,
                          const int* skip = nullptr);
// out (rows x p, float32) = A (rows x m, float32) * C (m x p, float32)
//   [+ rank-one term: - r1_alpha * r1_u[r] * r1_v[c]] [then * colscale[c]]
otm_status gemm_nn_small(const float* A, int64_t rows, int64_t m, const float* C, int64_t p,
                         float* out, const double* r1_u, const double* r1_v, double r1_alpha,
                         cudaStream_t st, const int* skip = nullptr);
otm_status f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t st);
// out (rows x p, FP64) = A (rows x m, float32) * C (m x p, FP64), sums accurate to
// about 2^-48 (double-float arithmetic on the FP32 units).
otm_status gemm_nn_f64(const float* A, int64_t rows, int64_t m, const double* C, int64_t p,
                       double* out, cudaStream_t st);
// Small FP64 GEMM: C (m x n) = op(A) op(B), op = transpose if flag set.
otm_status dgemm_small(int ta, int tb, int64_t m, int64_t n, int64_t kk, double alpha,
                       const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                       double* C, int64_t ldc, cudaStream_t st);
// FP32 STGD (Lemma 3) as one cooperative launch over many SMs (sgd_grid.cu):
// the minibatch split over up to one CTA per SM, partial products reduced
// through L2 by the owners of the columns; same arguments and results as
// otm_sgd_run.  Applicable for k <= 128 and 16 <= b <= 32 x (SM count).
bool sgd_grid_applicable(int64_t k, int64_t b);
size_t sgd_grid_workspace(int64_t k, int64_t b);  // 0 where not applicable
otm_status sgd_grid_run(float* V, const float* YA, const float* YB, const float* YC, int64_t n,
                        int64_t k, const double* ybar3, const int32_t* perm, int64_t epochs,
                        int64_t b, double beta0, double theta, double alpha0,
                        int64_t snapshot_every, float* V_snap, void* ws, size_t ws_bytes,
                        cudaStream_t st);
// FP32 STGD, split form (sgd_split.cu): clusters own blocks of components, the
// CTAs of a cluster split every minibatch, partial columns reduced through
// distributed shared memory, one grid barrier per step; same arguments and
// results as otm_sgd_run.  Applicable for k <= 128 when all its clusters can be
// resident at once.
bool sgd_split_applicable(int64_t k, int64_t b, bool sym);
size_t sgd_split_workspace(int64_t k);  // 0 where k is out of range
otm_status sgd_split_run(float* V, const float* YA, const float* YB, const float* YC, int64_t n,
                         int64_t k, const double* ybar3, const int32_t* perm, int64_t epochs,
                         int64_t b, double beta0, double theta, double alpha0,
                         int64_t snapshot_every, float* V_snap, void* ws, size_t ws_bytes,
                         cudaStream_t st);
size_t orth_workspace(int64_t m);
// Device-side failure flags: *dflag is set to 1 (QR: non-finite Gram matrix) or
// 2 (eigensolver: non-finite eigenvalues) or 3 (eigensolver: the refinement's grid
// barrier timed out); callers zero it and check it once.
// passes: Cholesky-QR passes (pass 0 shifted, pass 1 plain, passes 2-3 only while
// the basis is not yet orthonormal to 1e-5); the one shifted pass suffices for
// the intermediate bases of a power iteration, whose span is all that matters
// (it leaves a well-conditioned, not an orthonormal, basis).
otm_status orthonormalize(float* A, int64_t rows, int64_t m, Workspace& ws, cudaStream_t st,
                          int* dflag, int passes = 4);
size_t syev_workspace(int64_t n);
otm_status syev(const double* A, int64_t n, double* evals, double* evecs, Workspace& ws,
                cudaStream_t st, int* dflag);
// out[j] = sum_r u[r] * A[r, j]  (FP64 u, float32 A rows x m)
otm_status vec_tn(const double* u, const float* A, int64_t rows, int64_t m, double* out,
                  cudaStream_t st);
// From evals (descending, n) and evecs (n x n): Cw[:, i] = U[:, i] / sqrt(l_i),
// Cp[:, i] = U[:, i] * sqrt(l_i) for i < k (n x k each, FP64); eig[i] = l_i.
// Sets *flag (device int) to 1 if l_{k-1} <= 0.
otm_status whitening_factors(const double* evals, const double* evecs, int64_t n, int64_t k,
                             double* Cw, double* Cp, double* eig, int* flag, cudaStream_t st,
                             float* Cw32 = nullptr);

// ---- whitening composites (whiten.cu) ----

// ---- tensor-core GEMM (gemm_tc.cu) ----
// C[z] = alpha A[z] B[z]^T (BF16 row-major operands, K-major; FP32 accumulate).
// mode 0: C = acc (FP32, optional) and H = bf16(acc) (optional);
// mode 1: as 0 with + bias[col]; mode 2: C = acc + bias (pre-activation, optional),
// H = bf16(GELU(C)).  K, lda, ldb, batch strides multiples of 8.  *err is set
// non-zero if a device wait timed out.
otm_status gemm_bf16_nt(const void* A, const void* B, int64_t M, int64_t N, int64_t K,
                        int64_t batch, int64_t lda, int64_t ldb, int64_t sA, int64_t sB, int mode,
                        float alpha, const float* bias, float* C, int64_t ldc, int64_t sC, void* H,
                        int64_t ldh, int64_t sH, int* err, cudaStream_t st);

}  // namespace otm
