// Dense kernels of the whitening (Section 4.2): tall-skinny products, the
// tall-thin QR (shifted Cholesky-QR, three passes) and the small symmetric
// eigensolver behind the "short-thin SVD" (Table 3).
//
// Precision policy: tall matrices (d x k~) are float32; reductions over their
// long dimension are accumulated in FP32 over short row blocks and in FP64
// across blocks.  The k~ x k~ eigenproblem is solved to FP64 accuracy: cyclic
// Jacobi in FP32 inside one CTA, then FP64 iterative refinement of the
// eigenvectors (Ogita & Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018), whose
// O(n^3) work is FP64 GEMMs spread over many CTAs (FP64 issue rate per SM is
// low on this part, so no FP64 loop runs inside a single CTA).
#include <math.h>

#include "otm_internal.cuh"

namespace otm {
namespace {

// ---------------------------------------------------------------------------
// C (m x p, FP64) (+)= alpha * A^T B.  A: rows x m, B: rows x p (float32).
// Block: 64 x 64 output tile, 256 threads (4 x 4 each).  Rows are split over
// gridDim.z; inside a block 32-row slabs are summed in FP32, slabs in FP64.
// ---------------------------------------------------------------------------
constexpr int TN_T = 64, TN_R = 32;

__global__ void __launch_bounds__(256) gemm_tn_kernel(const float* __restrict__ A,
                                                      const float* __restrict__ B, int64_t rows,
                                                      int64_t m, int64_t p, double alpha,
                                                      double* __restrict__ C,
                                                      int64_t rows_per_split) {
  __shared__ float As[TN_R][TN_T];
  __shared__ float Bs[TN_R][TN_T];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * TN_T, j0 = (int64_t)blockIdx.y * TN_T;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t r_end = min(rows, r_begin + rows_per_split);
  double accd[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) accd[a][b] = 0.0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += TN_R) {
    for (int idx = threadIdx.x; idx < TN_R * TN_T; idx += 256) {
      const int rr = idx / TN_T, cc = idx % TN_T;
      const int64_t r = r0 + rr;
      As[rr][cc] = (r < r_end && i0 + cc < m) ? A[r * m + i0 + cc] : 0.f;
      Bs[rr][cc] = (r < r_end && j0 + cc < p) ? B[r * p + j0 + cc] : 0.f;
    }
    __syncthreads();
    float acc[4][4] = {};
#pragma unroll 8
    for (int rr = 0; rr < TN_R; ++rr) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[rr][ty + 16 * q];
        b[q] = Bs[rr][tx + 16 * q];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) accd[x][y] += (double)acc[x][y];
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t i = i0 + ty + 16 * x, j = j0 + tx + 16 * y;
      if (i < m && j < p) atomicAdd(&C[i * p + j], alpha * accd[x][y]);
    }
}

// ---------------------------------------------------------------------------
// out (rows x p) = A (rows x m) * C (m x p, FP64 staged as float32)
//                  - r1_alpha * r1_u[r] * r1_v[c]   (optional rank-one term)
// One block owns 32 whole rows (all p <= 256 columns), so A may alias out.
// ---------------------------------------------------------------------------
constexpr int NN_R = 32, NN_K = 32, NN_PMAX = 256;

__global__ void __launch_bounds__(256) gemm_nn_small_kernel(
    const float* A, int64_t rows, int64_t m, const double* __restrict__ C, int64_t p, float* out,
    const double* __restrict__ r1_u, const double* __restrict__ r1_v, double r1_alpha) {
  __shared__ float As[NN_R][NN_K + 1];
  __shared__ float Cs[NN_K][NN_PMAX];
  const int cg = threadIdx.x & 31;   // column group: columns cg + 32 j
  const int rg = threadIdx.x >> 5;   // row group: rows 4 rg .. 4 rg + 3
  const int64_t r0 = (int64_t)blockIdx.x * NN_R;
  const int ncj = (int)((p + 31) / 32);
  float acc[4][NN_PMAX / 32];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int j = 0; j < NN_PMAX / 32; ++j) acc[a][j] = 0.f;
  for (int64_t k0 = 0; k0 < m; k0 += NN_K) {
    for (int idx = threadIdx.x; idx < NN_R * NN_K; idx += 256) {
      const int rr = idx / NN_K, kk = idx % NN_K;
      const int64_t r = r0 + rr, k = k0 + kk;
      As[rr][kk] = (r < rows && k < m) ? A[r * m + k] : 0.f;
    }
    for (int idx = threadIdx.x; idx < NN_K * NN_PMAX; idx += 256) {
      const int kk = idx / NN_PMAX, c = idx % NN_PMAX;
      const int64_t k = k0 + kk;
      Cs[kk][c] = (k < m && c < p) ? (float)C[k * p + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < NN_K; ++kk) {
      float a[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = As[4 * rg + q][kk];
#pragma unroll
      for (int j = 0; j < NN_PMAX / 32; ++j) {
        if (j < ncj) {
          const float c = Cs[kk][cg + 32 * j];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q][j] = fmaf(a[q], c, acc[q][j]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t r = r0 + 4 * rg + q;
    if (r >= rows) continue;
    const double u = r1_u ? r1_u[r] * r1_alpha : 0.0;
#pragma unroll
    for (int j = 0; j < NN_PMAX / 32; ++j) {
      const int64_t c = cg + 32 * j;
      if (j < ncj && c < p) {
        float v = acc[q][j];
        if (r1_u) v = (float)((double)v - u * r1_v[c]);
        out[r * p + c] = v;
      }
    }
  }
}

// out (rows x p, FP64) = A (rows x m, float32) * C (m x p, FP64), FP64 FMAs.
constexpr int D_R = 32, D_C = 32, D_K = 32;
__global__ void __launch_bounds__(256) gemm_nn_f64_kernel(const float* __restrict__ A,
                                                          int64_t rows, int64_t m,
                                                          const double* __restrict__ C,
                                                          int64_t p, double* __restrict__ out) {
  __shared__ double As[D_R][D_K + 1];
  __shared__ double Cs[D_K][D_C];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 4 rows per thread
  const int64_t r0 = (int64_t)blockIdx.x * D_R, c0 = (int64_t)blockIdx.y * D_C;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t k0 = 0; k0 < m; k0 += D_K) {
    for (int idx = threadIdx.x; idx < D_R * D_K; idx += 256) {
      const int rr = idx / D_K, kk = idx % D_K;
      As[rr][kk] = (r0 + rr < rows && k0 + kk < m) ? (double)A[(r0 + rr) * m + k0 + kk] : 0.0;
      Cs[rr][kk] = (k0 + rr < m && c0 + kk < p) ? C[(k0 + rr) * p + c0 + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < D_K; ++kk) {
      const double c = Cs[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty * 4 + q][kk], c, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t r = r0 + ty * 4 + q, c = c0 + tx;
    if (r < rows && c < p) out[r * p + c] = acc[q];
  }
}

// Small FP64 GEMM, C = alpha op(A) op(B) + beta C, 16 x 16 tiles, one output
// per thread.  A is m x kk (or kk x m when ta), B is kk x n (or n x kk when tb).
__global__ void __launch_bounds__(256) dgemm_small_kernel(int ta, int tb, int64_t m, int64_t n,
                                                          int64_t kk, double alpha,
                                                          const double* __restrict__ A,
                                                          int64_t lda,
                                                          const double* __restrict__ B,
                                                          int64_t ldb, double beta, double* C,
                                                          int64_t ldc) {
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i = (int64_t)blockIdx.y * 16 + ty, j = (int64_t)blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int64_t k0 = 0; k0 < kk; k0 += 16) {
    {
      const int64_t ii = (int64_t)blockIdx.y * 16 + ty, k = k0 + tx;
      double v = 0.0;
      if (ii < m && k < kk) v = ta ? A[k * lda + ii] : A[ii * lda + k];
      As[ty][tx] = v;
    }
    {
      const int64_t k = k0 + ty, jj = (int64_t)blockIdx.x * 16 + tx;
      double v = 0.0;
      if (k < kk && jj < n) v = tb ? B[jj * ldb + k] : B[k * ldb + jj];
      Bs[ty][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc = fma(As[ty][q], Bs[q][tx], acc);
    __syncthreads();
  }
  if (i < m && j < n) C[i * ldc + j] = alpha * acc + (beta != 0.0 ? beta * C[i * ldc + j] : 0.0);
}

__global__ void vec_tn_kernel(const double* __restrict__ u, const float* __restrict__ A,
                              int64_t rows, int64_t m, int64_t rows_per_block,
                              double* __restrict__ out) {
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r_end = min(rows, r_begin + rows_per_block);
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
    double acc = 0.0;
    for (int64_t r = r_begin; r < r_end; ++r) acc = fma(u[r], (double)A[r * m + j], acc);
    atomicAdd(&out[j], acc);
  }
}

// ---------------------------------------------------------------------------
// Cholesky of G (+ shift) and the inverse of its upper factor R = L^T.
// One CTA, FP32 in shared memory (n <= 160).  Output Rinv (n x n, FP64,
// row-major, upper triangular) so that Q = A Rinv.
// shift_scale > 0 adds shift_scale * n * u * trace(G) to the diagonal
// (u = 2^-24), which keeps the factorisation positive definite for Gram
// matrices of ill-conditioned A (shifted Cholesky-QR: Fukaya, Kannan,
// Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 42, 2020).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) chol_inv_kernel(const double* __restrict__ G, int n,
                                                        double shift_scale,
                                                        double* __restrict__ Rinv,
                                                        int* __restrict__ flag) {
  extern __shared__ float sm[];
  float* L = sm;              // n x n, lower triangle used
  float* Li = sm + n * n;     // n x n, inverse of L (lower)
  __shared__ float s_shift;
  __shared__ int s_bad;
  const int tid = threadIdx.x, T = blockDim.x;
  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += G[i * n + i];
    s_shift = (float)(shift_scale * (double)n * 5.9604644775390625e-8 * tr);
    s_bad = 0;
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx % n;
    float v = (float)(0.5 * (G[i * n + j] + G[j * n + i]));
    if (i == j) v += s_shift;
    L[idx] = v;
    Li[idx] = 0.f;
  }
  __syncthreads();
  // right-looking Cholesky, column by column
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const float d = L[j * n + j];
      if (!(d > 0.f)) {
        s_bad = 1;
        L[j * n + j] = 1.f;
      } else {
        L[j * n + j] = sqrtf(d);
      }
    }
    __syncthreads();
    const float djj = L[j * n + j];
    for (int i = j + 1 + tid; i < n; i += T) L[i * n + j] /= djj;
    __syncthreads();
    const int rem = n - j - 1;
    for (int idx = tid; idx < rem * rem; idx += T) {
      const int i = j + 1 + idx / rem, l = j + 1 + idx % rem;
      if (l <= i) L[i * n + l] -= L[i * n + j] * L[l * n + j];
    }
    __syncthreads();
  }
  // inverse of lower-triangular L: column c by forward substitution (thread per column)
  for (int c = tid; c < n; c += T) {
    Li[c * n + c] = 1.f / L[c * n + c];
    for (int i = c + 1; i < n; ++i) {
      float s = 0.f;
      for (int l = c; l < i; ++l) s = fmaf(L[i * n + l], Li[l * n + c], s);
      Li[i * n + c] = -s / L[i * n + i];
    }
  }
  __syncthreads();
  // Rinv = (L^T)^{-1} = (L^{-1})^T
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx % n;
    Rinv[idx] = (double)Li[j * n + i];
  }
  if (tid == 0 && s_bad) *flag = 1;
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi (FP32, one CTA), round-robin parallel ordering: each round
// applies n/2 disjoint rotations, first to columns (A J, V J) then to rows
// (J^T A).  Rotation angle from the 2 x 2 symmetric Schur decomposition.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int rr_member(int pos, int round, int np) {
  // circle method: position 0 fixed, the others rotate by `round`
  if (pos == 0) return 0;
  return 1 + (pos - 1 + round) % (np - 1);
}

__global__ void __launch_bounds__(1024) jacobi_f32_kernel(const double* __restrict__ A0, int n,
                                                          int max_sweeps, double* __restrict__ V_out,
                                                          int* __restrict__ flag) {
  extern __shared__ float sm[];
  float* A = sm;              // n x n
  float* V = sm + n * n;      // n x n, columns = eigenvectors
  float* cs = V + n * n;      // [np/2] cos, [np/2] sin
  int* pq = reinterpret_cast<int*>(cs + n + 2);  // [np/2] p, [np/2] q
  __shared__ float s_red[32];
  __shared__ int s_done;
  const int tid = threadIdx.x, T = blockDim.x;
  const int np = n + (n & 1), half = np / 2;
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx % n;
    A[idx] = (float)(0.5 * (A0[i * n + j] + A0[j * n + i]));
    V[idx] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence test: off(A)^2 <= tol^2 * ||A||_F^2
    float off = 0.f, tot = 0.f;
    for (int idx = tid; idx < n * n; idx += T) {
      const float v = A[idx] * A[idx];
      tot += v;
      if (idx / n != idx % n) off += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) s_red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      float o2 = 0.f;
      for (int w = 0; w < (T + 31) / 32; ++w) o2 += s_red[w];
      s_red[0] = o2;
    }
    __syncthreads();
    const float off_all = s_red[0];
    __syncthreads();
    if ((tid & 31) == 0) s_red[tid >> 5] = tot;
    __syncthreads();
    if (tid == 0) {
      float t2 = 0.f;
      for (int w = 0; w < (T + 31) / 32; ++w) t2 += s_red[w];
      s_done = (off_all <= 1e-11f * t2) ? 1 : 0;
    }
    __syncthreads();
    if (s_done) break;
    for (int round = 0; round < np - 1; ++round) {
      if (tid < half) {
        int p = rr_member(tid, round, np), q = rr_member(np - 1 - tid, round, np);
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < n) {
          const float apq = A[p * n + q];
          const float app = A[p * n + p], aqq = A[q * n + q];
          if (fabsf(apq) > 1e-30f && fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq))) {
            const float tau = (aqq - app) / (2.f * apq);
            const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            s = t * c;
          }
        }
        cs[tid] = c;
        cs[half + tid] = s;
        pq[tid] = p;
        pq[half + tid] = q;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int idx = tid; idx < half * n; idx += T) {
        const int w = idx / n, r = idx % n;
        const int p = pq[w], q = pq[half + w];
        if (q >= n) continue;
        const float c = cs[w], s = cs[half + w];
        if (s == 0.f) continue;
        const float ap = A[r * n + p], aq = A[r * n + q];
        A[r * n + p] = c * ap - s * aq;
        A[r * n + q] = s * ap + c * aq;
        const float vp = V[r * n + p], vq = V[r * n + q];
        V[r * n + p] = c * vp - s * vq;
        V[r * n + q] = s * vp + c * vq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = tid; idx < half * n; idx += T) {
        const int w = idx / n, col = idx % n;
        const int p = pq[w], q = pq[half + w];
        if (q >= n) continue;
        const float c = cs[w], s = cs[half + w];
        if (s == 0.f) continue;
        const float ap = A[p * n + col], aq = A[q * n + col];
        A[p * n + col] = c * ap - s * aq;
        A[q * n + col] = s * ap + c * aq;
      }
      __syncthreads();
      if (tid < half) {
        const int p = pq[tid], q = pq[half + tid];
        if (q < n && cs[half + tid] != 0.f) {
          A[p * n + q] = 0.f;
          A[q * n + p] = 0.f;
        }
      }
      __syncthreads();
    }
  }
  for (int idx = tid; idx < n * n; idx += T) V_out[idx] = (double)V[idx];
  if (tid == 0 && sweep >= max_sweeps) *flag = 2;
}

// One step of the FP64 refinement: from S = X^T A X and P = X^T X build
// lambda_i = S_ii / P_ii  [= S_ii / (1 - R_ii), R = I - P: Rayleigh quotients] and
// E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) (i != j, separated),
//      = R_ij / 2 otherwise,
// so that X <- X + X E.  One CTA (n <= 160).
__global__ void __launch_bounds__(1024) refine_e_kernel(const double* __restrict__ S,
                                                        const double* __restrict__ P,
                                                        const double* __restrict__ A, int n,
                                                        double* __restrict__ E,
                                                        double* __restrict__ lam_out) {
  extern __shared__ double dsm[];
  double* lam = dsm;  // n
  __shared__ double s_red[3][32];
  __shared__ double s_delta;
  const int tid = threadIdx.x, T = blockDim.x;
  for (int i = tid; i < n; i += T) lam[i] = S[i * n + i] / P[i * n + i];
  __syncthreads();
  // delta = 2 (||S - diag(lam)||_F + ||A||_F ||R||_F)
  double a = 0.0, b = 0.0, c = 0.0;
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx % n;
    const double sd = S[idx] - (i == j ? lam[i] : 0.0);
    const double rr = (i == j ? 1.0 : 0.0) - P[idx];
    a += sd * sd;
    b += A[idx] * A[idx];
    c += rr * rr;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((tid & 31) == 0) {
    s_red[0][tid >> 5] = a;
    s_red[1][tid >> 5] = b;
    s_red[2][tid >> 5] = c;
  }
  __syncthreads();
  if (tid == 0) {
    double x = 0.0, y = 0.0, z = 0.0;
    for (int w = 0; w < (T + 31) / 32; ++w) {
      x += s_red[0][w];
      y += s_red[1][w];
      z += s_red[2][w];
    }
    s_delta = 2.0 * (sqrt(x) + sqrt(y) * sqrt(z));
  }
  __syncthreads();
  const double delta = s_delta;
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx % n;
    const double rij = (i == j ? 1.0 : 0.0) - P[idx];
    double e;
    if (i == j) {
      e = 0.5 * rij;
    } else {
      const double gap = lam[j] - lam[i];
      e = (fabs(gap) > delta) ? (S[idx] + lam[j] * rij) / gap : 0.5 * rij;
    }
    E[idx] = e;
  }
  for (int i = tid; i < n; i += T) lam_out[i] = lam[i];
}

// Sort eigenpairs descending, fix signs (largest-magnitude entry positive).
__global__ void __launch_bounds__(1024) eig_finalize_kernel(const double* __restrict__ lam,
                                                            const double* __restrict__ X, int n,
                                                            double* __restrict__ evals,
                                                            double* __restrict__ evecs) {
  extern __shared__ int ism[];
  int* dest = ism;  // n
  const int tid = threadIdx.x, T = blockDim.x;
  for (int i = tid; i < n; i += T) {
    int rank = 0;
    for (int j = 0; j < n; ++j)
      if (lam[j] > lam[i] || (lam[j] == lam[i] && j < i)) ++rank;
    dest[i] = rank;
  }
  __syncthreads();
  for (int i = tid; i < n; i += T) {
    double best = 0.0;
    for (int r = 0; r < n; ++r) {
      const double v = X[r * n + i];
      if (fabs(v) > fabs(best)) best = v;
    }
    const double sgn = best < 0.0 ? -1.0 : 1.0;
    const int c = dest[i];
    evals[c] = lam[i];
    for (int r = 0; r < n; ++r) evecs[r * n + c] = sgn * X[r * n + i];
  }
}

__global__ void whitening_factors_kernel(const double* __restrict__ evals,
                                         const double* __restrict__ evecs, int64_t n, int64_t k,
                                         double* __restrict__ Cw, double* __restrict__ Cp,
                                         double* __restrict__ eig, int* __restrict__ flag) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < k) eig[idx] = evals[idx];
  if (idx == 0 && !(evals[k - 1] > 0.0)) *flag = 1;
  if (idx >= n * k) return;
  const int64_t r = idx / k, i = idx % k;
  const double l = evals[i];
  const double s = l > 0.0 ? sqrt(l) : 1.0;
  Cw[idx] = evecs[r * n + i] / s;
  Cp[idx] = evecs[r * n + i] * s;
}

__global__ void copy_f64_kernel(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

}  // namespace

otm_status gemm_tn_f64acc(const float* A, const float* B, int64_t rows, int64_t m, int64_t p,
                          double alpha, double* C, int accumulate, cudaStream_t st) {
  if (!accumulate) OTM_CHECK_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * m * p, st));
  if (rows == 0 || m == 0 || p == 0) return OTM_OK;
  const int64_t tiles = ((m + TN_T - 1) / TN_T) * ((p + TN_T - 1) / TN_T);
  int64_t splits = (2 * num_sms() + tiles - 1) / tiles;
  const int64_t max_splits = (rows + TN_R - 1) / TN_R;
  splits = splits < 1 ? 1 : (splits > max_splits ? max_splits : splits);
  int64_t rps = (rows + splits - 1) / splits;
  rps = (rps + TN_R - 1) / TN_R * TN_R;
  splits = (rows + rps - 1) / rps;
  dim3 grid((unsigned)((m + TN_T - 1) / TN_T), (unsigned)((p + TN_T - 1) / TN_T),
            (unsigned)splits);
  gemm_tn_kernel<<<grid, 256, 0, st>>>(A, B, rows, m, p, alpha, C, rps);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status gemm_nn_small(const float* A, int64_t rows, int64_t m, const double* C, int64_t p,
                         float* out, const double* r1_u, const double* r1_v, double r1_alpha,
                         cudaStream_t st) {
  if (p > NN_PMAX) return set_error(OTM_EINVAL, "gemm_nn_small: p=%lld > %d", (long long)p, NN_PMAX);
  if (rows == 0 || p == 0) return OTM_OK;
  gemm_nn_small_kernel<<<(unsigned)((rows + NN_R - 1) / NN_R), 256, 0, st>>>(
      A, rows, m, C, p, out, r1_u, r1_v, r1_alpha);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status gemm_nn_f64(const float* A, int64_t rows, int64_t m, const double* C, int64_t p,
                       double* out, cudaStream_t st) {
  if (rows == 0 || p == 0) return OTM_OK;
  dim3 grid((unsigned)((rows + D_R - 1) / D_R), (unsigned)((p + D_C - 1) / D_C));
  gemm_nn_f64_kernel<<<grid, 256, 0, st>>>(A, rows, m, C, p, out);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status dgemm_small(int ta, int tb, int64_t m, int64_t n, int64_t kk, double alpha,
                       const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                       double* C, int64_t ldc, cudaStream_t st) {
  if (m == 0 || n == 0) return OTM_OK;
  dim3 grid((unsigned)((n + 15) / 16), (unsigned)((m + 15) / 16));
  dgemm_small_kernel<<<grid, 256, 0, st>>>(ta, tb, m, n, kk, alpha, A, lda, B, ldb, beta, C, ldc);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status vec_tn(const double* u, const float* A, int64_t rows, int64_t m, double* out,
                  cudaStream_t st) {
  OTM_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * m, st));
  if (rows == 0 || m == 0) return OTM_OK;
  const int64_t rpb = 64;
  vec_tn_kernel<<<(unsigned)((rows + rpb - 1) / rpb), 128, 0, st>>>(u, A, rows, m, rpb, out);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

size_t orth_workspace(int64_t m) {
  WorkspaceSize w;
  w.add<double>(m * m).add<double>(m * m).add<int>(1);
  return w.bytes();
}

otm_status orthonormalize(float* A, int64_t rows, int64_t m, Workspace& ws, cudaStream_t st) {
  if (m > 160) return set_error(OTM_EINVAL, "orthonormalize: m=%lld > 160", (long long)m);
  if (rows < m) return set_error(OTM_EINVAL, "orthonormalize: rows < m");
  double* G = ws.take<double>(m * m);
  double* Rinv = ws.take<double>(m * m);
  int* flag = ws.take<int>(1);
  if (!G || !Rinv || !flag) return set_error(OTM_EINVAL, "orthonormalize: workspace too small");
  OTM_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  const size_t smem = 2 * sizeof(float) * m * m;
  OTM_CHECK_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  for (int pass = 0; pass < 3; ++pass) {
    OTM_TRY(gemm_tn_f64acc(A, A, rows, m, m, 1.0, G, 0, st));
    chol_inv_kernel<<<1, 1024, smem, st>>>(G, (int)m, pass == 0 ? 11.0 : 0.0, Rinv, flag);
    OTM_CHECK_LAUNCH();
    OTM_TRY(gemm_nn_small(A, rows, m, Rinv, m, A, nullptr, nullptr, 0.0, st));
  }
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h) return set_error(OTM_ENOTCONVERGED, "orthonormalize: Cholesky pivot failed");
  return OTM_OK;
}

size_t syev_workspace(int64_t n) {
  WorkspaceSize w;
  for (int i = 0; i < 6; ++i) w.add<double>(n * n);
  w.add<double>(n).add<int>(1);
  return w.bytes();
}

otm_status syev(const double* A, int64_t n, double* evals, double* evecs, Workspace& ws,
                cudaStream_t st) {
  if (n < 1 || n > 160) return set_error(OTM_EINVAL, "syev: n=%lld outside [1, 160]", (long long)n);
  double* X = ws.take<double>(n * n);
  double* Xn = ws.take<double>(n * n);
  double* AX = ws.take<double>(n * n);
  double* S = ws.take<double>(n * n);
  double* P = ws.take<double>(n * n);
  double* E = ws.take<double>(n * n);
  double* lam = ws.take<double>(n);
  int* flag = ws.take<int>(1);
  if (!flag) return set_error(OTM_EINVAL, "syev: workspace too small");
  OTM_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  const int np = (int)(n + (n & 1));
  const size_t smem = sizeof(float) * (2 * n * n + n + 2) + sizeof(int) * np + 16;
  OTM_CHECK_CUDA(cudaFuncSetAttribute(jacobi_f32_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  jacobi_f32_kernel<<<1, 1024, smem, st>>>(A, (int)n, 40, X, flag);
  OTM_CHECK_LAUNCH();
  const int iters = 3;
  for (int it = 0; it < iters; ++it) {
    // AX = A X, S = X^T (A X), P = X^T X   (A read symmetrically: A^T = A assumed after
    // symmetrisation; use (A + A^T)/2 X = 0.5 A X + 0.5 A^T X)
    OTM_TRY(dgemm_small(0, 0, n, n, n, 0.5, A, n, X, n, 0.0, AX, n, st));
    OTM_TRY(dgemm_small(1, 0, n, n, n, 0.5, A, n, X, n, 1.0, AX, n, st));
    OTM_TRY(dgemm_small(1, 0, n, n, n, 1.0, X, n, AX, n, 0.0, S, n, st));
    OTM_TRY(dgemm_small(1, 0, n, n, n, 1.0, X, n, X, n, 0.0, P, n, st));
    refine_e_kernel<<<1, 1024, sizeof(double) * n, st>>>(S, P, A, (int)n, E, lam);
    OTM_CHECK_LAUNCH();
    copy_f64_kernel<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(X, Xn, n * n);
    OTM_CHECK_LAUNCH();
    OTM_TRY(dgemm_small(0, 0, n, n, n, 1.0, X, n, E, n, 1.0, Xn, n, st));
    double* t = X;
    X = Xn;
    Xn = t;
  }
  eig_finalize_kernel<<<1, 256, sizeof(int) * n, st>>>(lam, X, (int)n, evals, evecs);
  OTM_CHECK_LAUNCH();
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h) return set_error(OTM_ENOTCONVERGED, "syev: Jacobi sweep limit reached");
  return OTM_OK;
}

otm_status whitening_factors(const double* evals, const double* evecs, int64_t n, int64_t k,
                             double* Cw, double* Cp, double* eig, int* flag, cudaStream_t st) {
  const int64_t tot = n * k > k ? n * k : k;
  whitening_factors_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(evals, evecs, n, k, Cw,
                                                                           Cp, eig, flag);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

}  // namespace otm
