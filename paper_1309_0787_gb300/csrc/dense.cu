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

#include "grid_sync.cuh"
#include "otm_internal.cuh"

namespace otm {
namespace {

// ---------------------------------------------------------------------------
// C (m x p, FP64) (+)= alpha * A^T B.  A: rows x m, B: rows x p (float32).
// Block: 64 x 64 output tile, 256 threads (4 x 4 consecutive rows and columns
// each, read from shared memory as float4).  Rows are split over
// gridDim.z (at least 256 rows per block); a block sums its rows in FP32 and
// adds its tile to C in FP64.
// ---------------------------------------------------------------------------
constexpr int TN_T = 64, TN_R = 32;

// Each thread stages 8 elements of A and 8 of B per 32-row slab: thread t
// covers slab rows rr = (t >> 4) + 16 q (q = 0, 1) and tile columns
// cc = 4 (t & 15) .. +3.  Loads for the next slab are issued into registers
// before the current slab is multiplied (software pipelining).
__device__ __forceinline__ void tn_load(const float* __restrict__ X, int64_t ld, int64_t r0,
                                        int64_t r_end, int64_t c0, int64_t cmax, int t,
                                        float (&v)[2][4]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int64_t r = r0 + (t >> 4) + 16 * q;
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      const int64_t c = c0 + 4 * (t & 15) + z;
      v[q][z] = (r < r_end && c < cmax) ? __ldg(X + r * ld + c) : 0.f;
    }
  }
}

__global__ void __launch_bounds__(256) gemm_tn_kernel(const float* __restrict__ A,
                                                      const float* __restrict__ B, int64_t rows,
                                                      int64_t m, int64_t p, double alpha,
                                                      double* __restrict__ C,
                                                      int64_t rows_per_split,
                                                      const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ __align__(16) float As[TN_R][TN_T];
  __shared__ __align__(16) float Bs[TN_R][TN_T];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * TN_T, j0 = (int64_t)blockIdx.y * TN_T;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t r_end = min(rows, r_begin + rows_per_split);
  // FP32 sums over this block's rows (<= a few hundred), FP64 across blocks
  float acc[4][4] = {};
  float va[2][4], vb[2][4];
  tn_load(A, m, r_begin, r_end, i0, m, t, va);
  tn_load(B, p, r_begin, r_end, j0, p, t, vb);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += TN_R) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      *reinterpret_cast<float4*>(&As[ty + 16 * q][4 * tx]) =
          make_float4(va[q][0], va[q][1], va[q][2], va[q][3]);
      *reinterpret_cast<float4*>(&Bs[ty + 16 * q][4 * tx]) =
          make_float4(vb[q][0], vb[q][1], vb[q][2], vb[q][3]);
    }
    __syncthreads();
    if (r0 + TN_R < r_end) {  // prefetch the next slab while this one is multiplied
      tn_load(A, m, r0 + TN_R, r_end, i0, m, t, va);
      tn_load(B, p, r0 + TN_R, r_end, j0, p, t, vb);
    }
#pragma unroll 8
    for (int rr = 0; rr < TN_R; ++rr) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[rr][4 * ty]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[rr][4 * tx]);
      const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t i = i0 + 4 * ty + x, j = j0 + 4 * tx + y;
      if (i < m && j < p) atomicAdd(&C[i * p + j], alpha * (double)acc[x][y]);
    }
}

// ---------------------------------------------------------------------------
// out (rows x p) = A (rows x m) * C (m x p, float32)
//                  - r1_alpha * r1_u[r] * r1_v[c]   (optional rank-one term)
// One block owns 32 whole rows (all p <= 256 columns), so A may alias out.
// Staging loads of a K-chunk are all issued into registers before they are
// stored to shared memory.
// ---------------------------------------------------------------------------
constexpr int NN_R = 32, NN_K = 32, NN_PMAX = 256;

__global__ void __launch_bounds__(256) gemm_nn_small_kernel(
    const float* A, int64_t rows, int64_t m, const float* __restrict__ C, int64_t p, float* out,
    const double* __restrict__ r1_u, const double* __restrict__ r1_v, double r1_alpha,
    const int* __restrict__ skip) {
  if (skip && *skip) return;
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
    float av[4], cv[4][NN_PMAX / 32];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t r = r0 + rg + 8 * q, k = k0 + cg;
      av[q] = (r < rows && k < m) ? A[r * m + k] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t k = k0 + rg + 8 * q;
#pragma unroll
      for (int j = 0; j < NN_PMAX / 32; ++j) {
        const int64_t c = cg + 32 * j;
        cv[q][j] = (j < ncj && k < m && c < p) ? __ldg(C + k * p + c) : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      As[rg + 8 * q][cg] = av[q];
#pragma unroll
      for (int j = 0; j < NN_PMAX / 32; ++j)
        if (j < ncj) Cs[rg + 8 * q][cg + 32 * j] = cv[q][j];
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

// The same product for m and p multiples of 4 and p <= 128 (the whitening's shapes):
// a CTA computes 32 rows x all p columns (so out may alias A), each thread a 4 x 4
// block read as float4 from K-major shared tiles, and the next 32-wide K chunk is
// loaded into registers while the current one is multiplied.
constexpr int T_R = 32, T_K = 32, T_P = 128;
__global__ void __launch_bounds__(256) gemm_nn_tile_kernel(
    const float* A, int64_t rows, int64_t m, const float* __restrict__ C, int64_t p, float* out,
    const double* __restrict__ r1_u, const double* __restrict__ r1_v, double r1_alpha,
    const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ __align__(16) float As[T_K][T_R + 4];  // As[kk][row]
  __shared__ __align__(16) float Cs[T_K][T_P + 4];  // Cs[kk][col]
  const int tid = threadIdx.x;
  const int ty = tid >> 5, tx = tid & 31;  // rows 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3
  const int64_t r0 = (int64_t)blockIdx.x * T_R;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const int ar = tid >> 3, ak = (tid & 7) * 4;  // A chunk: row ar, K columns ak .. ak + 3
  float4 ra, rc[4];
  auto load = [&](int64_t k0) {
    const int64_t gr = r0 + ar, gk = k0 + ak;
    ra = (gr < rows && gk < m) ? *reinterpret_cast<const float4*>(A + gr * m + gk) : zero;
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // C chunk: K row ck, columns c4 .. c4 + 3
      const int idx = tid + 256 * i, ck = idx >> 5, c4 = (idx & 31) * 4;
      const int64_t gc = k0 + ck;
      rc[i] = (gc < m && c4 < p) ? __ldg(reinterpret_cast<const float4*>(C + gc * p + c4)) : zero;
    }
  };
  float acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[q][j] = 0.f;
  load(0);
  for (int64_t k0 = 0; k0 < m; k0 += T_K) {
    As[ak][ar] = ra.x;
    As[ak + 1][ar] = ra.y;
    As[ak + 2][ar] = ra.z;
    As[ak + 3][ar] = ra.w;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + 256 * i;
      *reinterpret_cast<float4*>(&Cs[idx >> 5][(idx & 31) * 4]) = rc[i];
    }
    __syncthreads();
    if (k0 + T_K < m) load(k0 + T_K);
#pragma unroll 8
    for (int kk = 0; kk < T_K; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
      const float4 c = *reinterpret_cast<const float4*>(&Cs[kk][4 * tx]);
      const float av[4] = {a.x, a.y, a.z, a.w}, cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[q][j] = fmaf(av[q], cv[j], acc[q][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t r = r0 + 4 * ty + q;
    if (r >= rows) continue;
    const double u = r1_u ? r1_u[r] * r1_alpha : 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = 4 * tx + j;
      if (c < p) {
        float v = acc[q][j];
        if (r1_u) v = (float)((double)v - u * r1_v[c]);
        out[r * p + c] = v;
      }
    }
  }
}

// out (rows x p, FP64) = A (rows x m, float32) * C (m x p, FP64) to about 2^-48
// relative to sum_j |A[r][j] C[j][c]|, on the FP32 units (FP64 issues at 1/64 of
// the FP32 rate on this part).  Each C entry is split into two float32 terms,
// c = c_hi + c_lo (c_hi = fl32(c), c_lo = fl32(c - c_hi)); a * c_hi is formed
// exactly as the pair (p, e) with one FMA (Dekker's product, FMA form); a * c_lo
// is rounded (its error is 2^-24 of a term already 2^-24 below a * c).  The sum
// is a double-float (hi, lo): hi takes p by Knuth's branch-free TwoSum, whose
// rounding error joins lo together with e and a * c_lo, and (hi, lo) is
// renormalised by a second TwoSum after every term (cancellation can leave
// |lo| > |hi|).  The _rn intrinsics keep the compiler from contracting the
// product into the following add, which the exact-error steps rely on.  Tile:
// 64 rows x 32 columns per 256 threads, 8 rows per thread; the row of A is a
// shared-memory broadcast.
constexpr int D_R = 64, D_C = 32, D_K = 32;
__global__ void __launch_bounds__(256) gemm_nn_f64_kernel(const float* __restrict__ A,
                                                          int64_t rows, int64_t m,
                                                          const double* __restrict__ C,
                                                          int64_t p, double* __restrict__ out) {
  __shared__ float As[D_R][D_K + 1];
  __shared__ float Ch[D_K][D_C];
  __shared__ float Cl[D_K][D_C];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows per thread
  const int64_t r0 = (int64_t)blockIdx.x * D_R, c0 = (int64_t)blockIdx.y * D_C;
  float hi[8], lo[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) hi[q] = lo[q] = 0.f;
  for (int64_t k0 = 0; k0 < m; k0 += D_K) {
    for (int idx = threadIdx.x; idx < D_R * D_K; idx += 256) {
      const int rr = idx / D_K, kk = idx % D_K;
      As[rr][kk] = (r0 + rr < rows && k0 + kk < m) ? A[(r0 + rr) * m + k0 + kk] : 0.f;
    }
    for (int idx = threadIdx.x; idx < D_K * D_C; idx += 256) {
      const int kk = idx / D_C, cc = idx % D_C;
      const double c = (k0 + kk < m && c0 + cc < p) ? C[(k0 + kk) * p + c0 + cc] : 0.0;
      const float ch = (float)c;
      Ch[kk][cc] = ch;
      Cl[kk][cc] = (float)(c - (double)ch);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < D_K; ++kk) {
      const float ch = Ch[kk][tx], cl = Cl[kk][tx];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float a = As[ty * 8 + q][kk];
        const float pr = __fmul_rn(a, ch);
        const float e = fmaf(a, ch, -pr);  // a * ch = pr + e exactly
        const float s = __fadd_rn(hi[q], pr);  // TwoSum(hi, pr)
        const float bv = __fsub_rn(s, hi[q]);
        const float err = __fadd_rn(__fsub_rn(hi[q], __fsub_rn(s, bv)), __fsub_rn(pr, bv));
        const float l = __fadd_rn(lo[q], __fadd_rn(err, fmaf(a, cl, e)));
        const float h2 = __fadd_rn(s, l);      // TwoSum(s, l)
        const float b2 = __fsub_rn(h2, s);
        lo[q] = __fadd_rn(__fsub_rn(s, __fsub_rn(h2, b2)), __fsub_rn(l, b2));
        hi[q] = h2;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t r = r0 + ty * 8 + q, c = c0 + tx;
    if (r < rows && c < p) out[r * p + c] = (double)hi[q] + (double)lo[q];
  }
}

// Small FP64 GEMM, C = alpha op(A) op(B) + beta C, 8 x 8 tiles, one output
// per thread (many small blocks: the FP64 rate per SM is low, so the work is
// spread over as many SMs as possible).  A is m x kk (or kk x m when ta), B is
// kk x n (or n x kk when tb).
__global__ void __launch_bounds__(64) dgemm_small_kernel(int ta, int tb, int64_t m, int64_t n,
                                                         int64_t kk, double alpha,
                                                         const double* __restrict__ A,
                                                         int64_t lda,
                                                         const double* __restrict__ B,
                                                         int64_t ldb, double beta, double* C,
                                                         int64_t ldc) {
  constexpr int KC = 32;
  __shared__ double As[8][KC + 1];
  __shared__ double Bs[KC][9];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int64_t i = (int64_t)blockIdx.y * 8 + ty, j = (int64_t)blockIdx.x * 8 + tx;
  double acc = 0.0;
  for (int64_t k0 = 0; k0 < kk; k0 += KC) {
    double av[KC / 8], bv[KC / 8];
#pragma unroll
    for (int q = 0; q < KC / 8; ++q) {
      // A tile: row ii = blockIdx.y*8 + ty, k = k0 + tx + 8q ; B tile: k = k0 + ty + 8q, col jj
      const int64_t ka = k0 + tx + 8 * q, ii = (int64_t)blockIdx.y * 8 + ty;
      av[q] = (ii < m && ka < kk) ? (ta ? A[ka * lda + ii] : A[ii * lda + ka]) : 0.0;
      const int64_t kb = k0 + ty + 8 * q, jj = (int64_t)blockIdx.x * 8 + tx;
      bv[q] = (kb < kk && jj < n) ? (tb ? B[jj * ldb + kb] : B[kb * ldb + jj]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < KC / 8; ++q) {
      As[ty][tx + 8 * q] = av[q];
      Bs[ty + 8 * q][tx] = bv[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < KC; ++q) acc = fma(As[ty][q], Bs[q][tx], acc);
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
// One CTA of 1024 threads, FP32 in shared memory (n <= 160), right-looking
// and blocked by 8 columns, with L^{-1} built in the same sweep.  Block J:
//  (a) one warp factors the 8 x 8 diagonal block L_JJ in registers;
//  (b) the block row J of X = L^{-1} is finished: X_J = L_JJ^{-1} B_J by
//      forward substitution, where B starts as the identity and has taken the
//      updates of earlier blocks;
//  (c) the panel below, L_{>J,J} = A_{>J,J} L_JJ^{-T} (row by row by forward
//      substitution, in parallel with (b));
//  (d) every row i below takes one rank-8 update over its columns 0..i: the
//      trailing Cholesky matrix (columns past the block) and B (columns up to
//      the block), B_{i,:} -= L_{i,J} X_J.
// Look-ahead: while warps 1.. run (d), warp 0 updates and factors the next
// diagonal block, so two barriers per block column.  Output Rinv (n x n,
// float32, row-major, upper triangular) so that Q = A Rinv.
// shift_scale > 0 adds shift_scale * n * u * trace(G) to the diagonal
// (u = 2^-24), which keeps the factorisation positive definite for Gram
// matrices of ill-conditioned A (shifted Cholesky-QR: Fukaya, Kannan,
// Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 42, 2020).
// Pivots below 10 u trace(G) (numerically rank-deficient A) are raised to
// that floor: the matching columns of Q become normalised rounding noise,
// which the following passes orthonormalise -- still a valid orthonormal
// basis of a space containing range(A).  Only a non-finite pivot is an error.
// G is read from its lower triangle (it is the symmetric product A^T A).
// ---------------------------------------------------------------------------
constexpr int CH_T = 1024, CH_B = 8;

__host__ __device__ inline size_t chol_smem_floats(int n) {
  return (size_t)2 * n * (n | 1) + (size_t)(CH_B + 1) * n + CH_B * CH_B;
}

__global__ void __launch_bounds__(CH_T) chol_inv_kernel(const double* __restrict__ G, int n,
                                                        double shift_scale,
                                                        float* __restrict__ Rinv,
                                                        int* __restrict__ flag, int* skip,
                                                        float check_tol) {
  extern __shared__ float sm[];
  __shared__ float s_red[CH_T / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = CH_T / 32;
  // conditional pass: nothing to do once the columns are orthonormal to check_tol
  if (skip && *skip) return;
  if (check_tol > 0.f) {
    float dev = 0.f;
    for (int idx = tid; idx < n * n; idx += CH_T) {
      const int i = idx / n, j = idx % n;
      dev = fmaxf(dev, fabsf((float)G[idx] - (i == j ? 1.f : 0.f)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if (lane == 0) s_red[warp] = dev;
    __syncthreads();
    float mx = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) mx = fmaxf(mx, s_red[w]);
    if (mx <= check_tol) {
      if (tid == 0) *skip = 1;
      return;
    }
    __syncthreads();  // s_red is reused below
  }
  const int ldn = n | 1;         // odd row stride: column walks are bank-conflict free
  const int nblk = (n + CH_B - 1) / CH_B;
  float* L = sm;                 // n x ldn: G, then L (lower triangle)
  float* X = L + n * ldn;        // n x ldn: B, then X = L^{-1} (lower triangle)
  float* rdg = X + n * ldn;      // n reciprocal pivots 1 / L_jj
  float* PT = rdg + n;           // 8 x n: the current panel, transposed
  float* Ljj = PT + CH_B * n;    // 8 x 8 diagonal block
  __shared__ float s_shift, s_floor;
  __shared__ int s_bad;
  if (warp == 0) {
    double tr = 0.0;
    for (int i = lane; i < n; i += 32) tr += G[(int64_t)i * n + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (lane == 0) {
      s_shift = (float)(shift_scale * (double)n * 5.9604644775390625e-8 * tr);
      s_floor = (float)(10.0 * 5.9604644775390625e-8 * tr) + 1e-30f;
      s_bad = 0;
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int idx = tid; idx < n * n; idx += CH_T) {
    const int i = idx / n, j = idx % n;
    if (j <= i) {
      float v = (float)G[idx];
      if (i == j) v += s_shift;
      L[i * ldn + j] = v;
    }
    X[i * ldn + j] = i == j ? 1.f : 0.f;
  }
  __syncthreads();

  // (a) factor the diagonal block starting at j0 in warp 0: lane r holds row
  // j0 + r in a[] (already updated); writes L, Ljj and the reciprocal pivots
  auto factor_diag = [&](int j0, float (&a)[CH_B]) {
    const int jb = min(CH_B, n - j0);
#pragma unroll
    for (int c = 0; c < CH_B; ++c) {
      if (c < jb) {
        float d = __shfl_sync(0xffffffffu, a[c], c);
        if (!isfinite(d)) {
          if (lane == 0) s_bad = 1;
          d = 1.f;
        }
        const float pinv = rsqrtf(fmaxf(d, s_floor));
        if (lane == c) {
          a[c] = fmaxf(d, s_floor) * pinv;
          rdg[j0 + c] = pinv;
        }
        if (lane > c) a[c] *= pinv;
#pragma unroll
        for (int kk = c + 1; kk < CH_B; ++kk) {
          const float lkc = __shfl_sync(0xffffffffu, a[c], kk);
          if (kk < jb && lane >= kk && lane < jb) a[kk] -= a[c] * lkc;
        }
      }
    }
    if (lane < CH_B) {
#pragma unroll
      for (int c = 0; c < CH_B; ++c) {
        const float v = (lane < jb && c <= lane) ? a[c] : 0.f;
        Ljj[lane * CH_B + c] = v;
        if (lane < jb && c <= lane) L[(j0 + lane) * ldn + j0 + c] = v;
      }
    }
  };
  if (warp == 0) {
    float a[CH_B];
#pragma unroll
    for (int c = 0; c < CH_B; ++c) a[c] = (lane < min(CH_B, n) && c <= lane) ? L[lane * ldn + c] : 0.f;
    factor_diag(0, a);
  }
  __syncthreads();

  for (int J = 0; J < nblk; ++J) {
    const int j0 = J * CH_B, jb = min(CH_B, n - j0), je = j0 + jb;
    // (b) block row J of X = L_JJ^{-1} B_J by forward substitution: threads
    // [0, je) take one column each
    if (tid < je) {
      const int c = tid;
      float x[CH_B];
#pragma unroll
      for (int r = 0; r < CH_B; ++r) {
        if (r < jb) {
          float v = X[(j0 + r) * ldn + c];
#pragma unroll
          for (int m = 0; m < r; ++m) v = fmaf(-Ljj[r * CH_B + m], x[m], v);
          x[r] = v * rdg[j0 + r];
        }
      }
#pragma unroll
      for (int r = 0; r < CH_B; ++r)
        if (r < jb) X[(j0 + r) * ldn + c] = x[r];
    }
    // (c) panel rows i >= je, l L_JJ^T = a by forward substitution: threads
    // [CH_T/2, ...) take one row each
    {
      const int i = je + (tid - CH_T / 2);
      if (tid >= CH_T / 2 && i < n) {
        float l[CH_B];
#pragma unroll
        for (int c = 0; c < CH_B; ++c) {
          float v = c < jb ? L[i * ldn + j0 + c] : 0.f;
#pragma unroll
          for (int m = 0; m < c; ++m) v = fmaf(-l[m], Ljj[c * CH_B + m], v);
          l[c] = c < jb ? v * rdg[j0 + c] : 0.f;
          if (c < jb) L[i * ldn + j0 + c] = l[c];
          PT[c * n + i] = l[c];
        }
      }
    }
    __syncthreads();
    // (d) rank-8 update of rows i >= je over columns 0..i: B for columns < je,
    // the trailing Cholesky matrix for columns je..i.  Look-ahead: warp 0
    // updates the next diagonal block (rows and columns je .. je + 7) and
    // factors it at once; warps 1.. update everything else.
    const int je2 = min(je + CH_B, n);
    if (warp == 0) {
      if (je < n) {
        float a[CH_B];
        const int i = je + lane;
#pragma unroll
        for (int c = 0; c < CH_B; ++c) {
          float acc = 0.f;
          if (i < je2 && c <= lane) {
            acc = L[i * ldn + je + c];
#pragma unroll
            for (int m = 0; m < CH_B; ++m) acc = fmaf(-PT[m * n + i], PT[m * n + je + c], acc);
          }
          a[c] = acc;
        }
        factor_diag(je, a);
      }
    } else {
      for (int i = je + warp - 1; i < n; i += NW - 1) {
        float li[CH_B];
#pragma unroll
        for (int m = 0; m < CH_B; ++m) li[m] = PT[m * n + i];
        // columns je .. min(i, je2 - 1) of rows in the next diagonal block are warp 0's
        const int c_skip_hi = i < je2 ? i : je - 1;
        for (int c = lane; c <= i; c += 32) {
          if (c < je) {
            float acc = X[i * ldn + c];
#pragma unroll
            for (int m = 0; m < CH_B; ++m)
              if (m < jb) acc = fmaf(-li[m], X[(j0 + m) * ldn + c], acc);
            X[i * ldn + c] = acc;
          } else if (c > c_skip_hi || c >= je2) {
            float acc = L[i * ldn + c];
#pragma unroll
            for (int m = 0; m < CH_B; ++m) acc = fmaf(-li[m], PT[m * n + c], acc);
            L[i * ldn + c] = acc;
          }
        }
      }
    }
    __syncthreads();
  }
  // Rinv = (L^T)^{-1} = (L^{-1})^T, zero below the diagonal
  for (int i = warp; i < n; i += NW)
    for (int j = lane; j < n; j += 32)
      Rinv[(int64_t)i * n + j] = j >= i ? X[j * ldn + i] : 0.f;
  if (tid == 0 && s_bad) *flag = 1;
}

// ---------------------------------------------------------------------------
// FP32 starting eigenvectors for the FP64 refinement, one CTA of 1024 threads
// (n <= 160), all in shared memory:
//  1. Householder reduction to tridiagonal form T = H^T A H (classical
//     two-sided reflections v, tau; eight threads per row for p = tau A v, a
//     warp per row and lanes over columns for the rank-2 update; the next
//     column's norm is summed during the update, so two barriers per column);
//  2. every eigenvalue of T by multisection on Sturm counts (G threads per
//     eigenvalue);
//  3. eigenvectors of T from twisted factorisations (the forward LDL^T and
//     backward UDU^T factorisations of T - lambda I, twisted where the
//     diagonal of the twisted factorisation is smallest; Parlett & Dhillon,
//     "Relatively robust representations of symmetric tridiagonals", 2000),
//     one thread per eigenvector, Gram-Schmidt inside groups of eigenvalues
//     closer than 1e-4 ||T||;
//  4. back-transformation X = H Z by blocks of 8 reflectors in compact WY
//     form, eight threads per four columns (no barriers between blocks).
// Output: X (n x n FP64, row-major, column i = eigenvector i, eigenvalues
// ascending).  fac: 2 n^2 floats of global scratch for the factorisations.
// ---------------------------------------------------------------------------
constexpr int TE_T = 1024;
constexpr int TE_CW = 5;  // columns per lane, rows per warp in the rank-2 update (n <= 160)

static_assert(TE_T == 32 * 32, "block sums read one partial per lane");

// Sum of v over the block (every thread gets it); one barrier.
__device__ __forceinline__ float block_sum_f(float v, float* red, int tid) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  float t = red[tid & 31];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

__global__ void __launch_bounds__(TE_T) tridiag_eig_kernel(const double* __restrict__ A0, int n,
                                                           double* __restrict__ X_out,
                                                           float* __restrict__ fac) {
  extern __shared__ float sm[];
  const int ldn = n | 1;
  float* Ah = sm;               // n x ldn: the matrix, then the reflectors (column j, rows > j)
  float* Z = Ah + n * ldn;      // n x ldn: eigenvectors of T, then of A
  float* d = Z + n * ldn;       // n  diagonal of T
  float* e = d + n;             // n  off-diagonal of T (e[j] couples j and j+1)
  float* tau = e + n;           // n
  float* P = tau + n;           // n  p = tau A v
  float* lam = P + n;           // n  eigenvalues of T (ascending)
  float* Tw = lam + n;          // 64 per block of 8 reflectors: T_b of the compact WY form
  __shared__ float red[2][TE_T / 32];
  __shared__ float s_alpha, s_tau, s_v0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = TE_T / 32;
  // A0 is symmetric (the caller symmetrises it): coalesced row-major reads
#pragma unroll 4
  for (int idx = tid; idx < n * n; idx += TE_T) Ah[(idx / n) * ldn + idx % n] = (float)A0[idx];
  __syncthreads();

  // 1. Householder tridiagonalisation
  __shared__ float s_sig[NW];  // per-warp squares of the next column, from the update
  for (int j = 0; j + 2 < n; ++j) {
    const int r0 = j + 1;  // first row of the column part x = A[r0:, j]
    float sigma;
    if (j == 0) {
      float part = 0.f;
      for (int r = r0 + tid; r < n; r += TE_T) part += Ah[r * ldn + j] * Ah[r * ldn + j];
      sigma = block_sum_f(part, red[0], tid);
    } else {
      sigma = s_sig[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sigma += __shfl_xor_sync(0xffffffffu, sigma, o);
    }
    const float x0 = Ah[r0 * ldn + j];
    float alpha, tj, v0;
    if (sigma <= 1e-36f) {
      alpha = x0;
      tj = 0.f;
      v0 = 0.f;
    } else {
      // fast square root and reciprocal (a few ulp): this is a float32 start
      // for the FP64 refinement, and tau stays consistent with v
      alpha = -copysignf(sigma * rsqrtf(sigma), x0);
      v0 = x0 - alpha;
      tj = __fdividef(1.f, sigma - x0 * alpha);  // 2 / (v^T v), v^T v = 2 (sigma - x0 alpha)
    }
    // p = tau A_trail v (eight threads per trailing row, interleaved columns,
    // two accumulators each), and p^T v
    float pv = 0.f;
    for (int base = r0; base < n; base += TE_T >> 3) {  // trip count uniform per block
      const int i = base + (tid >> 3);
      const int sub = tid & 7;
      float a0 = 0.f, a1 = 0.f;
      if (i < n) {
        int c = r0 + sub;
        if (sub == 0) {
          a0 = Ah[i * ldn + r0] * v0;
          c += 8;
        }
        for (; c + 8 < n; c += 16) {
          a0 = fmaf(Ah[i * ldn + c], Ah[c * ldn + j], a0);
          a1 = fmaf(Ah[i * ldn + c + 8], Ah[(c + 8) * ldn + j], a1);
        }
        if (c < n) a0 = fmaf(Ah[i * ldn + c], Ah[c * ldn + j], a0);
      }
      float acc = a0 + a1;
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      if (i < n && sub == 0) {
        const float pi = tj * acc;
        P[i] = pi;
        pv = fmaf(pi, i == r0 ? v0 : Ah[i * ldn + j], pv);
      }
    }
    const float ptv = block_sum_f(pv, red[1], tid);  // includes a barrier: P complete
    const float K = 0.5f * tj * ptv;
    // A_trail -= v w^T + w v^T, w = p - K v; the squares of the updated column
    // r0 below its diagonal are the next step's sigma
    float sq = 0.f;
    float vcs[TE_CW], wcs[TE_CW];  // v_c, w_c of this lane's columns c = r0 + lane + 32 t
#pragma unroll
    for (int t = 0; t < TE_CW; ++t) {
      const int c = r0 + lane + 32 * t;
      const float vc = c < n ? (c == r0 ? v0 : Ah[c * ldn + j]) : 0.f;
      vcs[t] = vc;
      wcs[t] = c < n ? P[c] - K * vc : 0.f;
    }
#pragma unroll
    for (int t2 = 0; t2 < TE_CW; ++t2) {
      const int i = r0 + warp + NW * t2;
      if (i < n) {
        const float vi = i == r0 ? v0 : Ah[i * ldn + j];
        const float wi = P[i] - K * vi;
#pragma unroll
        for (int t = 0; t < TE_CW; ++t) {
          const int c = r0 + lane + 32 * t;
          if (c < n) {
            const float nv = Ah[i * ldn + c] - (vi * wcs[t] + wi * vcs[t]);
            Ah[i * ldn + c] = nv;
            if (t == 0 && lane == 0 && i > r0) sq = fmaf(nv, nv, sq);
          }
        }
      }
    }
    if (lane == 0) s_sig[warp] = sq;  // column r0 is handled by lane 0 only
    if (tid == 0) {
      d[j] = Ah[j * ldn + j];
      e[j] = alpha;
      tau[j] = tj;
    }
    __syncthreads();
    if (tid == 0) Ah[r0 * ldn + j] = v0;  // reflector kept in place for step 4
  }
  __syncthreads();
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = Ah[(n - 2) * ldn + n - 2];
      e[n - 2] = Ah[(n - 1) * ldn + n - 2];
    }
    d[n - 1] = Ah[(n - 1) * ldn + n - 1];
    e[n - 1] = 0.f;
  }
  __syncthreads();

  // 2. bisection: thread i finds the i-th smallest eigenvalue.  Gershgorin
  // bounds per warp (lanes over rows, shuffle min / max); e2 = e^2 (in P).
  float* e2 = P;
  for (int k = tid; k < n; k += TE_T) e2[k] = e[k] * e[k];
  float tnorm = 0.f, glo = 3.0e38f, ghi = -3.0e38f;
  for (int k = lane; k < n; k += 32) {
    const float off = (k > 0 ? fabsf(e[k - 1]) : 0.f) + (k + 1 < n ? fabsf(e[k]) : 0.f);
    glo = fminf(glo, d[k] - off);
    ghi = fmaxf(ghi, d[k] + off);
    tnorm = fmaxf(tnorm, fabsf(d[k]) + off);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    tnorm = fmaxf(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  }
  __syncthreads();  // e2 complete
  const float pad = 1e-6f * tnorm + 1e-30f;
  glo -= pad;
  ghi += pad;
  const float piv_min = 1e-30f + 1e-12f * tnorm;
  // multisection: G lanes per eigenvalue evaluate the Sturm count at G interior
  // points of the current interval, which then shrinks by G + 1 (13 rounds of
  // 5 for G = 4: below 2^-28 of the Gershgorin range)
  // (the Sturm counts are bound by the reciprocal unit's throughput, so the
  // fewer evaluations of G = 4 beat the fewer rounds of G = 8)
  const int G = 4;
  const int rounds = 13;
  if ((warp * 32) / G < n) {  // warps holding at least one eigenvalue (ballots are warp-wide)
    const int i = tid / G, sub = tid % G;
    const int gbase = (lane / G) * G;  // first lane of this eigenvalue's group
    float lo = glo, hi = ghi;
    for (int it = 0; it < rounds; ++it) {
      const float w = (hi - lo) / (float)(G + 1);
      const float x = lo + w * (float)(sub + 1);
      int cnt = 0;
      float q = d[0] - x;
      if (fabsf(q) < piv_min) q = -piv_min;
      cnt += q < 0.f;
      for (int k = 1; k < n; ++k) {
        q = d[k] - x - __fdividef(e2[k - 1], q);
        if (fabsf(q) < piv_min) q = -piv_min;
        cnt += q < 0.f;
      }
      // first interior point with more than i eigenvalues below it
      const unsigned m = (__ballot_sync(0xffffffffu, cnt > i) >> gbase) & ((1u << G) - 1u);
      const int first = m ? __ffs(m) - 1 : G;
      const float nlo = lo + w * (float)first;
      hi = first < G ? lo + w * (float)(first + 1) : hi;
      lo = nlo;
    }
    if (i < n && sub == 0) lam[i] = 0.5f * (lo + hi);
  }
  __syncthreads();

  // 3. eigenvectors of T by twisted factorisation (thread per eigenvector).
  // The forward pivots Dp go to this thread's column of Z (and to global
  // scratch for the regeneration below); the backward pivots Dm to global
  // scratch, with the twist index found in the same backward pass.
  if (tid < n) {
    const float mu = lam[tid];
    float* Dpg = fac;                     // [k * n + tid]
    float* Dm = fac + (int64_t)n * n;
    float q = d[0] - mu;
    if (fabsf(q) < piv_min) q = piv_min;
    Z[tid] = q;
    Dpg[tid] = q;
    for (int k = 1; k < n; ++k) {
      q = d[k] - mu - __fdividef(e2[k - 1], q);
      if (fabsf(q) < piv_min) q = piv_min;
      Z[k * ldn + tid] = q;
      Dpg[(int64_t)k * n + tid] = q;
    }
    q = d[n - 1] - mu;
    if (fabsf(q) < piv_min) q = piv_min;
    Dm[(int64_t)(n - 1) * n + tid] = q;
    int rt = n - 1;
    float best = fabsf(Z[(n - 1) * ldn + tid] + q - (d[n - 1] - mu));
    for (int k = n - 2; k >= 0; --k) {
      q = d[k] - mu - __fdividef(e2[k], q);
      if (fabsf(q) < piv_min) q = piv_min;
      Dm[(int64_t)k * n + tid] = q;
      const float g = fabsf(Z[k * ldn + tid] + q - (d[k] - mu));
      if (g <= best) {  // ties go to the smaller index
        best = g;
        rt = k;
      }
    }
    float z = 1.f, nrm = 1.f;
    for (int k = rt - 1; k >= 0; --k) {
      z = -__fdividef(e[k], Z[k * ldn + tid]) * z;  // Dp_k, then overwritten by z
      Z[k * ldn + tid] = z;
      nrm = fmaf(z, z, nrm);
    }
    Z[rt * ldn + tid] = 1.f;
    z = 1.f;
    for (int k = rt + 1; k < n; ++k) {
      z = -__fdividef(e[k - 1], Dm[(int64_t)k * n + tid]) * z;
      Z[k * ldn + tid] = z;
      nrm = fmaf(z, z, nrm);
    }
    const float inv = rsqrtf(nrm);
    for (int k = 0; k < n; ++k) Z[k * ldn + tid] *= inv;
  }
  __syncthreads();
  // Gram-Schmidt inside groups of close eigenvalues (warp 0; groups are rare).
  // A repeated eigenvalue makes the twisted factorisation return the same
  // vector for every member; when Gram-Schmidt leaves less than half of a
  // vector, it is regenerated by two inverse-iteration solves with the stored
  // LDL^T factors of T - lambda I from a fixed pseudo-random start, and
  // orthogonalised again.
  if (warp == 0) {
    const float ctol = 1e-4f * tnorm;
    for (int i = 1; i < n; ++i) {
      int j0 = i - 1;
      if (lam[i] - lam[j0] > ctol) continue;
      while (j0 > 0 && lam[i] - lam[j0 - 1] <= ctol) --j0;
      for (int attempt = 0; attempt < 2; ++attempt) {
        for (int jj = j0; jj < i; ++jj) {
          float dot = 0.f;
          for (int k = lane; k < n; k += 32) dot = fmaf(Z[k * ldn + jj], Z[k * ldn + i], dot);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
          for (int k = lane; k < n; k += 32) Z[k * ldn + i] -= dot * Z[k * ldn + jj];
          __syncwarp();
        }
        float nn = 0.f;
        for (int k = lane; k < n; k += 32) nn = fmaf(Z[k * ldn + i], Z[k * ldn + i], nn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        if (nn > 0.25f || attempt == 1) {
          const float inv = nn > 0.f ? rsqrtf(nn) : 0.f;
          for (int k = lane; k < n; k += 32) Z[k * ldn + i] *= inv;
          __syncwarp();
          break;
        }
        // regenerate: x = (L D L^T)^{-2} r, L D L^T = T - lambda_i I (forward factors of column i)
        if (lane == 0) {
          const float* Dp = fac;
          for (int k = 0; k < n; ++k)
            Z[k * ldn + i] = sinf(12.9898f * (float)(k + 1) + 78.233f * (float)(i + 1));
          for (int rep = 0; rep < 2; ++rep) {
            float y = Z[i];  // row 0
            for (int k = 1; k < n; ++k) {
              const float lk = e[k - 1] / Dp[(int64_t)(k - 1) * n + i];
              y = Z[k * ldn + i] - lk * y;
              Z[k * ldn + i] = y;
            }
            for (int k = 0; k < n; ++k) Z[k * ldn + i] /= Dp[(int64_t)k * n + i];
            float x = Z[(n - 1) * ldn + i], sq = x * x;
            for (int k = n - 2; k >= 0; --k) {
              const float lk = e[k] / Dp[(int64_t)k * n + i];
              x = Z[k * ldn + i] - lk * x;
              Z[k * ldn + i] = x;
              sq = fmaf(x, x, sq);
            }
            const float inv = sq > 0.f ? rsqrtf(sq) : 0.f;
            for (int k = 0; k < n; ++k) Z[k * ldn + i] *= inv;
          }
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();

  // 4. back-transformation X = H_0 ... H_{n-3} Z in blocks of 8 reflectors:
  // H_{8b} ... H_{8b+7} = I - V_b T_b V_b^T (compact WY form, T_b upper
  // triangular: Schreiber & Van Loan, SIAM J. Sci. Stat. Comput. 10, 1989),
  // blocks applied last to first as Z -= V_b (T_b (V_b^T Z)).  Reflector j
  // is column j of Ah below the diagonal (rows > j).
  const int nr = n >= 3 ? n - 2 : 0;
  const int nb = (nr + 7) / 8;
  // keep only the reflectors in Ah (entries below the diagonal of columns < nr)
  for (int idx = tid; idx < n * n; idx += TE_T) {
    const int r = idx / n, c = idx % n;
    if (c >= nr || r <= c) Ah[r * ldn + c] = 0.f;
  }
  __syncthreads();
  // (i) T_b[r][i] holds v_r^T v_i (r < i) ...
  for (int pidx = warp; pidx < nb * 28; pidx += NW) {
    const int b = pidx / 28, pr = pidx % 28;
    int a = 0, c = pr;  // pair (a, c), a < c, row-major over the strict upper triangle
    while (c >= 7 - a) {
      c -= 7 - a;
      ++a;
    }
    c += a + 1;
    const int ja = 8 * b + a, jc = 8 * b + c;
    float dot = 0.f;
    if (jc < nr)
      for (int r = jc + 1 + lane; r < n; r += 32) dot = fmaf(Ah[r * ldn + ja], Ah[r * ldn + jc], dot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if (lane == 0) Tw[b * 64 + a * 8 + c] = dot;
  }
  __syncthreads();
  // ... (ii) then T_b itself, one thread per block (columns in order, rows ascending)
  if (tid < nb) {
    float* T = Tw + tid * 64;
    for (int i = 0; i < 8; ++i) {
      const int ji = 8 * tid + i;
      const float ti = ji < nr ? tau[ji] : 0.f;
      // T[m][i] (m < i) still holds v_m^T v_i where row r reads it: rows ascend
      for (int r = 0; r < i; ++r) {
        float acc = 0.f;
        for (int m = r; m < i; ++m) acc = fmaf(T[r * 8 + m], T[m * 8 + i], acc);
        T[r * 8 + i] = -ti * acc;
      }
      T[i * 8 + i] = ti;
      for (int r = i + 1; r < 8; ++r) T[r * 8 + i] = 0.f;
    }
  }
  __syncthreads();
  // (iii) 8 threads (rows interleaved by 8) per group of 4 columns c = cbase +
  // g + 32 q, so that each reflector entry loaded serves four columns; 256
  // threads; columns are independent, so no barriers
  if (tid < 256) {
    constexpr int CPT = 4;
    const int sub = tid & 7, g = tid >> 3;
    for (int cbase = 0; cbase < n; cbase += 32 * CPT) {
      for (int b = nb - 1; b >= 0; --b) {
        const int j0 = 8 * b, cnt = min(8, nr - j0);  // reflectors in this block
        const float* T = Tw + b * 64;
        float w[CPT][8];
#pragma unroll
        for (int q = 0; q < CPT; ++q)
#pragma unroll
          for (int m = 0; m < 8; ++m) w[q][m] = 0.f;
        // first row of this thread's interleave that is > j0
        const int rs = j0 + 1 + ((sub - (j0 + 1)) & 7);
        for (int r = rs; r < n; r += 8) {
          float v[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) v[m] = m < cnt ? Ah[r * ldn + j0 + m] : 0.f;
#pragma unroll
          for (int q = 0; q < CPT; ++q) {
            const int c = cbase + g + 32 * q;
            const float z = c < n ? Z[r * ldn + c] : 0.f;
#pragma unroll
            for (int m = 0; m < 8; ++m) w[q][m] = fmaf(v[m], z, w[q][m]);
          }
        }
#pragma unroll
        for (int q = 0; q < CPT; ++q)
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            w[q][m] += __shfl_xor_sync(0xffffffffu, w[q][m], 1);
            w[q][m] += __shfl_xor_sync(0xffffffffu, w[q][m], 2);
            w[q][m] += __shfl_xor_sync(0xffffffffu, w[q][m], 4);
          }
        // y = T w in place (row r of T reads w[m] for m >= r only)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
          for (int q = 0; q < CPT; ++q) {
            float acc = 0.f;
#pragma unroll
            for (int m = r; m < 8; ++m) acc = fmaf(T[r * 8 + m], w[q][m], acc);
            w[q][r] = acc;
          }
        }
        for (int r = rs; r < n; r += 8) {
          float v[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) v[m] = m < cnt ? Ah[r * ldn + j0 + m] : 0.f;
#pragma unroll
          for (int q = 0; q < CPT; ++q) {
            const int c = cbase + g + 32 * q;
            if (c < n) {
              float z = Z[r * ldn + c];
#pragma unroll
              for (int m = 0; m < 8; ++m) z = fmaf(-v[m], w[q][m], z);
              Z[r * ldn + c] = z;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  for (int i = warp; i < n; i += NW)
    for (int j = lane; j < n; j += 32) X_out[(int64_t)i * n + j] = (double)Z[i * ldn + j];
}

// ---------------------------------------------------------------------------
// FP64 refinement of the float32 eigenvectors (Ogita & Aishima, "Iterative
// refinement for symmetric eigenvalue decomposition", Japan J. Indust. Appl.
// Math. 35, 2018), one cooperative kernel over the whole GPU.  Per iteration:
//   AX = A X;  S = X^T AX,  P = X^T X  (R = I - P);
//   lambda_i = S_ii / P_ii,
//   delta = 2 (||S - diag(S)||_F + ||A||_F ||R||_F);
//   E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) where
//          |lambda_j - lambda_i| > delta, else R_ij / 2 (clusters, diagonal);
//   X <- X + X E,
// stopping once max |E_ij| <= REFINE_TOL (the next correction would be of
// order REFINE_TOL^2 ||A|| / gap, below FP64 rounding) or after REFINE_MAX
// iterations.  The eigenvalues are the last Rayleigh quotients; the pairs are
// then sorted descending and each vector signed so that its largest-magnitude
// entry is positive.  The FP64 products are spread over every SM (output
// tiles whose operand rows / columns are staged in shared memory, the k range
// split over the CTA's warps; S and P only on the upper block triangle);
// phases are separated by a grid barrier whose wait is bounded (on time-out
// the kernel sets the failure flag and returns).  Data written inside the
// kernel is read with L2 loads (__ldcg).
// ---------------------------------------------------------------------------
constexpr int RF_T = 256;
constexpr int REFINE_MAX = 8;
constexpr double REFINE_TOL = 1e-10;
constexpr int RF_MAX_GRID = 1024;  // per-CTA partial slots per quantity
constexpr int RF_NMAX = 160;
constexpr int PT_COLS = (RF_NMAX * 8 + RF_T - 1) / RF_T;  // panel entries per thread (n x 8)
constexpr int PT_ROWS = (RF_NMAX * 4 + RF_T - 1) / RF_T;  // (4 x n)

struct RefineArgs {
  const double* A;   // n x n symmetric
  double* X;         // n x n: the starting vectors
  double* Xn;        // n x n scratch
  double* AX;        // n x n scratch: A X, kept up to date as X changes
  double* AXn;       // n x n scratch
  double* S;         // n x n scratch
  double* P;         // n x n scratch
  double* E;         // n x n scratch
  double* lam;       // n
  double* part;      // 4 x RF_MAX_GRID per-CTA partials: ||A||^2, ||S - diag S||^2, ||R||^2, max|E|
  unsigned* bar;     // barrier counter (zero on entry)
  int* flag;         // 2: non-finite eigenvalue; 3: barrier time-out
  double* evals;     // n, descending
  double* evecs;     // n x n, column i = eigenvector i
  int n;
};

// Sum (is_max: maximum) of v over the block, to every thread.
__device__ __forceinline__ double block_reduce_d(double v, double* red, bool is_max) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, u) : v + u;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = red[0];
#pragma unroll
  for (int w = 1; w < RF_T / 32; ++w) t = is_max ? fmax(t, red[w]) : t + red[w];
  return t;
}

// Sum (is_max: maximum) of the per-CTA partials slot[0, gridDim.x), reduced by
// every warp in the same order (so every CTA gets the same value); the first
// 256 partials are loaded at once.
__device__ __forceinline__ double grid_total(const double* slot, bool is_max) {
  const int lane = threadIdx.x & 31, G = (int)gridDim.x;
  double v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = lane + 32 * q < G ? __ldcg(slot + lane + 32 * q) : 0.0;
  double t = v[0];
#pragma unroll
  for (int q = 1; q < 8; ++q) t = is_max ? fmax(t, v[q]) : t + v[q];
  for (int b = lane + 256; b < G; b += 32) {
    const double u = __ldcg(slot + b);
    t = is_max ? fmax(t, u) : t + u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, t, o);
    t = is_max ? fmax(t, u) : t + u;
  }
  return t;
}

// Operand staging: every load of a panel is issued before its stores, so a
// panel costs one L2 round trip.
struct Cols8 {  // columns [c0, c0 + 8) of an n x n matrix as n x 8
  double v[PT_COLS];
};
struct Rows4 {  // rows [r0, r0 + 4) as 4 x n
  double v[PT_ROWS];
};
__device__ __forceinline__ void load_cols8(Cols8& p, const double* M, int c0, int n) {
#pragma unroll
  for (int t = 0; t < PT_COLS; ++t) {
    const int idx = threadIdx.x + t * RF_T, k = idx >> 3, c = idx & 7;
    p.v[t] = (k < n && c0 + c < n) ? __ldcg(M + k * n + c0 + c) : 0.0;
  }
}
__device__ __forceinline__ void store_cols8(double* dst, const Cols8& p, int n) {
#pragma unroll
  for (int t = 0; t < PT_COLS; ++t) {
    const int idx = threadIdx.x + t * RF_T;
    if (idx < n * 8) dst[idx] = p.v[t];
  }
}
__device__ __forceinline__ void load_rows4(Rows4& p, const double* M, int r0, int n) {
#pragma unroll
  for (int t = 0; t < PT_ROWS; ++t) {
    const int idx = threadIdx.x + t * RF_T, r = idx / n, k = idx % n;
    p.v[t] = (r < 4 && r0 + r < n) ? __ldcg(M + (r0 + r) * n + k) : 0.0;
  }
}
__device__ __forceinline__ void store_rows4(double* dst, const Rows4& p, int n) {
#pragma unroll
  for (int t = 0; t < PT_ROWS; ++t) {
    const int idx = threadIdx.x + t * RF_T;
    if (idx < 4 * n) dst[idx] = p.v[t];
  }
}

// C[i][j] = (Add ? Add[i][j] : 0) + sum_k L[i][k] R[k][j] over 4 x 8 output
// tiles, and when L2 is given also C2 = L2 + L2 R (same R): a tile's 4 rows of
// L (and L2) and 8 columns of R are staged in shared memory, the k range is
// split over 8 warps and the partial sums added by warp 0.
__device__ void gemm_tiles_4x8(const double* L, const double* R, const double* Add, double* C,
                               const double* L2, double* C2, int n, double* sm) {
  const int ntr = (n + 3) / 4, ntc = (n + 7) / 8, items = ntr * ntc;
  double* sl = sm;            // 4 x n
  double* sl2 = sl + 4 * n;   // 4 x n
  double* sr = sl2 + 4 * n;   // n x 8
  double* part = sr + 8 * n;  // 8 x 32 x 2
  const int ks = threadIdx.x >> 5, o = threadIdx.x & 31, ty = o >> 3, tx = o & 7;
  const bool two = L2 != nullptr;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int i0 = (item / ntc) * 4, j0 = (item % ntc) * 8;
    Rows4 pl, pl2;
    Cols8 pr;
    load_rows4(pl, L, i0, n);
    if (two) load_rows4(pl2, L2, i0, n);
    load_cols8(pr, R, j0, n);
    store_rows4(sl, pl, n);
    if (two) store_rows4(sl2, pl2, n);
    store_cols8(sr, pr, n);
    __syncthreads();
    double acc = 0.0, acc2 = 0.0;
    if (two) {
      for (int k = ks; k < n; k += 8) {
        const double r = sr[k * 8 + tx];
        acc = fma(sl[ty * n + k], r, acc);
        acc2 = fma(sl2[ty * n + k], r, acc2);
      }
    } else {
      for (int k = ks; k < n; k += 8) acc = fma(sl[ty * n + k], sr[k * 8 + tx], acc);
    }
    part[(ks * 32 + o) * 2] = acc;
    part[(ks * 32 + o) * 2 + 1] = acc2;
    __syncthreads();
    if (ks == 0) {
      double t = 0.0, t2 = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        t += part[(q * 32 + o) * 2];
        t2 += part[(q * 32 + o) * 2 + 1];
      }
      const int i = i0 + ty, j = j0 + tx;
      if (i < n && j < n) {
        C[i * n + j] = (Add ? __ldcg(Add + i * n + j) : 0.0) + t;
        if (two) C2[i * n + j] = __ldcg(L2 + i * n + j) + t2;
      }
    }
    __syncthreads();  // shared buffers are reused by the next item
  }
}

__global__ void __launch_bounds__(RF_T) refine_kernel(RefineArgs a) {
  extern __shared__ double rsm[];
  __shared__ double red[RF_T / 32];
  const int n = a.n;
  const int tid = threadIdx.x;
  const int gtid = blockIdx.x * RF_T + tid, gthreads = gridDim.x * RF_T;
  double* pA2 = a.part;
  double* pS = a.part + RF_MAX_GRID;
  double* pR = a.part + 2 * RF_MAX_GRID;
  double* pE = a.part + 3 * RF_MAX_GRID;
  // ||A||_F^2
  {
    double v = 0.0;
    for (int idx = gtid; idx < n * n; idx += gthreads) v = fma(a.A[idx], a.A[idx], v);
    const double t = block_reduce_d(v, red, false);
    if (tid == 0) pA2[blockIdx.x] = t;
  }
  double* X = a.X;
  double* Xn = a.Xn;
  double* AX = a.AX;
  double* AXn = a.AXn;
  const int nb8 = (n + 7) / 8, npairs = nb8 * (nb8 + 1) / 2;
  gemm_tiles_4x8(a.A, X, nullptr, AX, nullptr, nullptr, n, rsm);  // AX = A X
  if (!grid_barrier(a.bar, a.flag, 3)) return;
  for (int it = 0; it < REFINE_MAX; ++it) {
    // S = X^T AX and P = X^T X on the upper block triangle (both symmetric),
    // lambda, and the two norms
    double s_off = 0.0, r2 = 0.0;
    {
      double* xi = rsm;          // n x 8: X columns of block bi
      double* axj = xi + 8 * n;  // n x 8: AX columns of block bj
      double* xj = axj + 8 * n;  // n x 8: X columns of block bj
      double* part = xj + 8 * n; // 4 x 64 x 2
      const int ks = tid >> 6, o = tid & 63, ty = o >> 3, tx = o & 7;
      for (int item = blockIdx.x; item < npairs; item += gridDim.x) {
        int bi = 0, rem = item;  // item -> (bi, bj), bi <= bj, row-major
        while (rem >= nb8 - bi) {
          rem -= nb8 - bi;
          ++bi;
        }
        const int bj = bi + rem;
        Cols8 p1, p2, p3;
        load_cols8(p1, X, 8 * bi, n);
        load_cols8(p2, AX, 8 * bj, n);
        load_cols8(p3, X, 8 * bj, n);
        store_cols8(xi, p1, n);
        store_cols8(axj, p2, n);
        store_cols8(xj, p3, n);
        __syncthreads();
        double sv = 0.0, pv = 0.0;
        for (int k = ks; k < n; k += 4) {
          const double x = xi[k * 8 + ty];
          sv = fma(x, axj[k * 8 + tx], sv);
          pv = fma(x, xj[k * 8 + tx], pv);
        }
        part[(ks * 64 + o) * 2] = sv;
        part[(ks * 64 + o) * 2 + 1] = pv;
        __syncthreads();
        if (ks == 0) {
          double st = 0.0, pt = 0.0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            st += part[(q * 64 + o) * 2];
            pt += part[(q * 64 + o) * 2 + 1];
          }
          const int i = 8 * bi + ty, j = 8 * bj + tx;
          if (i < n && j < n) {
            a.S[i * n + j] = st;
            a.P[i * n + j] = pt;
            const double w = bi == bj ? 1.0 : 2.0;  // mirrored entries count twice
            const double rr = (i == j ? 1.0 : 0.0) - pt;
            r2 = fma(w * rr, rr, r2);
            if (i != j) s_off = fma(w * st, st, s_off);
            else a.lam[i] = st / pt;
            if (bi != bj) {
              a.S[j * n + i] = st;
              a.P[j * n + i] = pt;
            }
          }
        }
        __syncthreads();
      }
    }
    {
      const double t1 = block_reduce_d(s_off, red, false);
      const double t2 = block_reduce_d(r2, red, false);
      if (tid == 0) {
        pS[blockIdx.x] = t1;
        pR[blockIdx.x] = t2;
      }
    }
    if (!grid_barrier(a.bar, a.flag, 3)) return;
    // E and its largest entry
    {
      const double ts = grid_total(pS, false), ta = grid_total(pA2, false),
                   tr = grid_total(pR, false);
      const double delta = 2.0 * (sqrt(ts) + sqrt(ta) * sqrt(tr));
      double mx = 0.0;
      for (int idx = gtid; idx < n * n; idx += gthreads) {
        const int i = idx / n, j = idx % n;
        const double rij = (i == j ? 1.0 : 0.0) - __ldcg(a.P + idx);
        double e = 0.5 * rij;
        if (i != j) {
          const double lj = __ldcg(a.lam + j), gap = lj - __ldcg(a.lam + i);
          if (fabs(gap) > delta) e = (__ldcg(a.S + idx) + lj * rij) / gap;
        }
        a.E[idx] = e;
        mx = fmax(mx, fabs(e));
      }
      const double t = block_reduce_d(mx, red, true);
      if (tid == 0) pE[blockIdx.x] = t;
    }
    if (!grid_barrier(a.bar, a.flag, 3)) return;
    // X <- X + X E, and AX <- AX + (AX) E = A X for the next iteration (not
    // needed after the last one)
    const bool last = grid_total(pE, true) <= REFINE_TOL;
    gemm_tiles_4x8(X, a.E, X, Xn, last ? nullptr : AX, AXn, n, rsm);
    if (!grid_barrier(a.bar, a.flag, 3)) return;
    double* t = X;
    X = Xn;
    Xn = t;
    t = AX;
    AX = AXn;
    AXn = t;
    if (last) break;
  }
  // sort descending, fix signs: one warp per eigenpair
  const int lane = tid & 31;
  for (int i = gtid >> 5; i < n; i += gthreads >> 5) {
    const double li = __ldcg(a.lam + i);
    int rank = 0;
    double best = 0.0;
    for (int j = lane; j < n; j += 32) {
      const double lj = __ldcg(a.lam + j);
      if (lj > li || (lj == li && j < i)) ++rank;
      const double v = __ldcg(X + j * n + i);
      if (fabs(v) > fabs(best)) best = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rank += __shfl_xor_sync(0xffffffffu, rank, o);
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      if (fabs(ob) > fabs(best) || (fabs(ob) == fabs(best) && ob > best)) best = ob;
    }
    const double sgn = best < 0.0 ? -1.0 : 1.0;
    if (lane == 0) {
      a.evals[rank] = li;
      if (!isfinite(li)) atomicExch(a.flag, 2);  // non-finite input or breakdown
    }
    for (int r = lane; r < n; r += 32) a.evecs[r * n + rank] = sgn * __ldcg(X + r * n + i);
  }
}

__global__ void whitening_factors_kernel(const double* __restrict__ evals,
                                         const double* __restrict__ evecs, int64_t n, int64_t k,
                                         double* __restrict__ Cw, double* __restrict__ Cp,
                                         double* __restrict__ eig, int* __restrict__ flag,
                                         float* __restrict__ Cw32) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < k) eig[idx] = evals[idx];
  // the k-th eigenvalue must be positive and resolvable above the float32
  // accuracy of the range finder that produced the matrix
  if (idx == 0 && !(evals[k - 1] > 1e-5 * fabs(evals[0]))) *flag = 1;
  if (idx >= n * k) return;
  const int64_t r = idx / k, i = idx % k;
  const double l = evals[i];
  const double s = l > 0.0 ? sqrt(l) : 1.0;
  Cw[idx] = evecs[r * n + i] / s;
  Cp[idx] = evecs[r * n + i] * s;
  if (Cw32) Cw32[idx] = (float)(evecs[r * n + i] / s);
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
                          double alpha, double* C, int accumulate, cudaStream_t st,
                          const int* skip) {
  if (!accumulate) OTM_CHECK_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * m * p, st));
  if (rows == 0 || m == 0 || p == 0) return OTM_OK;
  // about two blocks per SM, but at least 128 rows per block: every block adds
  // its tile to C with FP64 atomics, so fewer, longer splits mean less contention
  const int64_t tiles = ((m + TN_T - 1) / TN_T) * ((p + TN_T - 1) / TN_T);
  int64_t splits = (2 * num_sms() + tiles - 1) / tiles;
  const int64_t max_splits = (rows + 127) / 128;
  splits = splits < 1 ? 1 : (splits > max_splits ? max_splits : splits);
  int64_t rps = (rows + splits - 1) / splits;
  rps = (rps + TN_R - 1) / TN_R * TN_R;
  splits = (rows + rps - 1) / rps;
  dim3 grid((unsigned)((m + TN_T - 1) / TN_T), (unsigned)((p + TN_T - 1) / TN_T),
            (unsigned)splits);
  gemm_tn_kernel<<<grid, 256, 0, st>>>(A, B, rows, m, p, alpha, C, rps, skip);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status gemm_nn_small(const float* A, int64_t rows, int64_t m, const float* C, int64_t p,
                         float* out, const double* r1_u, const double* r1_v, double r1_alpha,
                         cudaStream_t st, const int* skip) {
  if (p > NN_PMAX) return set_error(OTM_EINVAL, "gemm_nn_small: p=%lld > %d", (long long)p, NN_PMAX);
  if (rows == 0 || p == 0) return OTM_OK;
  const bool a16 = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(C)) & 15u) == 0;
  if (m % 4 == 0 && p % 4 == 0 && p <= T_P && m >= 1 && a16) {
    gemm_nn_tile_kernel<<<(unsigned)((rows + T_R - 1) / T_R), 256, 0, st>>>(
        A, rows, m, C, p, out, r1_u, r1_v, r1_alpha, skip);
  } else {
    gemm_nn_small_kernel<<<(unsigned)((rows + NN_R - 1) / NN_R), 256, 0, st>>>(
        A, rows, m, C, p, out, r1_u, r1_v, r1_alpha, skip);
  }
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
  dim3 grid((unsigned)((n + 7) / 8), (unsigned)((m + 7) / 8));
  dgemm_small_kernel<<<grid, 64, 0, st>>>(ta, tb, m, n, kk, alpha, A, lda, B, ldb, beta, C, ldc);
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
  w.add<double>(m * m).add<float>(m * m).add<int>(1);
  return w.bytes();
}

otm_status orthonormalize(float* A, int64_t rows, int64_t m, Workspace& ws, cudaStream_t st,
                          int* dflag, int passes) {
  if (m > 160) return set_error(OTM_EINVAL, "orthonormalize: m=%lld > 160", (long long)m);
  if (rows < m) return set_error(OTM_EINVAL, "orthonormalize: rows < m");
  double* G = ws.take<double>(m * m);
  float* Rinv = ws.take<float>(m * m);
  int* skip = ws.take<int>(1);
  if (!G || !Rinv || !skip) return set_error(OTM_EINVAL, "orthonormalize: workspace too small");
  const size_t smem = sizeof(float) * chol_smem_floats((int)m);
  OTM_CHECK_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  OTM_CHECK_CUDA(cudaMemsetAsync(skip, 0, sizeof(int), st));
  // pass 0: shifted (ill-conditioned input); pass 1: plain Cholesky-QR; passes
  // 2-3 run only while the columns are not yet orthonormal to 1e-5 (the test
  // and the skip happen on the device, without a host round trip)
  for (int pass = 0; pass < passes; ++pass) {
    const int* sk = pass >= 2 ? skip : nullptr;
    OTM_TRY(gemm_tn_f64acc(A, A, rows, m, m, 1.0, G, 0, st, sk));
    chol_inv_kernel<<<1, CH_T, smem, st>>>(G, (int)m, pass == 0 ? 11.0 : 0.0, Rinv, dflag,
                                           pass >= 2 ? skip : nullptr, pass >= 2 ? 1e-5f : 0.f);
    OTM_CHECK_LAUNCH();
    OTM_TRY(gemm_nn_small(A, rows, m, Rinv, m, A, nullptr, nullptr, 0.0, st, sk));
  }
  return OTM_OK;
}

// One CTA per SM (the cooperative launch needs every CTA resident), at most
// RF_MAX_GRID.
unsigned refine_grid() {
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (sms[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? (v < RF_MAX_GRID ? v : RF_MAX_GRID) : 1;
  }
  return (unsigned)sms[dev];
}

size_t syev_workspace(int64_t n) {
  WorkspaceSize w;
  for (int i = 0; i < 8; ++i) w.add<double>(n * n);
  w.add<double>(n).add<double>(4 * RF_MAX_GRID);
  w.add<unsigned>(1).add<float>(2 * n * n);
  return w.bytes();
}

__global__ void symmetrize_kernel(const double* __restrict__ A, int64_t n, double* __restrict__ B) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  B[idx] = 0.5 * (A[i * n + j] + A[j * n + i]);
}

otm_status syev(const double* A_in, int64_t n, double* evals, double* evecs, Workspace& ws,
                cudaStream_t st, int* dflag) {
  if (n < 1 || n > 160) return set_error(OTM_EINVAL, "syev: n=%lld outside [1, 160]", (long long)n);
  double* A = ws.take<double>(n * n);
  double* X = ws.take<double>(n * n);
  double* Xn = ws.take<double>(n * n);
  double* AX = ws.take<double>(n * n);
  double* AXn = ws.take<double>(n * n);
  double* S = ws.take<double>(n * n);
  double* P = ws.take<double>(n * n);
  double* E = ws.take<double>(n * n);
  double* lam = ws.take<double>(n);
  double* part = ws.take<double>(4 * RF_MAX_GRID);
  unsigned* bar = ws.take<unsigned>(1);
  float* fac = ws.take<float>(2 * n * n);
  if (!fac) return set_error(OTM_EINVAL, "syev: workspace too small");
  const unsigned nb = (unsigned)((n * n + 255) / 256);
  symmetrize_kernel<<<nb, 256, 0, st>>>(A_in, n, A);
  OTM_CHECK_LAUNCH();
  const int64_t ldn = n | 1;
  const size_t smem = sizeof(float) * (2 * n * ldn + 5 * n + 64 * ((n + 5) / 8));
  OTM_CHECK_CUDA(cudaFuncSetAttribute(tridiag_eig_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tridiag_eig_kernel<<<1, TE_T, smem, st>>>(A, (int)n, X, fac);
  OTM_CHECK_LAUNCH();
  // FP64 refinement: quadratic convergence from the float32 eigenvectors
  RefineArgs ra{A, X, Xn, AX, AXn, S, P, E, lam, part, bar, dflag, evals, evecs, (int)n};
  OTM_CHECK_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
  void* kargs[] = {&ra};
  const size_t rsmem = sizeof(double) * (24 * n + 4 * 64 * 2);  // the largest phase (S, P)
  OTM_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)refine_kernel, dim3(refine_grid()),
                                             dim3(RF_T), kargs, rsmem, st));
  count_launch();
  return OTM_OK;
}

otm_status whitening_factors(const double* evals, const double* evecs, int64_t n, int64_t k,
                             double* Cw, double* Cp, double* eig, int* flag, cudaStream_t st,
                             float* Cw32) {
  const int64_t tot = n * k > k ? n * k : k;
  whitening_factors_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(evals, evecs, n, k, Cw,
                                                                           Cp, eig, flag, Cw32);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

otm_status f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t st) {
  if (n <= 0) return OTM_OK;
  f64_to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

}  // namespace otm
