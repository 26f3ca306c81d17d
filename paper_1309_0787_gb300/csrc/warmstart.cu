// Learned warm start for the STGD (not in the paper): instance generation,
// tensor sketches, the MLP's training and inference, Gram-Schmidt and the
// scaling of the initial components.
//
// Sketch of the whitened tensor of Section 3.2 (symmetric views), for a unit
// direction theta:
//   S = T(I, I, theta) = c1 P - c2 <theta, ybar> Q - c2 (m ybar^T + ybar m^T)
//                        + c3 <theta, ybar> ybar ybar^T,
//   Q = (1/n) Y^T Y,  P = (1/n) Y^T diag(Y theta) Y,  m = Q theta,
// with c1, c2, c3 the Dirichlet coefficients of Lemma 3.  Q and the P_j of all
// directions are one batched tensor-core GEMM per instance: Y^T times the
// stacked [Y^T; Y^T diag(p_1); ...] (BF16 operands, FP32 accumulation).
//
// Network (row-major weights): x -> GELU(W1 x + b1) -> GELU(W2 h1 + b2) ->
// W3 h2 + b3, read as the k x k matrix M (row-major) whose columns are
// orthonormalised by Gram-Schmidt.  Dense products run on the tcgen05 GEMM
// (gemm_tc.cu); the rest are the small kernels below.
#include <cmath>
#include <mutex>

#include <cuda_bf16.h>

#include "otm_internal.cuh"

namespace otm {
namespace {

constexpr int WS_KMAX = 64;  // largest k of the warm-start kernels

// ---------------------------------------------------------------------------
// Counter-based generator: Philox4x32-10 (Salmon et al., SC 2011)
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// uniform strictly inside (0, 1): ((x >> 9) + 0.5) * 2^-23, exact in float32
__device__ __forceinline__ float unit01(uint32_t x) {
  return __fmul_rn(__fadd_rn(__uint2float_rn(x >> 9), 0.5f), 1.1920928955078125e-07f);
}

constexpr int GAMMA_ATTEMPTS = 16;

// log of a Gamma(a, 1) draw: Marsaglia & Tsang (ACM TOMS 2000) with the a < 1
// boost G(a) = G(a + 1) U^(1/a).  Counter (t, c, instance, attempt).
__device__ float log_gamma_draw(float a, uint32_t t, uint32_t c, uint32_t inst, uint32_t k0,
                                uint32_t k1) {
  const bool small = a < 1.f;
  const float ab = small ? __fadd_rn(a, 1.f) : a;
  const float d = __fsub_rn(ab, 1.f / 3.f);
  const float cc = __fdiv_rn(1.f, __fsqrt_rn(__fmul_rn(9.f, d)));
  float logg = logf(d);
  float boost_u = 0.5f;
  for (int att = 0; att < GAMMA_ATTEMPTS; ++att) {
    const U4 r = philox(t, c, inst, (uint32_t)att, k0, k1);
    if (att == 0) boost_u = unit01(r.w);
    const float u1 = unit01(r.x), u2 = unit01(r.y);
    const float x = __fmul_rn(__fsqrt_rn(__fmul_rn(-2.f, logf(u1))),
                              cosf(__fmul_rn(6.2831855f, u2)));
    const float v = __fadd_rn(1.f, __fmul_rn(cc, x));
    if (v > 0.f) {
      const float v3 = __fmul_rn(__fmul_rn(v, v), v);
      const float lv3 = logf(v3);
      const float rhs = __fadd_rn(
          __fsub_rn(__fadd_rn(__fmul_rn(__fmul_rn(0.5f, x), x), d), __fmul_rn(d, v3)),
          __fmul_rn(d, lv3));
      if (logf(unit01(r.z)) < rhs) {
        logg = __fadd_rn(logf(d), lv3);
        break;
      }
    }
  }
  if (small) logg = __fadd_rn(logg, __fdiv_rn(logf(boost_u), a));
  return logg;
}

// y_t = m h_t, h_t ~ Dir(alpha): one warp per sample, lane owns components
// (and rows) lane + 32 q.  grid (sample blocks, instances).
constexpr int GEN_WARPS = 8;
constexpr int GEN_SAMPLES = 64;  // samples per block

__global__ void __launch_bounds__(GEN_WARPS * 32) ws_generate_kernel(
    const float* __restrict__ m, const float* __restrict__ alpha, int64_t n, int k, uint32_t k0,
    uint32_t k1, int64_t first, float* __restrict__ Y) {
  __shared__ float sm[WS_KMAX * (WS_KMAX + 1)];
  __shared__ float sa[WS_KMAX];
  const int inst = blockIdx.y;
  const float* mi = m + (int64_t)inst * k * k;
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) sm[(i / k) * (k + 1) + i % k] = mi[i];
  for (int i = threadIdx.x; i < k; i += blockDim.x) sa[i] = alpha[(int64_t)inst * k + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t gi = (uint32_t)(first + inst);
  for (int s = warp; s < GEN_SAMPLES; s += GEN_WARPS) {
    const int64_t t = (int64_t)blockIdx.x * GEN_SAMPLES + s;
    if (t >= n) break;
    float L[2];
    float mx = -INFINITY;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = lane + 32 * q;
      L[q] = c < k ? log_gamma_draw(sa[c], (uint32_t)t, (uint32_t)c, gi, k0, k1) : -INFINITY;
      mx = fmaxf(mx, L[q]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float e[2], sum = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = lane + 32 * q;
      e[q] = c < k ? expf(__fsub_rn(L[q], mx)) : 0.f;
      sum += e[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    float h[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) h[q] = __fdiv_rn(e[q], sum);
    float y[2] = {0.f, 0.f};
    for (int c = 0; c < k; ++c) {
      const float hc = __shfl_sync(0xffffffffu, h[c >> 5], c & 31);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int a = lane + 32 * q;
        if (a < k) y[q] = __fadd_rn(y[q], __fmul_rn(hc, sm[a * (k + 1) + c]));
      }
    }
    float* yr = Y + ((int64_t)inst * n + t) * k;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int a = lane + 32 * q;
      if (a < k) yr[a] = y[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Sketches
// ---------------------------------------------------------------------------
constexpr int SK_TS = 64;  // samples per block of the operand preparation

// From Y (instances x n x k): At = Y^T (k x ldn, BF16), Bt = [Y^T; Y^T diag(p_1);
// ...; Y^T diag(p_J)] ((J+1) k x ldn), p_j = Y theta_j, zero beyond n; and the
// per-block column sums of Y.  grid (ceil(ldn / SK_TS), instances).
__global__ void __launch_bounds__(256) ws_sketch_prep_kernel(
    const float* __restrict__ Y, int64_t n, int k, int64_t ldn, const float* __restrict__ thetas,
    int J, __nv_bfloat16* __restrict__ At, __nv_bfloat16* __restrict__ Bt,
    float* __restrict__ psum) {
  __shared__ float ys[SK_TS][WS_KMAX + 1];
  __shared__ float th[4][WS_KMAX];
  __shared__ float p[4][SK_TS];
  const int inst = blockIdx.y, tid = threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.x * SK_TS;
  const float* Yi = Y + (int64_t)inst * n * k;
  for (int i = tid; i < SK_TS * k; i += 256) {
    const int s = i / k, a = i % k;
    const int64_t t = t0 + s;
    ys[s][a] = t < n ? Yi[t * k + a] : 0.f;
  }
  for (int i = tid; i < J * k; i += 256) th[i / k][i % k] = thetas[i];
  __syncthreads();
  for (int i = tid; i < J * SK_TS; i += 256) {
    const int j = i / SK_TS, s = i % SK_TS;
    float acc = 0.f;
    for (int a = 0; a < k; ++a) acc = fmaf(ys[s][a], th[j][a], acc);
    p[j][s] = acc;
  }
  if (tid < k) {
    float acc = 0.f;
    for (int s = 0; s < SK_TS; ++s) acc += ys[s][tid];
    psum[((int64_t)inst * gridDim.x + blockIdx.x) * k + tid] = acc;
  }
  __syncthreads();
  __nv_bfloat16* Ai = At + (int64_t)inst * k * ldn;
  __nv_bfloat16* Bi = Bt + (int64_t)inst * (J + 1) * k * ldn;
  for (int i = tid; i < k * SK_TS; i += 256) {
    const int a = i / SK_TS, s = i % SK_TS;
    const int64_t t = t0 + s;
    if (t >= ldn) continue;
    const float v = ys[s][a];
    Ai[(int64_t)a * ldn + t] = __float2bfloat16_rn(v);
    Bi[(int64_t)a * ldn + t] = __float2bfloat16_rn(v);
    for (int j = 0; j < J; ++j)
      Bi[((int64_t)(j + 1) * k + a) * ldn + t] = __float2bfloat16_rn(v * p[j][s]);
  }
}

// S_j from C = At Bt^T (k x (J+1) k per instance) and the column sums; also the
// network input x = vec(S) scaled to unit root-mean-square (BF16).  One block
// per instance.
__global__ void __launch_bounds__(256) ws_sketch_combine_kernel(
    const float* __restrict__ C, const float* __restrict__ psum, int nblk, int64_t n, int k, int J,
    const double* __restrict__ alpha0, const float* __restrict__ thetas, float* __restrict__ S,
    __nv_bfloat16* __restrict__ x16) {
  __shared__ float yb[WS_KMAX];
  __shared__ float mj[4][WS_KMAX];
  __shared__ float ty[4];
  __shared__ double red[8];
  const int inst = blockIdx.x, tid = threadIdx.x, ldc = (J + 1) * k;
  const float* Ci = C + (int64_t)inst * k * ldc;
  const float inv_n = 1.f / (float)n;
  if (tid < k) {
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += psum[((int64_t)inst * nblk + b) * k + tid];
    yb[tid] = (float)(acc / (double)n);
  }
  __syncthreads();
  for (int i = tid; i < J * k; i += 256) {
    const int j = i / k, a = i % k;
    float acc = 0.f;
    for (int b = 0; b < k; ++b) acc = fmaf(Ci[(int64_t)a * ldc + b], thetas[j * k + b], acc);
    mj[j][a] = acc * inv_n;
  }
  if (tid < J) {
    float acc = 0.f;
    for (int a = 0; a < k; ++a) acc = fmaf(thetas[tid * k + a], yb[a], acc);
    ty[tid] = acc;
  }
  __syncthreads();
  const double a0 = alpha0[inst];
  const float c1 = (float)((a0 + 1.0) * (a0 + 2.0) / 2.0), c2 = (float)(a0 * (a0 + 1.0) / 2.0),
              c3 = (float)(a0 * a0);
  const int tot = J * k * k;
  double ss = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    float scale = 1.f;
    if (pass == 1) {
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if ((tid & 31) == 0) red[tid >> 5] = ss;
      __syncthreads();
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      scale = t > 0.0 ? (float)sqrt((double)tot / t) : 0.f;
    }
    for (int e = tid; e < tot; e += 256) {
      const int j = e / (k * k), a = (e / k) % k, b = e % k;
      const float q = Ci[(int64_t)a * ldc + b] * inv_n;
      const float pj = Ci[(int64_t)a * ldc + (j + 1) * k + b] * inv_n;
      const float s = c1 * pj - c2 * ty[j] * q - c2 * (mj[j][a] * yb[b] + yb[a] * mj[j][b]) +
                      c3 * ty[j] * yb[a] * yb[b];
      if (pass == 0) {
        ss += (double)s * s;
        if (S) S[(int64_t)inst * tot + e] = s;
      } else {
        x16[(int64_t)inst * tot + e] = __float2bfloat16_rn(s * scale);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Initial components: v_i = sign(t_i) (|t_i| / kappa)^(1/3) u_i with
// t_i = T(u_i, u_i, u_i) = c1 E[(y.u)^3] - 3 c2 E[(y.u)^2] (ybar.u) + c3 (ybar.u)^3.
// ---------------------------------------------------------------------------
constexpr int IC_TS = 64;  // samples per block

// partial sums of (y.u_i), (y.u_i)^2, (y.u_i)^3.  grid (blocks, instances),
// block 256 = 4 sample lanes x 64 components.
__global__ void __launch_bounds__(256) ws_init_partial_kernel(
    const float* __restrict__ U0, const float* __restrict__ Y, int64_t n, int k,
    double* __restrict__ part) {
  __shared__ float us[WS_KMAX][WS_KMAX + 1];
  __shared__ float ys[IC_TS][WS_KMAX + 1];
  __shared__ double red[4][3][WS_KMAX];
  const int inst = blockIdx.y, tid = threadIdx.x;
  const float* Ui = U0 + (int64_t)inst * k * k;
  for (int i = tid; i < k * k; i += 256) us[i / k][i % k] = Ui[i];
  const int64_t t0 = (int64_t)blockIdx.x * IC_TS;
  const float* Yi = Y + (int64_t)inst * n * k;
  for (int i = tid; i < IC_TS * k; i += 256) {
    const int s = i / k, a = i % k;
    ys[s][a] = t0 + s < n ? Yi[(t0 + s) * k + a] : 0.f;
  }
  __syncthreads();
  const int comp = tid & 63, lane4 = tid >> 6;
  double s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (comp < k) {
    for (int s = lane4; s < IC_TS; s += 4) {
      if (t0 + s >= n) break;
      float d = 0.f;
      for (int a = 0; a < k; ++a) d = fmaf(ys[s][a], us[a][comp], d);
      s1 += d;
      s2 += (double)d * d;
      s3 += (double)d * d * d;
    }
  }
  red[lane4][0][comp] = s1;
  red[lane4][1][comp] = s2;
  red[lane4][2][comp] = s3;
  __syncthreads();
  if (tid < 3 * k) {
    const int w = tid / k, c = tid % k;
    const double v = red[0][w][c] + red[1][w][c] + red[2][w][c] + red[3][w][c];
    part[(((int64_t)inst * gridDim.x + blockIdx.x) * 3 + w) * k + c] = v;
  }
}

// V0 (instances x k x k, component i contiguous) from the partial sums.
__global__ void ws_init_final_kernel(const float* __restrict__ U0, const double* __restrict__ part,
                                     int nblk, int64_t n, int k, const double* __restrict__ alpha0,
                                     double kappa, float* __restrict__ V0) {
  const int inst = blockIdx.x;
  __shared__ float scl[WS_KMAX];
  if (threadIdx.x < k) {
    const int c = threadIdx.x;
    double s1 = 0, s2 = 0, s3 = 0;
    for (int b = 0; b < nblk; ++b) {
      const double* pb = part + ((int64_t)inst * nblk + b) * 3 * k;
      s1 += pb[c];
      s2 += pb[k + c];
      s3 += pb[2 * k + c];
    }
    const double a0 = alpha0[inst];
    const double c1 = (a0 + 1) * (a0 + 2) / 2, c2 = a0 * (a0 + 1) / 2, c3 = a0 * a0;
    const double mu = s1 / (double)n;
    const double t = c1 * s3 / (double)n - 3 * c2 * (s2 / (double)n) * mu + c3 * mu * mu * mu;
    const double mag = cbrt(fabs(t) / kappa);
    scl[c] = (float)(t < 0 ? -mag : mag);
  }
  __syncthreads();
  const float* Ui = U0 + (int64_t)inst * k * k;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, a = e % k;  // V0[i][a] = scl_i U0[a][i]
    V0[(int64_t)inst * k * k + e] = scl[i] * Ui[(int64_t)a * k + i];
  }
}

// ---------------------------------------------------------------------------
// Gram-Schmidt (classical, applied twice per column), its backward pass and
// the training loss.  One block per instance; matrices k x k row-major.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// dynamic shared memory of the per-instance kernels: nmat k x (k + 1) FP32
// matrices plus 4 k + 64 floats of vectors
constexpr size_t inst_smem(int nmat) {
  return sizeof(float) * ((size_t)nmat * WS_KMAX * (WS_KMAX + 1) + 4 * WS_KMAX + 64);
}
#define MAT(base, i, j) base[(i) * (WS_KMAX + 1) + (j)]

__global__ void __launch_bounds__(256) ws_gram_schmidt_kernel(const float* __restrict__ M, int k,
                                                              float* __restrict__ U,
                                                              float* __restrict__ R) {
  extern __shared__ float dsm[];
  float* u = dsm;
  float* r = u + WS_KMAX * (WS_KMAX + 1);
  float* coef = r + WS_KMAX * (WS_KMAX + 1);
  float* red = coef + 4 * WS_KMAX;
  const int inst = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t off = (int64_t)inst * k * k;
  for (int e = tid; e < k * k; e += 256) {
    MAT(u, e / k, e % k) = M[off + e];
    MAT(r, e / k, e % k) = 0.f;
  }
  __syncthreads();
  for (int i = 0; i < k; ++i) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = warp; j < i; j += 8) {
        float d = 0.f;
        for (int a = lane; a < k; a += 32) d = fmaf(MAT(u, a, j), MAT(u, a, i), d);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) coef[j] = d;
      }
      __syncthreads();
      if (tid < k) {
        float v = MAT(u, tid, i);
        for (int j = 0; j < i; ++j) v = fmaf(-coef[j], MAT(u, tid, j), v);
        MAT(u, tid, i) = v;
      }
      if (tid < i) MAT(r, tid, i) += coef[tid];
      __syncthreads();
    }
    const float v = tid < k ? MAT(u, tid, i) : 0.f;
    const float nrm = sqrtf(block_sum(v * v, red));
    const float inv = 1.f / fmaxf(nrm, 1e-30f);
    if (tid < k) MAT(u, tid, i) = v * inv;
    if (tid == 0) MAT(r, i, i) = nrm;
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += 256) {
    U[off + e] = MAT(u, e / k, e % k);
    R[off + e] = MAT(r, e / k, e % k);
  }
}

// dM = (dU + U copyltu(-dU^T U)) R^{-T} for M = U R (positive diagonal R).
__global__ void __launch_bounds__(256) ws_gram_schmidt_bwd_kernel(
    const float* __restrict__ U, const float* __restrict__ R, const float* __restrict__ dU, int k,
    float* __restrict__ dM) {
  extern __shared__ float dsm[];
  float* u = dsm;
  float* du = u + WS_KMAX * (WS_KMAX + 1);
  float* c = du + WS_KMAX * (WS_KMAX + 1);
  float* r = c + WS_KMAX * (WS_KMAX + 1);
  const int inst = blockIdx.x, tid = threadIdx.x;
  const int64_t off = (int64_t)inst * k * k;
  for (int e = tid; e < k * k; e += 256) {
    MAT(u, e / k, e % k) = U[off + e];
    MAT(du, e / k, e % k) = dU[off + e];
    MAT(r, e / k, e % k) = R[off + e];
  }
  __syncthreads();
  // A = -dU^T U; C = tril(A) + tril(A, -1)^T
  for (int e = tid; e < k * k; e += 256) {
    const int i = e / k, j = e % k;
    const int p = i >= j ? i : j, q = i >= j ? j : i;  // C[i][j] = A[p][q]
    float acc = 0.f;
    for (int a = 0; a < k; ++a) acc = fmaf(MAT(du, a, p), MAT(u, a, q), acc);
    MAT(c, i, j) = -acc;
  }
  __syncthreads();
  // X = dU + U C (row a in registers of thread a), then dM = X R^{-T} by back
  // substitution: dM[a][i] = (X[a][i] - sum_{j > i} dM[a][j] R[i][j]) / R[i][i]
  if (tid < k) {
    const int a = tid;
    float x[WS_KMAX];
#pragma unroll
    for (int j = 0; j < WS_KMAX; ++j) {
      if (j < k) {
        float acc = MAT(du, a, j);
        for (int i = 0; i < k; ++i) acc = fmaf(MAT(u, a, i), MAT(c, i, j), acc);
        x[j] = acc;
      }
    }
#pragma unroll
    for (int i = WS_KMAX - 1; i >= 0; --i) {
      if (i < k) {
        float acc = x[i];
#pragma unroll
        for (int j = i + 1; j < WS_KMAX; ++j)
          if (j < k) acc = fmaf(-x[j], MAT(r, i, j), acc);
        x[i] = acc / MAT(r, i, i);
      }
    }
#pragma unroll
    for (int j = 0; j < WS_KMAX; ++j)
      if (j < k) dM[off + (int64_t)a * k + j] = x[j];
  }
}

// loss_b = -sum_i T*(u_i,u_i,u_i)^2 / sum lam^2 and dU = scale * dloss/dU,
// T* = sum_j lam_j u*_j^(x)3.
__global__ void __launch_bounds__(256) ws_loss_grad_kernel(
    const float* __restrict__ U, const float* __restrict__ Us, const float* __restrict__ lam,
    int k, float scale, float* __restrict__ loss, float* __restrict__ dU) {
  extern __shared__ float dsm[];
  float* u = dsm;
  float* us = u + WS_KMAX * (WS_KMAX + 1);
  float* cm = us + WS_KMAX * (WS_KMAX + 1);  // C[j][i] = <u*_j, u_i>
  float* t3 = cm + WS_KMAX * (WS_KMAX + 1);
  float* lm = t3 + WS_KMAX;
  float* red = lm + WS_KMAX;
  const int inst = blockIdx.x, tid = threadIdx.x;
  const int64_t off = (int64_t)inst * k * k;
  for (int e = tid; e < k * k; e += 256) {
    MAT(u, e / k, e % k) = U[off + e];
    MAT(us, e / k, e % k) = Us[off + e];
  }
  if (tid < k) lm[tid] = lam[(int64_t)inst * k + tid];
  __syncthreads();
  for (int e = tid; e < k * k; e += 256) {
    const int j = e / k, i = e % k;
    float acc = 0.f;
    for (int a = 0; a < k; ++a) acc = fmaf(MAT(us, a, j), MAT(u, a, i), acc);
    MAT(cm, j, i) = acc;
  }
  __syncthreads();
  float l2 = 0.f;
  for (int j = 0; j < k; ++j) l2 = fmaf(lm[j], lm[j], l2);
  float part = 0.f;
  if (tid < k) {
    float acc = 0.f;
    for (int j = 0; j < k; ++j) {
      const float cv = MAT(cm, j, tid);
      acc = fmaf(lm[j], cv * cv * cv, acc);
    }
    t3[tid] = acc;
    part = acc * acc;
  }
  const float tot = block_sum(part, red);
  if (tid == 0) loss[inst] = -tot / l2;
  __syncthreads();
  const float g = -6.f * scale / l2;
  for (int e = tid; e < k * k; e += 256) {
    const int a = e / k, i = e % k;
    float acc = 0.f;
    for (int j = 0; j < k; ++j) {
      const float cv = MAT(cm, j, i);
      acc = fmaf(MAT(us, a, j), lm[j] * cv * cv, acc);
    }
    dU[off + e] = g * acc * t3[i];
  }
}

// ---------------------------------------------------------------------------
// Canonical frame: eigenvectors E of the first sketch (cyclic Jacobi, FP32,
// round-robin parallel ordering; rotations as in Golub & Van Loan, Algorithm
// 8.5.2), sorted by descending eigenvalue with the largest-magnitude entry of
// each vector positive.  The network sees the sketches in this frame,
// E^T S_j E, and its output directions are rotated back by E.
// ---------------------------------------------------------------------------
constexpr int JAC_SWEEPS = 24;

__device__ __forceinline__ int rr_index(int pos, int round, int np) {
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (np - 1);
}

// In-place Jacobi on the symmetric k x k matrix a (stride WS_KMAX + 1); v
// receives the eigenvectors (columns).  Eigenvalues are left on diag(a).
__device__ void jacobi_sym(float* a, float* v, int k, float* cs, int* pq, float* red) {
  const int tid = threadIdx.x;
  const int np = k + (k & 1), half = np / 2;
  for (int e = tid; e < k * k; e += blockDim.x) MAT(v, e / k, e % k) = (e / k == e % k) ? 1.f : 0.f;
  float fro = 0.f;
  for (int e = tid; e < k * k; e += blockDim.x) fro += MAT(a, e / k, e % k) * MAT(a, e / k, e % k);
  fro = block_sum(fro, red);
  for (int sweep = 0; sweep < JAC_SWEEPS; ++sweep) {
    float off = 0.f;
    for (int e = tid; e < k * k; e += blockDim.x)
      if (e / k != e % k) off += MAT(a, e / k, e % k) * MAT(a, e / k, e % k);
    off = block_sum(off, red);
    if (off <= 1e-14f * fro) break;
    for (int round = 0; round < np - 1; ++round) {
      if (tid < half) {
        int p = rr_index(tid, round, np), q = rr_index(np - 1 - tid, round, np);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        float c = 1.f, s = 0.f;
        if (q < k) {
          const float apq = MAT(a, p, q);
          if (fabsf(apq) > 1e-30f) {
            const float tau = (MAT(a, q, q) - MAT(a, p, p)) / (2.f * apq);
            const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            s = t * c;
          }
        }
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
        pq[2 * tid] = p;
        pq[2 * tid + 1] = q;
      }
      __syncthreads();
      for (int e = tid; e < half * k; e += blockDim.x) {  // rows p, q of J^T A
        const int i = e / k, j = e % k, p = pq[2 * i], q = pq[2 * i + 1];
        if (q < k) {
          const float c = cs[2 * i], s = cs[2 * i + 1];
          const float ap = MAT(a, p, j), aq = MAT(a, q, j);
          MAT(a, p, j) = c * ap - s * aq;
          MAT(a, q, j) = s * ap + c * aq;
        }
      }
      __syncthreads();
      for (int e = tid; e < half * k; e += blockDim.x) {  // columns p, q of (.) J and V J
        const int i = e / k, j = e % k, p = pq[2 * i], q = pq[2 * i + 1];
        if (q < k) {
          const float c = cs[2 * i], s = cs[2 * i + 1];
          const float ap = MAT(a, j, p), aq = MAT(a, j, q);
          MAT(a, j, p) = c * ap - s * aq;
          MAT(a, j, q) = s * ap + c * aq;
          const float vp = MAT(v, j, p), vq = MAT(v, j, q);
          MAT(v, j, p) = c * vp - s * vq;
          MAT(v, j, q) = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
  }
}

// Per instance: E from S_1, x16 = vec(E^T S_j E) scaled to unit root-mean-square
// (the Frobenius norm is rotation invariant, so the scale comes from S).
__global__ void __launch_bounds__(256) ws_canon_kernel(const float* __restrict__ S, int k, int J,
                                                       float* __restrict__ E,
                                                       float* __restrict__ evals,
                                                       __nv_bfloat16* __restrict__ x16) {
  extern __shared__ float dsm[];
  float* a = dsm;
  float* v = a + WS_KMAX * (WS_KMAX + 1);
  float* e_s = v + WS_KMAX * (WS_KMAX + 1);
  float* t1 = e_s + WS_KMAX * (WS_KMAX + 1);
  float* cs = t1 + WS_KMAX * (WS_KMAX + 1);
  int* pq = reinterpret_cast<int*>(cs + WS_KMAX);
  float* red = cs + 2 * WS_KMAX;
  float* lam = red + 8;
  int* rank = reinterpret_cast<int*>(lam + WS_KMAX);
  const int inst = blockIdx.x, tid = threadIdx.x, kk = k * k;
  const float* Si = S + (int64_t)inst * J * kk;
  float ss = 0.f;
  for (int e = tid; e < J * kk; e += 256) ss += Si[e] * Si[e];
  ss = block_sum(ss, red);
  const float scale = ss > 0.f ? sqrtf((float)(J * kk) / ss) : 0.f;
  for (int e = tid; e < kk; e += 256)
    MAT(a, e / k, e % k) = 0.5f * (Si[e] + Si[(e % k) * k + e / k]);
  __syncthreads();
  jacobi_sym(a, v, k, cs, pq, red);
  // order by descending eigenvalue (ties by index), sign of the largest entry
  if (tid < k) lam[tid] = MAT(a, tid, tid);
  __syncthreads();
  if (tid < k) {
    int r = 0;
    for (int j = 0; j < k; ++j) r += (lam[j] > lam[tid]) || (lam[j] == lam[tid] && j < tid);
    rank[tid] = r;
    float best = 0.f;
    for (int i = 0; i < k; ++i)
      if (fabsf(MAT(v, i, tid)) > fabsf(best)) best = MAT(v, i, tid);
    const float sg = best < 0.f ? -1.f : 1.f;
    for (int i = 0; i < k; ++i) MAT(e_s, i, r) = sg * MAT(v, i, tid);
    if (evals) evals[(int64_t)inst * k + r] = lam[tid];
  }
  __syncthreads();
  for (int e = tid; e < kk; e += 256) E[(int64_t)inst * kk + e] = MAT(e_s, e / k, e % k);
  for (int j = 0; j < J; ++j) {
    const float* Sj = Si + (int64_t)j * kk;
    for (int e = tid; e < kk; e += 256) {  // t1 = S_j E
      const int r = e / k, c = e % k;
      float acc = 0.f;
      for (int m = 0; m < k; ++m) acc = fmaf(Sj[r * k + m], MAT(e_s, m, c), acc);
      MAT(t1, r, c) = acc;
    }
    __syncthreads();
    for (int e = tid; e < kk; e += 256) {  // E^T t1
      const int r = e / k, c = e % k;
      float acc = 0.f;
      for (int m = 0; m < k; ++m) acc = fmaf(MAT(e_s, m, r), MAT(t1, m, c), acc);
      x16[(int64_t)inst * J * kk + (int64_t)j * kk + e] = __float2bfloat16_rn(acc * scale);
    }
    __syncthreads();
  }
}

// out = E U (transpose = 0) or E^T U (transpose = 1), per instance.
__global__ void __launch_bounds__(256) ws_rotate_kernel(const float* __restrict__ E,
                                                        const float* __restrict__ U, int k,
                                                        int transpose, float* __restrict__ out) {
  __shared__ float es[WS_KMAX][WS_KMAX + 1];
  __shared__ float us[WS_KMAX][WS_KMAX + 1];
  const int inst = blockIdx.x, tid = threadIdx.x, kk = k * k;
  for (int e = tid; e < kk; e += 256) {
    es[e / k][e % k] = E[(int64_t)inst * kk + e];
    us[e / k][e % k] = U[(int64_t)inst * kk + e];
  }
  __syncthreads();
  for (int e = tid; e < kk; e += 256) {
    const int r = e / k, c = e % k;
    float acc = 0.f;
    for (int m = 0; m < k; ++m) acc = fmaf(transpose ? es[m][r] : es[r][m], us[m][c], acc);
    out[(int64_t)inst * kk + e] = acc;
  }
}

// ---------------------------------------------------------------------------
// MLP helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) +
         z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

// dst (cols x rows) = src^T for a rows x cols BF16 or FP32 source; 32 x 32 tiles.
template <typename T>
__global__ void transpose_to_bf16_kernel(const T* __restrict__ src, int64_t rows, int64_t cols,
                                         __nv_bfloat16* __restrict__ dst) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? (float)src[r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[c * rows + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
  }
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b,
                                   int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// dZ = dH o GELU'(Z) in place (FP32) and its BF16 copy.
__global__ void gelu_bwd_kernel(float* __restrict__ dH, const float* __restrict__ Z, int64_t n,
                                __nv_bfloat16* __restrict__ dZ16) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float v = dH[i] * gelu_grad(Z[i]);
    dH[i] = v;
    dZ16[i] = __float2bfloat16_rn(v);
  }
}

// out[c] = sum_r X[r][c] (thread per column).
__global__ void colsum_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                              float* __restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float acc = 0.f;
  for (int64_t r = 0; r < rows; ++r) acc += X[r * cols + c];
  out[c] = acc;
}

// Adam (Kingma & Ba 2015, Algorithm 1) on the FP32 master parameters; also
// refreshes their BF16 copy.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v,
                            __nv_bfloat16* __restrict__ p16, int64_t n, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  p[i] = pi;
  p16[i] = __float2bfloat16_rn(pi);
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace otm

namespace otm {
namespace {

// Dynamic shared-memory limits of the per-instance kernels, once per device.
otm_status configure_ws() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  OTM_CHECK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return OTM_OK;
  OTM_CHECK_CUDA(cudaFuncSetAttribute(ws_gram_schmidt_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inst_smem(2)));
  OTM_CHECK_CUDA(cudaFuncSetAttribute(ws_gram_schmidt_bwd_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inst_smem(4)));
  OTM_CHECK_CUDA(cudaFuncSetAttribute(ws_loss_grad_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inst_smem(3)));
  OTM_CHECK_CUDA(cudaFuncSetAttribute(ws_canon_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inst_smem(5)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return OTM_OK;
}

// Parameter offsets (elements) of the network; every segment starts at a
// multiple of 8 elements when d_in, width and d_out are multiples of 8.
struct MlpOff {
  int64_t W1, b1, W2, b2, W3, b3, total;
};
MlpOff mlp_off(int64_t din, int64_t h, int64_t dout) {
  MlpOff o;
  o.W1 = 0;
  o.b1 = o.W1 + h * din;
  o.W2 = o.b1 + h;
  o.b2 = o.W2 + h * h;
  o.W3 = o.b2 + h;
  o.b3 = o.W3 + dout * h;
  o.total = o.b3 + dout;
  return o;
}

// Forward/backward cache and scratch of the MLP for a batch of B inputs.
struct MlpWs {
  int* err;
  float *Z1, *Z2, *dH2, *dH1;
  __nv_bfloat16 *H1, *H2, *dout16, *doutT, *H2T, *H1T, *xT, *dZ2, *dZ2T, *dZ1, *dZ1T;
};

template <typename W>
void mlp_layout(W& w, int64_t B, int64_t din, int64_t h, int64_t dout, MlpWs* o) {
  o->err = w.template take<int>(64);
  o->Z1 = w.template take<float>(B * h);
  o->Z2 = w.template take<float>(B * h);
  o->dH2 = w.template take<float>(B * h);
  o->dH1 = w.template take<float>(B * h);
  o->H1 = w.template take<__nv_bfloat16>(B * h);
  o->H2 = w.template take<__nv_bfloat16>(B * h);
  o->dout16 = w.template take<__nv_bfloat16>(B * dout);
  o->doutT = w.template take<__nv_bfloat16>(B * dout);
  o->H2T = w.template take<__nv_bfloat16>(B * h);
  o->H1T = w.template take<__nv_bfloat16>(B * h);
  o->xT = w.template take<__nv_bfloat16>(B * din);
  o->dZ2 = w.template take<__nv_bfloat16>(B * h);
  o->dZ2T = w.template take<__nv_bfloat16>(B * h);
  o->dZ1 = w.template take<__nv_bfloat16>(B * h);
  o->dZ1T = w.template take<__nv_bfloat16>(B * h);
}

// Size accounting with the same call sequence as mlp_layout.
struct SizeTaker {
  WorkspaceSize s;
  template <typename T>
  T* take(size_t n) {
    s.add<T>(n);
    return nullptr;
  }
};

size_t mlp_ws_bytes(int64_t B, int64_t din, int64_t h, int64_t dout) {
  SizeTaker t;
  MlpWs o;
  mlp_layout(t, B, din, h, dout, &o);
  return t.s.bytes();
}

otm_status check_net(const otm_mlp* net, int64_t B, const char* who) {
  if (!net || !net->p || !net->p16 || !net->w2t16 || !net->w3t16)
    return set_error(OTM_EINVAL, "%s: incomplete network descriptor", who);
  if (net->d_in < 8 || net->width < 8 || net->d_out < 8 || net->d_in % 8 || net->width % 8 ||
      net->d_out % 8)
    return set_error(OTM_EINVAL, "%s: d_in, width and d_out must be positive multiples of 8", who);
  if (B < 8 || B % 8 || B > 65535)
    return set_error(OTM_EINVAL, "%s: batch must be a multiple of 8 in [8, 65528]", who);
  return OTM_OK;
}

template <typename T>
otm_status transpose_bf16(const T* src, int64_t rows, int64_t cols, __nv_bfloat16* dst,
                          cudaStream_t st) {
  const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  transpose_to_bf16_kernel<T><<<grid, dim3(32, 8), 0, st>>>(src, rows, cols, dst);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status mlp_forward_impl(const otm_mlp* net, const void* x16, int64_t B, float* out,
                            const MlpWs& w, cudaStream_t st) {
  const int64_t din = net->d_in, h = net->width, dout = net->d_out;
  const MlpOff o = mlp_off(din, h, dout);
  const __nv_bfloat16* p16 = static_cast<const __nv_bfloat16*>(net->p16);
  OTM_TRY(gemm_bf16_nt(x16, p16 + o.W1, B, h, din, 1, din, din, 0, 0, 2, 1.f, net->p + o.b1,
                       w.Z1, h, 0, w.H1, h, 0, w.err, st));
  OTM_TRY(gemm_bf16_nt(w.H1, p16 + o.W2, B, h, h, 1, h, h, 0, 0, 2, 1.f, net->p + o.b2, w.Z2, h,
                       0, w.H2, h, 0, w.err, st));
  OTM_TRY(gemm_bf16_nt(w.H2, p16 + o.W3, B, dout, h, 1, h, h, 0, 0, 1, 1.f, net->p + o.b3, out,
                       dout, 0, nullptr, 0, 0, w.err, st));
  return OTM_OK;
}

otm_status mlp_backward_impl(const otm_mlp* net, const void* x16, int64_t B, const float* dout_in,
                             const MlpWs& w, cudaStream_t st) {
  const int64_t din = net->d_in, h = net->width, dout = net->d_out;
  const MlpOff o = mlp_off(din, h, dout);
  float* g = net->grad;
  f32_to_bf16_kernel<<<blocks_for(B * dout, 256), 256, 0, st>>>(dout_in, w.dout16, B * dout);
  OTM_CHECK_LAUNCH();
  OTM_TRY(transpose_bf16(dout_in, B, dout, w.doutT, st));
  colsum_kernel<<<blocks_for(dout, 256), 256, 0, st>>>(dout_in, B, dout, g + o.b3);
  OTM_CHECK_LAUNCH();
  OTM_TRY(transpose_bf16(w.H2, B, h, w.H2T, st));
  // dW3 = dout^T H2 ; dH2 = dout W3
  OTM_TRY(gemm_bf16_nt(w.doutT, w.H2T, dout, h, B, 1, B, B, 0, 0, 0, 1.f, nullptr, g + o.W3, h, 0,
                       nullptr, 0, 0, w.err, st));
  OTM_TRY(gemm_bf16_nt(w.dout16, net->w3t16, B, h, dout, 1, dout, dout, 0, 0, 0, 1.f, nullptr,
                       w.dH2, h, 0, nullptr, 0, 0, w.err, st));
  gelu_bwd_kernel<<<blocks_for(B * h, 256), 256, 0, st>>>(w.dH2, w.Z2, B * h, w.dZ2);
  OTM_CHECK_LAUNCH();
  colsum_kernel<<<blocks_for(h, 256), 256, 0, st>>>(w.dH2, B, h, g + o.b2);
  OTM_CHECK_LAUNCH();
  OTM_TRY(transpose_bf16(w.dZ2, B, h, w.dZ2T, st));
  OTM_TRY(transpose_bf16(w.H1, B, h, w.H1T, st));
  // dW2 = dZ2^T H1 ; dH1 = dZ2 W2
  OTM_TRY(gemm_bf16_nt(w.dZ2T, w.H1T, h, h, B, 1, B, B, 0, 0, 0, 1.f, nullptr, g + o.W2, h, 0,
                       nullptr, 0, 0, w.err, st));
  OTM_TRY(gemm_bf16_nt(w.dZ2, net->w2t16, B, h, h, 1, h, h, 0, 0, 0, 1.f, nullptr, w.dH1, h, 0,
                       nullptr, 0, 0, w.err, st));
  gelu_bwd_kernel<<<blocks_for(B * h, 256), 256, 0, st>>>(w.dH1, w.Z1, B * h, w.dZ1);
  OTM_CHECK_LAUNCH();
  colsum_kernel<<<blocks_for(h, 256), 256, 0, st>>>(w.dH1, B, h, g + o.b1);
  OTM_CHECK_LAUNCH();
  OTM_TRY(transpose_bf16(w.dZ1, B, h, w.dZ1T, st));
  OTM_TRY(transpose_bf16(static_cast<const __nv_bfloat16*>(x16), B, din, w.xT, st));
  // dW1 = dZ1^T x
  OTM_TRY(gemm_bf16_nt(w.dZ1T, w.xT, h, din, B, 1, B, B, 0, 0, 0, 1.f, nullptr, g + o.W1, din, 0,
                       nullptr, 0, 0, w.err, st));
  return OTM_OK;
}

otm_status sync_weights_impl(const otm_mlp* net, cudaStream_t st) {
  const int64_t din = net->d_in, h = net->width, dout = net->d_out;
  const MlpOff o = mlp_off(din, h, dout);
  __nv_bfloat16* p16 = static_cast<__nv_bfloat16*>(net->p16);
  OTM_TRY(transpose_bf16(p16 + o.W2, h, h, static_cast<__nv_bfloat16*>(net->w2t16), st));
  OTM_TRY(transpose_bf16(p16 + o.W3, dout, h, static_cast<__nv_bfloat16*>(net->w3t16), st));
  return OTM_OK;
}

// Train-step scratch: the MLP workspace followed by out, U, R, dU, dM.
struct TrainWs {
  MlpWs m;
  float *out, *U, *R, *dU, *dM;
};
template <typename W>
void train_layout(W& w, int64_t B, int64_t din, int64_t h, int64_t dout, TrainWs* o) {
  mlp_layout(w, B, din, h, dout, &o->m);
  o->out = w.template take<float>(B * dout);
  o->U = w.template take<float>(B * dout);
  o->R = w.template take<float>(B * dout);
  o->dU = w.template take<float>(B * dout);
  o->dM = w.template take<float>(B * dout);
}

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

otm_status otm_ws_generate(const float* m, const float* alpha, int64_t nb, int64_t n, int64_t k,
                           uint64_t seed, int64_t first, float* Y, void* stream) {
  clear_error();
  OTM_REQUIRE(m && alpha && Y, "otm_ws_generate: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && nb >= 1 && nb <= 65535 && n >= 1 && first >= 0 &&
                  first + nb <= ((int64_t)1 << 32) && n <= ((int64_t)1 << 32),
              "otm_ws_generate: need 1 <= k <= %d, 1 <= nb <= 65535, n >= 1, instance and "
              "sample indices below 2^32", WS_KMAX);
  cudaStream_t st = as_stream(stream);
  const dim3 grid((unsigned)((n + GEN_SAMPLES - 1) / GEN_SAMPLES), (unsigned)nb);
  ws_generate_kernel<<<grid, GEN_WARPS * 32, 0, st>>>(m, alpha, n, (int)k,
                                                       (uint32_t)(seed & 0xFFFFFFFFu),
                                                       (uint32_t)(seed >> 32), first, Y);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

size_t otm_ws_sketch_workspace(int64_t nb, int64_t n, int64_t k, int J) {
  const int64_t ldn = (n + 7) & ~(int64_t)7;
  const int64_t nblk = (ldn + SK_TS - 1) / SK_TS;
  WorkspaceSize w;
  w.add<int>(64)
      .add<__nv_bfloat16>(nb * k * ldn)
      .add<__nv_bfloat16>(nb * (J + 1) * k * ldn)
      .add<float>(nb * nblk * k)
      .add<float>(nb * k * (J + 1) * k);
  return w.bytes();
}

otm_status otm_ws_sketch(const float* Y, int64_t nb, int64_t n, int64_t k, const double* alpha0,
                         const float* thetas, int J, float* S, void* x16, void* ws,
                         size_t ws_bytes, void* stream) {
  clear_error();
  OTM_REQUIRE(Y && alpha0 && thetas && x16, "otm_ws_sketch: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && J >= 1 && J <= 4 && nb >= 1 && nb <= 65535 && n >= 1,
              "otm_ws_sketch: need 1 <= k <= %d, 1 <= J <= 4, 1 <= nb <= 65535, n >= 1",
              WS_KMAX);
  OTM_REQUIRE(ws && ws_bytes >= otm_ws_sketch_workspace(nb, n, k, J),
              "otm_ws_sketch: workspace too small");
  cudaStream_t st = as_stream(stream);
  const int64_t ldn = (n + 7) & ~(int64_t)7;
  const int64_t nblk = (ldn + SK_TS - 1) / SK_TS;
  Workspace w(ws, ws_bytes);
  int* err = w.take<int>(64);
  __nv_bfloat16* At = w.take<__nv_bfloat16>(nb * k * ldn);
  __nv_bfloat16* Bt = w.take<__nv_bfloat16>(nb * (J + 1) * k * ldn);
  float* psum = w.take<float>(nb * nblk * k);
  float* C = w.take<float>(nb * k * (J + 1) * k);
  OTM_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  ws_sketch_prep_kernel<<<dim3((unsigned)nblk, (unsigned)nb), 256, 0, st>>>(Y, n, (int)k, ldn,
                                                                            thetas, J, At, Bt, psum);
  OTM_CHECK_LAUNCH();
  const int64_t N = (J + 1) * k;
  OTM_TRY(gemm_bf16_nt(At, Bt, k, N, ldn, nb, ldn, ldn, k * ldn, N * ldn, 0, 1.f, nullptr, C, N,
                       k * N, nullptr, 0, 0, err, st));
  ws_sketch_combine_kernel<<<(unsigned)nb, 256, 0, st>>>(C, psum, (int)nblk, n, (int)k, J, alpha0,
                                                         thetas, S,
                                                         static_cast<__nv_bfloat16*>(x16));
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

size_t otm_ws_init_workspace(int64_t nb, int64_t n, int64_t k) {
  WorkspaceSize w;
  w.add<double>(nb * ((n + IC_TS - 1) / IC_TS) * 3 * k);
  return w.bytes();
}

otm_status otm_ws_init_components(const float* U0, const float* Y, int64_t nb, int64_t n,
                                  int64_t k, const double* alpha0, double theta, float* V0,
                                  void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_REQUIRE(U0 && Y && alpha0 && V0, "otm_ws_init_components: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && nb >= 1 && nb <= 65535 && n >= 1,
              "otm_ws_init_components: need 1 <= k <= %d, 1 <= nb <= 65535, n >= 1", WS_KMAX);
  OTM_REQUIRE(ws && ws_bytes >= otm_ws_init_workspace(nb, n, k),
              "otm_ws_init_components: workspace too small");
  cudaStream_t st = as_stream(stream);
  const int64_t nblk = (n + IC_TS - 1) / IC_TS;
  Workspace w(ws, ws_bytes);
  double* part = w.take<double>(nb * nblk * 3 * k);
  ws_init_partial_kernel<<<dim3((unsigned)nblk, (unsigned)nb), 256, 0, st>>>(U0, Y, n, (int)k,
                                                                             part);
  OTM_CHECK_LAUNCH();
  ws_init_final_kernel<<<(unsigned)nb, 256, 0, st>>>(U0, part, (int)nblk, n, (int)k, alpha0,
                                                      0.5 * (1.0 + theta), V0);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status otm_gram_schmidt(const float* M, int64_t nb, int64_t k, float* U, float* R,
                            void* stream) {
  clear_error();
  OTM_REQUIRE(M && U && R, "otm_gram_schmidt: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && nb >= 1, "otm_gram_schmidt: need 1 <= k <= %d", WS_KMAX);
  OTM_TRY(configure_ws());
  cudaStream_t st = as_stream(stream);
  ws_gram_schmidt_kernel<<<(unsigned)nb, 256, inst_smem(2), st>>>(M, (int)k, U, R);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status otm_gram_schmidt_backward(const float* U, const float* R, const float* dU, int64_t nb,
                                     int64_t k, float* dM, void* stream) {
  clear_error();
  OTM_REQUIRE(U && R && dU && dM, "otm_gram_schmidt_backward: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && nb >= 1, "otm_gram_schmidt_backward: need 1 <= k <= %d",
              WS_KMAX);
  OTM_TRY(configure_ws());
  cudaStream_t st = as_stream(stream);
  ws_gram_schmidt_bwd_kernel<<<(unsigned)nb, 256, inst_smem(4), st>>>(U, R, dU, (int)k, dM);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status otm_ws_loss_grad(const float* U, const float* Ustar, const float* lam, int64_t nb,
                            int64_t k, double scale, float* loss, float* dU, void* stream) {
  clear_error();
  OTM_REQUIRE(U && Ustar && lam && loss && dU, "otm_ws_loss_grad: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && nb >= 1, "otm_ws_loss_grad: need 1 <= k <= %d", WS_KMAX);
  OTM_TRY(configure_ws());
  cudaStream_t st = as_stream(stream);
  ws_loss_grad_kernel<<<(unsigned)nb, 256, inst_smem(3), st>>>(U, Ustar, lam, (int)k,
                                                               (float)scale, loss, dU);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

int64_t otm_mlp_param_count(int64_t d_in, int64_t width, int64_t d_out) {
  return mlp_off(d_in, width, d_out).total;
}

size_t otm_mlp_workspace(const otm_mlp* net, int64_t batch) {
  if (!net) return 0;
  return mlp_ws_bytes(batch, net->d_in, net->width, net->d_out);
}

otm_status otm_mlp_sync_weights(const otm_mlp* net, void* stream) {
  clear_error();
  OTM_TRY(check_net(net, 8, "otm_mlp_sync_weights"));
  cudaStream_t st = as_stream(stream);
  const int64_t P = otm_mlp_param_count(net->d_in, net->width, net->d_out);
  f32_to_bf16_kernel<<<blocks_for(P, 256), 256, 0, st>>>(
      net->p, static_cast<__nv_bfloat16*>(net->p16), P);
  OTM_CHECK_LAUNCH();
  return sync_weights_impl(net, st);
}

otm_status otm_mlp_forward(const otm_mlp* net, const void* x16, int64_t batch, float* out,
                           void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_TRY(check_net(net, batch, "otm_mlp_forward"));
  OTM_REQUIRE(x16 && out, "otm_mlp_forward: null pointer");
  OTM_REQUIRE(ws && ws_bytes >= otm_mlp_workspace(net, batch), "otm_mlp_forward: workspace too small");
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  MlpWs m;
  mlp_layout(w, batch, net->d_in, net->width, net->d_out, &m);
  OTM_CHECK_CUDA(cudaMemsetAsync(m.err, 0, sizeof(int), st));
  return mlp_forward_impl(net, x16, batch, out, m, st);
}

otm_status otm_mlp_backward(const otm_mlp* net, const void* x16, int64_t batch, const float* dout,
                            void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_TRY(check_net(net, batch, "otm_mlp_backward"));
  OTM_REQUIRE(x16 && dout && net->grad, "otm_mlp_backward: null pointer");
  OTM_REQUIRE(ws && ws_bytes >= otm_mlp_workspace(net, batch), "otm_mlp_backward: workspace too small");
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  MlpWs m;
  mlp_layout(w, batch, net->d_in, net->width, net->d_out, &m);
  return mlp_backward_impl(net, x16, batch, dout, m, st);
}

otm_status otm_adam_step(const otm_mlp* net, double lr, double b1, double b2, double eps, int64_t t,
                         void* stream) {
  clear_error();
  OTM_TRY(check_net(net, 8, "otm_adam_step"));
  OTM_REQUIRE(net->grad && net->adam_m && net->adam_v && t >= 1,
              "otm_adam_step: need grad, moment buffers and t >= 1");
  cudaStream_t st = as_stream(stream);
  const int64_t P = otm_mlp_param_count(net->d_in, net->width, net->d_out);
  adam_kernel<<<blocks_for(P, 256), 256, 0, st>>>(
      net->p, net->grad, net->adam_m, net->adam_v, static_cast<__nv_bfloat16*>(net->p16), P,
      (float)lr, (float)b1, (float)b2, (float)eps, (float)(1.0 - pow(b1, (double)t)),
      (float)(1.0 - pow(b2, (double)t)));
  OTM_CHECK_LAUNCH();
  return sync_weights_impl(net, st);
}

size_t otm_ws_train_workspace(const otm_mlp* net, int64_t batch) {
  if (!net) return 0;
  SizeTaker t;
  TrainWs o;
  train_layout(t, batch, net->d_in, net->width, net->d_out, &o);
  return t.s.bytes();
}

otm_status otm_ws_train_step(const otm_mlp* net, const void* x16, const float* Ustar,
                             const float* lam, int64_t batch, int64_t k, double lr, int64_t t,
                             float* loss, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_TRY(check_net(net, batch, "otm_ws_train_step"));
  OTM_REQUIRE(x16 && Ustar && lam && loss && net->grad && net->adam_m && net->adam_v,
              "otm_ws_train_step: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && k * k == net->d_out,
              "otm_ws_train_step: need 1 <= k <= %d and d_out = k^2", WS_KMAX);
  OTM_REQUIRE(t >= 1, "otm_ws_train_step: Adam step t >= 1");
  OTM_REQUIRE(ws && ws_bytes >= otm_ws_train_workspace(net, batch),
              "otm_ws_train_step: workspace too small");
  OTM_TRY(configure_ws());
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  TrainWs o;
  train_layout(w, batch, net->d_in, net->width, net->d_out, &o);
  OTM_CHECK_CUDA(cudaMemsetAsync(o.m.err, 0, sizeof(int), st));
  OTM_TRY(mlp_forward_impl(net, x16, batch, o.out, o.m, st));
  ws_gram_schmidt_kernel<<<(unsigned)batch, 256, inst_smem(2), st>>>(o.out, (int)k, o.U, o.R);
  OTM_CHECK_LAUNCH();
  ws_loss_grad_kernel<<<(unsigned)batch, 256, inst_smem(3), st>>>(
      o.U, Ustar, lam, (int)k, 1.f / (float)batch, loss, o.dU);
  OTM_CHECK_LAUNCH();
  ws_gram_schmidt_bwd_kernel<<<(unsigned)batch, 256, inst_smem(4), st>>>(o.U, o.R, o.dU, (int)k,
                                                                          o.dM);
  OTM_CHECK_LAUNCH();
  OTM_TRY(mlp_backward_impl(net, x16, batch, o.dM, o.m, st));
  return otm_adam_step(net, lr, 0.9, 0.999, 1e-8, t, stream);
}

otm_status otm_ws_infer(const otm_mlp* net, const void* x16, int64_t batch, int64_t k, float* U0,
                        void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_TRY(check_net(net, batch, "otm_ws_infer"));
  OTM_REQUIRE(x16 && U0, "otm_ws_infer: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && k * k == net->d_out,
              "otm_ws_infer: need 1 <= k <= %d and d_out = k^2", WS_KMAX);
  OTM_REQUIRE(ws && ws_bytes >= otm_ws_train_workspace(net, batch),
              "otm_ws_infer: workspace too small (otm_ws_train_workspace bytes)");
  OTM_TRY(configure_ws());
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  TrainWs o;
  train_layout(w, batch, net->d_in, net->width, net->d_out, &o);
  OTM_CHECK_CUDA(cudaMemsetAsync(o.m.err, 0, sizeof(int), st));
  OTM_TRY(mlp_forward_impl(net, x16, batch, o.out, o.m, st));
  ws_gram_schmidt_kernel<<<(unsigned)batch, 256, inst_smem(2), st>>>(o.out, (int)k, U0, o.R);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status otm_ws_canonicalize(const float* S, int64_t nb, int64_t k, int J, float* E,
                               float* evals, void* x16, void* stream) {
  clear_error();
  OTM_REQUIRE(S && E && x16, "otm_ws_canonicalize: null pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && J >= 1 && J <= 4 && nb >= 1,
              "otm_ws_canonicalize: need 1 <= k <= %d, 1 <= J <= 4", WS_KMAX);
  OTM_TRY(configure_ws());
  cudaStream_t st = as_stream(stream);
  ws_canon_kernel<<<(unsigned)nb, 256, inst_smem(5), st>>>(S, (int)k, J, E, evals,
                                                            static_cast<__nv_bfloat16*>(x16));
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status otm_ws_rotate(const float* E, const float* U, int64_t nb, int64_t k, int transpose,
                         float* out, void* stream) {
  clear_error();
  OTM_REQUIRE(E && U && out && out != U, "otm_ws_rotate: null or aliased pointer");
  OTM_REQUIRE(k >= 1 && k <= WS_KMAX && nb >= 1, "otm_ws_rotate: need 1 <= k <= %d", WS_KMAX);
  cudaStream_t st = as_stream(stream);
  ws_rotate_kernel<<<(unsigned)nb, 256, 0, st>>>(E, U, (int)k, transpose ? 1 : 0, out);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status otm_ws_check(const void* ws, void* stream) {
  clear_error();
  OTM_REQUIRE(ws, "otm_ws_check: null workspace");
  cudaStream_t st = as_stream(stream);
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h) return set_error(OTM_ETIMEOUT, "a tensor-core wait timed out");
  return OTM_OK;
}

}  // extern "C"
