// STGD for the topic model with the whole third moment of Section 2.1, Eq. (3)
// -- the self-token terms kept -- instead of the sample tensor of Section 3.2,
// in the implicit form of Lemma 3: G = kappa V ((V^T V) o (V^T V)) - T(V, V, I),
// T the minibatch estimate of M3(W, W, W) (per-document normalisation, as for
// the moments), M1 the full-data first moment.  The tensor is never formed.
//
// For component v = v_i, document t with counts c_j over its distinct words j
// (length l), u_j = W_j . v (W_j row j of the whitening), y' = W^T c:
//   s = <y', v> = sum_j c_j u_j,   q = sum_j c_j u_j^2,   mu = <W^T M1, v>,
//   T_t(v, v, I) = a y' + sum_j c_j u_j (b + g u_j) W_j + e m,   m = W^T M1,
//   a = c1 (s^2 - q) / L3 - 2 c2 mu s / L2,    b = -2 c1 s / L3 + 2 c2 mu / L2,
//   g = 2 c1 / L3,                             e = -c2 (s^2 - q) / L2,
// L3 = l (l-1) (l-2) and L2 = l (l-1) (a term whose L is zero is dropped: a
// document too short for a term adds nothing to it).  Over the minibatch of
// b documents (its nnz word occurrences gathered into W_g, nnz x k):
//   U     = W_g V^T                        (nnz x k; U[e, i] = W_j(e) . v_i)
//   Coef  = c o U o (b_t(e) + g_t(e) U)     (elementwise, per occurrence)
//   data  = (W_g^T Coef + Y'^T A) / b + m (sum_t e_t / b + c3 mu o mu)^T
//   V    <- V - beta_t (kappa V ((V^T V) o (V^T V)) - data)
// The two large products are FP32 tiles accumulated in FP64 (gemm_tn_f64acc),
// or, in the BF16 form, tcgen05 products of BF16 operands with FP32
// accumulation: U = W_g V^T in one TMA-fed GEMM, and W_g^T Coef as a batch of
// GEMMs over slices of TE_KC occurrences (transposed BF16 copies of W_g and
// Coef), whose FP32 partials are added in FP64.  The per-document sums and
// coefficients stay as in the FP32 form.
// One step is a short sequence of launches; the host drives the steps.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "otm_internal.cuh"

namespace otm {
namespace {

constexpr int TE_KMAX = 128;
constexpr int TE_WPD = 4;  // warps per document in the gather
constexpr int TE_KC = 1536;  // occurrences per slice of the BF16 W_g^T Coef product

// Per-step preparation, one block per component i: mu_i = <m, v_i> and column
// i of the transpose of V (Vt[r][i] = v_i[r]) for the product U = W_g Vt.
__global__ void __launch_bounds__(TE_KMAX) te_prep_kernel(const float* __restrict__ V, int k,
                                                          const double* __restrict__ m,
                                                          double* __restrict__ mu,
                                                          float* __restrict__ Vt) {
  __shared__ double red[TE_KMAX / 32];
  const int i = blockIdx.x, r = threadIdx.x;
  double x = 0.0;
  if (r < k) {
    const float v = V[i * k + r];
    Vt[r * k + i] = v;
    x = m[r] * (double)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((r & 31) == 0) red[r >> 5] = x;
  __syncthreads();
  if (r == 0) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < TE_KMAX / 32; ++w) acc += red[w];
    mu[i] = acc;
  }
}

// Occurrences of each minibatch document (one thread per document) and their
// exclusive prefix sums (one block, sequential over chunks of 1,024).  doc[t]
// is the corpus row of minibatch position t (-1: outside the corpus, an empty
// document).  *flag |= 1 when the minibatch holds more than cap occurrences.
__global__ void __launch_bounds__(1024) te_offsets_kernel(const int32_t* __restrict__ row_ptr,
                                                          const int32_t* __restrict__ doc,
                                                          int64_t nb, int64_t cap,
                                                          int64_t* __restrict__ off,
                                                          int* __restrict__ flag) {
  __shared__ int64_t part[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t t = base + threadIdx.x;
    int64_t c = 0;
    if (t < nb && doc[t] >= 0) c = row_ptr[doc[t] + 1] - row_ptr[doc[t]];
    part[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan
      const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    if (t < nb) off[t] = carry + part[threadIdx.x] - c;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    off[nb] = carry;
    if (carry > cap) atomicOr(flag, 1);
  }
}

// TE_WPD warps per minibatch document, each over a contiguous part of its
// occurrences: their rows of W into W_g and their counts into cnt, and the
// part's sums of c_j W_j (Ypp[t][w], FP32) and of the counts (lenp[t][w]); the
// coefficient kernel adds the parts in a fixed order into y'_t and l_t.  The
// (word, count) pairs come 32 at a time (one coalesced load, broadcast by
// shuffles), so the W-row loads of consecutive occurrences are independent.
// Writes nothing past cap occurrences.
// BF: W_g as BF16 rows of kpad columns (zero beyond k) in Wg16, else FP32 rows
// of k columns in Wg.
template <bool BF>
__global__ void __launch_bounds__(256) te_gather_kernel(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, const int32_t* __restrict__ doc, int64_t nb,
    const float* __restrict__ W, int k, int kpad, const int64_t* __restrict__ off, int64_t cap,
    float* __restrict__ Wg, __nv_bfloat16* __restrict__ Wg16, float* __restrict__ cnt,
    float* __restrict__ Ypp, float* __restrict__ lenp) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int64_t t = wid / TE_WPD;
  const int part = (int)(wid % TE_WPD);
  if (t >= nb) return;
  float acc[TE_KMAX / 32];
#pragma unroll
  for (int q = 0; q < TE_KMAX / 32; ++q) acc[q] = 0.f;
  float l = 0.f;
  if (doc[t] >= 0) {
    const int32_t d0 = row_ptr[doc[t]], d1 = row_ptr[doc[t] + 1];
    const int32_t per = (d1 - d0 + TE_WPD - 1) / TE_WPD;
    const int32_t e0 = d0 + part * per < d1 ? d0 + part * per : d1;
    const int32_t e1 = e0 + per < d1 ? e0 + per : d1;
    const int64_t o = off[t] + (e0 - d0);
    for (int32_t base = e0; base < e1; base += 32) {
      const int cntb = e1 - base < 32 ? e1 - base : 32;
      int32_t my_j = 0;
      float my_c = 0.f;
      if (lane < cntb) {
        my_j = col[base + lane];
        my_c = val[base + lane];
        const int64_t g = o + (base + lane - e0);
        if (g < cap) cnt[g] = my_c;
      }
#pragma unroll 4
      for (int x = 0; x < cntb; ++x) {
        const int32_t j = __shfl_sync(0xffffffffu, my_j, x);
        const float c = __shfl_sync(0xffffffffu, my_c, x);
        const int64_t g = o + (base + x - e0);
        l += c;
        const bool keep = g < cap;
#pragma unroll
        for (int q = 0; q < TE_KMAX / 32; ++q) {
          const int r = lane + 32 * q;
          if (r < k) {
            const float w = __ldg(W + (int64_t)j * k + r);
            acc[q] = fmaf(c, w, acc[q]);
            if (keep) {
              if constexpr (BF)
                Wg16[g * kpad + r] = __float2bfloat16(w);
              else
                Wg[g * k + r] = w;
            }
          } else if (BF && r < kpad && keep) {
            Wg16[g * kpad + r] = __float2bfloat16(0.f);
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < TE_KMAX / 32; ++q) {
    const int r = lane + 32 * q;
    if (r < k) Ypp[wid * k + r] = acc[q];
  }
  if (lane == 0) lenp[wid] = l;
}

// One block per minibatch document, one thread per component: y'_t and l_t from
// the gather's parts, then s, q, the coefficients a (into A), e (summed into
// esum, FP64), and U -> Coef in place.
// BF: Coef into C16 (BF16, rows of kpad), else into U in place.
template <bool BF>
__global__ void __launch_bounds__(TE_KMAX) te_coef_kernel(
    const int64_t* __restrict__ off, int64_t cap, const float* __restrict__ cnt,
    const float* __restrict__ Ypp, const float* __restrict__ lenp, float* __restrict__ Yp,
    const float* __restrict__ V, const double* __restrict__ mu, int k, int kpad, float c1,
    float c2, float* __restrict__ U, __nv_bfloat16* __restrict__ C16, float* __restrict__ A,
    double* __restrict__ esum) {
  __shared__ float s_len;
  const int64_t t = blockIdx.x;
  const int i = threadIdx.x;
  if (i < k) {
    float y = 0.f;
#pragma unroll
    for (int w = 0; w < TE_WPD; ++w) y += Ypp[(t * TE_WPD + w) * k + i];
    Yp[t * k + i] = y;
  }
  if (i == 0) {
    float l = 0.f;
#pragma unroll
    for (int w = 0; w < TE_WPD; ++w) l += lenp[t * TE_WPD + w];
    s_len = l;
  }
  __syncthreads();
  if (i >= k) return;
  const int64_t e0 = off[t], e1 = min(off[t + 1], cap);
  const double l = (double)s_len;
  const double L2 = l >= 2.0 ? l * (l - 1.0) : 0.0;
  const double L3 = l >= 3.0 ? l * (l - 1.0) * (l - 2.0) : 0.0;
  // s = <y'_t, v_i> and q over the document's occurrences, accumulated in FP64
  // from FP32 partial sums of 4 (s) and 8 (q, all terms non-negative) terms, so
  // that s^2 - q (the pairs of distinct tokens) keeps the cancellation of the
  // self-pairs to the accuracy of the FP32 inputs while the FP64 pipe does
  // one addition per partial sum.
  double s2[2] = {0.0, 0.0};
  int r = 0;
  for (; r + 8 <= k; r += 8) {
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      float p = Yp[t * k + r + 4 * x] * V[i * k + r + 4 * x];
#pragma unroll
      for (int y = 1; y < 4; ++y) p = fmaf(Yp[t * k + r + 4 * x + y], V[i * k + r + 4 * x + y], p);
      s2[x] += (double)p;
    }
  }
  for (; r < k; ++r) s2[0] = fma((double)Yp[t * k + r], (double)V[i * k + r], s2[0]);
  const double sd = s2[0] + s2[1];
  double q2[2] = {0.0, 0.0};
  int64_t e = e0;
  for (; e + 16 <= e1; e += 16) {
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      float p = 0.f;
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        const float u = U[(e + 8 * x + y) * k + i];
        p = fmaf(cnt[e + 8 * x + y] * u, u, p);
      }
      q2[x] += (double)p;
    }
  }
  for (; e < e1; ++e) {
    const double u = U[e * k + i];
    q2[0] = fma((double)cnt[e] * u, u, q2[0]);
  }
  const double qd = q2[0] + q2[1];
  const double mi = mu[i];
  const double i3 = L3 > 0.0 ? 1.0 / L3 : 0.0, i2 = L2 > 0.0 ? 1.0 / L2 : 0.0;
  const double a = c1 * (sd * sd - qd) * i3 - 2.0 * c2 * mi * sd * i2;
  const double bc = -2.0 * c1 * sd * i3 + 2.0 * c2 * mi * i2;
  const double g = 2.0 * c1 * i3;
  const double ec = -c2 * (sd * sd - qd) * i2;
  A[t * k + i] = (float)a;
  atomicAdd(&esum[i], ec);
  const float bf = (float)bc, gf = (float)g;
#pragma unroll 4
  for (int64_t x = e0; x < e1; ++x) {
    const float u = U[x * k + i];
    const float cf = cnt[x] * u * fmaf(gf, u, bf);
    if constexpr (BF)
      C16[x * kpad + i] = __float2bfloat16(cf);
    else
      U[x * k + i] = cf;
  }
}

// One block per component i: the Gram term from V, the data term from the FP64
// products (Gd[r][i], already divided by b) and the m terms, the update into Vn.
__global__ void __launch_bounds__(TE_KMAX) te_finish_kernel(
    const float* __restrict__ V, int k, const double* __restrict__ Gd,
    const double* __restrict__ m, const double* __restrict__ mu,
    const double* __restrict__ esum, double inv_b, float c3, float kappa, float beta,
    float* __restrict__ Vn) {
  __shared__ float h[TE_KMAX];
  const int i = blockIdx.x, r = threadIdx.x;
  if (r < k) {
    float acc = 0.f;
    for (int c = 0; c < k; ++c) acc = fmaf(V[r * k + c], V[i * k + c], acc);
    h[r] = acc * acc;
  }
  __syncthreads();
  if (r < k) {
    float gg = 0.f;
    for (int j = 0; j < k; ++j) gg = fmaf(h[j], V[j * k + r], gg);
    const double data = Gd[(int64_t)r * k + i] + m[r] * (esum[i] * inv_b + (double)c3 * mu[i] * mu[i]);
    Vn[i * k + r] = V[i * k + r] - beta * (kappa * gg - (float)data);
  }
}

// Rows of W_g from this minibatch's last occurrence (off[nb], on the device) to
// the capacity are zeroed, so that the products over all cap rows see only
// this minibatch: U and Coef of those rows are then zero as well.
__global__ void te_zero_tail_kernel(const int64_t* __restrict__ off_end, int64_t cap, int k,
                                    float* __restrict__ Wg) {
  const int64_t start = min(*off_end, cap) * k, end = cap * k;
  for (int64_t i = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
       i += (int64_t)gridDim.x * blockDim.x)
    Wg[i] = 0.f;
}

// BF16 rows [*off_end, capp) of W_g and Coef are zeroed (this minibatch only).
__global__ void te_zero_tail16_kernel(const int64_t* __restrict__ off_end, int64_t cap,
                                      int64_t capp, int kpad, __nv_bfloat16* __restrict__ a,
                                      __nv_bfloat16* __restrict__ b) {
  const int64_t start = min(*off_end, cap) * kpad, end = capp * kpad;
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  for (int64_t i = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
       i += (int64_t)gridDim.x * blockDim.x) {
    a[i] = z;
    b[i] = z;
  }
}

// V16[i][r] = bf16(V[i][r]) for r < k, zero for k <= r < kpad (one block per i).
__global__ void te_v16_kernel(const float* __restrict__ V, int k, int kpad,
                              __nv_bfloat16* __restrict__ V16) {
  const int i = blockIdx.x;
  for (int r = threadIdx.x; r < kpad; r += blockDim.x)
    V16[i * kpad + r] = __float2bfloat16(r < k ? V[i * k + r] : 0.f);
}

// out[c][r] = in[r][c] for r < rows, c < cols (in: rows x ld_in, out: cols x ld_out;
// rows a multiple of 64, ld_in and ld_out even, cols <= ld_in), 64 x 64 tiles
// through shared memory moved as BF16 pairs.
__global__ void te_transpose16_kernel(const __nv_bfloat16* __restrict__ in, int64_t rows,
                                      int cols, int ld_in, __nv_bfloat16* __restrict__ out,
                                      int64_t ld_out) {
  __shared__ __nv_bfloat16 tile[64][66];
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  for (int y = ty; y < 64; y += 8) {
    const int64_t r = r0 + y;
    const int c = c0 + 2 * tx;
    __nv_bfloat162 v;
    v.x = z;
    v.y = z;
    if (r < rows && c < ld_in)
      v = *reinterpret_cast<const __nv_bfloat162*>(in + r * ld_in + c);
    tile[y][2 * tx] = v.x;
    tile[y][2 * tx + 1] = v.y;
  }
  __syncthreads();
  for (int y = ty; y < 64; y += 8) {
    const int c = c0 + y;
    const int64_t r = r0 + 2 * tx;
    if (c < cols && r < rows) {
      __nv_bfloat162 v;
      v.x = tile[2 * tx][y];
      v.y = tile[2 * tx + 1][y];
      *reinterpret_cast<__nv_bfloat162*>(out + (int64_t)c * ld_out + r) = v;
    }
  }
}

// Gd[e] = scale * sum_z part[z][e] in FP64, e < kk (eight slices in flight per
// thread, added in a fixed order).
__global__ void te_reduce_kernel(const float* __restrict__ part, int64_t nz, int64_t kk,
                                 double scale, double* __restrict__ Gd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kk) return;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int64_t z = 0;
  for (; z + 8 <= nz; z += 8) {
#pragma unroll
    for (int x = 0; x < 8; ++x) acc[x] += (double)part[(z + x) * kk + e];
  }
  for (; z < nz; ++z) acc[0] += (double)part[z * kk + e];
  Gd[e] = (((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]))) *
          scale;
}

__global__ void te_docs_kernel(const int32_t* __restrict__ perm, int64_t n, int64_t pos0,
                               int64_t nb, int32_t* __restrict__ doc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb) return;
  const int64_t row = perm ? (int64_t)perm[pos0 + t] : pos0 + t;
  doc[t] = (row >= 0 && row < n) ? (int32_t)row : -1;
}

struct TeWs {
  int32_t* doc;
  int64_t* off;
  float *Wg, *cnt, *Yp, *Ypp, *lenp, *U, *A, *Vt, *Vn;
  double *m, *mu, *esum, *Gd;
  int* flag;
  // BF16 form
  __nv_bfloat16 *Wg16, *C16, *Wt16, *Ct16, *V16;
  float* part;
};

// The BF16 form's row count: the capacity rounded up to whole slices.
inline int64_t te_capp(int64_t cap) { return (cap + TE_KC - 1) / TE_KC * TE_KC; }
inline int te_kpad(int64_t k) { return (int)((k + 7) / 8 * 8); }

TeWs te_take(Workspace& w, int64_t k, int64_t b, int64_t cap, int bf) {
  TeWs s;
  s.doc = w.take<int32_t>(b);
  s.off = w.take<int64_t>(b + 1);
  s.Wg = w.take<float>(bf ? 1 : (size_t)cap * k);
  s.cnt = w.take<float>(cap);
  s.Yp = w.take<float>((size_t)b * k);
  s.Ypp = w.take<float>((size_t)b * TE_WPD * k);
  s.lenp = w.take<float>((size_t)b * TE_WPD);
  s.U = w.take<float>((size_t)(bf ? te_capp(cap) : cap) * k);
  s.A = w.take<float>((size_t)b * k);
  s.Vt = w.take<float>((size_t)k * k);
  s.Vn = w.take<float>((size_t)k * k);
  s.m = w.take<double>(k);
  s.mu = w.take<double>(k);
  s.esum = w.take<double>(k);
  s.Gd = w.take<double>((size_t)k * k);
  s.flag = w.take<int>(2);
  s.Wg16 = s.C16 = s.Wt16 = s.Ct16 = s.V16 = nullptr;
  s.part = nullptr;
  if (bf) {
    const int64_t capp = te_capp(cap), kpad = te_kpad(k);
    s.Wg16 = w.take<__nv_bfloat16>((size_t)capp * kpad);
    s.C16 = w.take<__nv_bfloat16>((size_t)capp * kpad);
    s.Wt16 = w.take<__nv_bfloat16>((size_t)k * capp);
    s.Ct16 = w.take<__nv_bfloat16>((size_t)k * capp);
    s.V16 = w.take<__nv_bfloat16>((size_t)k * kpad);
    s.part = w.take<float>((size_t)(capp / TE_KC) * k * k);
  }
  return s;
}

// Gd = (W_g^T Coef + Y'^T A) / nb with BF16 tensor-core slices of W_g^T Coef.
otm_status te_products16(const TeWs& s, int64_t k, int64_t nb, int64_t cap, cudaStream_t st) {
  const int64_t capp = te_capp(cap), nz = capp / TE_KC;
  const int kpad = te_kpad(k);
  if (nz > 0) {
    const dim3 tg((unsigned)(capp / 64), (unsigned)((k + 63) / 64));
    te_transpose16_kernel<<<tg, 256, 0, st>>>(s.Wg16, capp, (int)k, kpad, s.Wt16, capp);
    OTM_CHECK_LAUNCH();
    te_transpose16_kernel<<<tg, 256, 0, st>>>(s.C16, capp, (int)k, kpad, s.Ct16, capp);
    OTM_CHECK_LAUNCH();
    OTM_TRY(gemm_bf16_nt(s.Wt16, s.Ct16, k, k, TE_KC, nz, capp, capp, TE_KC, TE_KC, 0, 1.f,
                         nullptr, s.part, k, k * k, nullptr, 0, 0, s.flag + 1, st));
    te_reduce_kernel<<<(unsigned)((k * k + 255) / 256), 256, 0, st>>>(s.part, nz, k * k,
                                                                    1.0 / (double)nb, s.Gd);
    OTM_CHECK_LAUNCH();
  } else {
    OTM_CHECK_CUDA(cudaMemsetAsync(s.Gd, 0, sizeof(double) * k * k, st));
  }
  return gemm_tn_f64acc(s.Yp, s.A, nb, k, k, 1.0 / (double)nb, s.Gd, 1, st);
}

// Gd = (W_g^T Coef + Y'^T A) / nb, FP32 tiles accumulated in FP64
otm_status te_products(const TeWs& s, int64_t k, int64_t nb, int64_t cap, cudaStream_t st) {
  OTM_TRY(gemm_tn_f64acc(s.Wg, s.U, cap, k, k, 1.0 / (double)nb, s.Gd, 0, st));
  OTM_TRY(gemm_tn_f64acc(s.Yp, s.A, nb, k, k, 1.0 / (double)nb, s.Gd, 1, st));
  return OTM_OK;
}

WorkspaceSize te_size(int64_t k, int64_t b, int64_t cap, int bf) {
  WorkspaceSize w;
  w.add<int32_t>(b).add<int64_t>(b + 1).add<float>(bf ? 1 : (size_t)cap * k).add<float>(cap);
  w.add<float>((size_t)b * k).add<float>((size_t)b * TE_WPD * k).add<float>((size_t)b * TE_WPD);
  w.add<float>((size_t)(bf ? te_capp(cap) : cap) * k).add<float>((size_t)b * k);
  w.add<float>((size_t)k * k).add<float>((size_t)k * k);
  w.add<double>(k).add<double>(k).add<double>(k).add<double>((size_t)k * k).add<int>(2);
  if (bf) {
    const int64_t capp = te_capp(cap), kpad = te_kpad(k);
    w.add<__nv_bfloat16>((size_t)capp * kpad).add<__nv_bfloat16>((size_t)capp * kpad);
    w.add<__nv_bfloat16>((size_t)k * capp).add<__nv_bfloat16>((size_t)k * capp);
    w.add<__nv_bfloat16>((size_t)k * kpad).add<float>((size_t)(capp / TE_KC) * k * k);
  }
  return w;
}

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

size_t otm_sgd_topic_exact_workspace(int64_t k, int64_t b, int64_t nnz_b_max, int precision) {
  if (k < 1 || k > TE_KMAX || b < 1 || nnz_b_max < 0 || precision < 0 || precision > 1) return 0;
  return te_size(k, b, nnz_b_max, precision).bytes();
}

otm_status otm_sgd_run_topic_exact(float* V, const otm_csr* X, const float* W, const double* M1,
                                   int64_t k, const int32_t* perm, int64_t epochs, int64_t b,
                                   int64_t nnz_b_max, double beta0, double theta, double alpha0,
                                   int precision, float* V_snap, int64_t snapshot_every, void* ws,
                                   size_t ws_bytes, void* stream) {
  clear_error();
  OTM_REQUIRE(precision == 0 || precision == 1,
              "otm_sgd_run_topic_exact: precision %d is not 0 (FP32) or 1 (BF16)", precision);
  const int bf = precision;
  OTM_TRY(check_csr(X, "otm_sgd_run_topic_exact: X"));
  OTM_REQUIRE(V && W && M1, "otm_sgd_run_topic_exact: null pointer");
  OTM_REQUIRE(k >= 1 && k <= TE_KMAX, "otm_sgd_run_topic_exact: k=%lld outside [1, %d]",
              (long long)k, TE_KMAX);
  OTM_REQUIRE(X->rows >= 1 && b >= 1 && epochs >= 0 && nnz_b_max >= 0,
              "otm_sgd_run_topic_exact: need n >= 1, b >= 1, epochs >= 0, nnz_b_max >= 0");
  OTM_REQUIRE(snapshot_every >= 0 && (snapshot_every == 0 || V_snap),
              "otm_sgd_run_topic_exact: V_snap required for snapshots");
  const int64_t n = X->rows, d = X->cols;
  const int64_t nb_max = std::min(b, n);
  OTM_REQUIRE(ws && ws_bytes >= te_size(k, nb_max, nnz_b_max, bf).bytes(),
              "otm_sgd_run_topic_exact: workspace too small (need %zu bytes)",
              te_size(k, nb_max, nnz_b_max, bf).bytes());
  if (epochs == 0) return OTM_OK;
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  const TeWs s = te_take(w, k, nb_max, nnz_b_max, bf);
  const int kpad = te_kpad(k);
  const int64_t capp = te_capp(nnz_b_max);
  OTM_CHECK_CUDA(cudaMemsetAsync(s.flag, 0, 2 * sizeof(int), st));
  OTM_TRY(vec_tn(M1, W, d, k, s.m, st));  // m = W^T M1
  const double a0 = alpha0;
  const float c1 = (float)((a0 + 1.0) * (a0 + 2.0) / 2.0), c2 = (float)(a0 * (a0 + 1.0) / 2.0),
              c3 = (float)(a0 * a0), kappa = (float)(0.5 * (1.0 + theta));
  const int64_t spe = (n + b - 1) / b;
  int64_t t = 0;
  for (int64_t e = 0; e < epochs; ++e)
    for (int64_t jb = 0; jb < spe; ++jb) {
      ++t;
      const int64_t pos0 = jb * b, nb = std::min(b, n - pos0);
      const float beta = (float)(beta0 / std::sqrt((double)t));
      te_docs_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
          perm ? perm + e * n : nullptr, n, pos0, nb, s.doc);
      OTM_CHECK_LAUNCH();
      te_prep_kernel<<<(unsigned)k, TE_KMAX, 0, st>>>(V, (int)k, s.m, s.mu, s.Vt);
      OTM_CHECK_LAUNCH();
      te_offsets_kernel<<<1, 1024, 0, st>>>(X->row_ptr, s.doc, nb, nnz_b_max, s.off, s.flag);
      OTM_CHECK_LAUNCH();
      const unsigned gg = (unsigned)((nb * TE_WPD + 7) / 8);
      if (bf) {
        te_gather_kernel<true><<<gg, 256, 0, st>>>(X->row_ptr, X->col, X->val, s.doc, nb, W,
                                                   (int)k, kpad, s.off, nnz_b_max, nullptr,
                                                   s.Wg16, s.cnt, s.Ypp, s.lenp);
        OTM_CHECK_LAUNCH();
        te_zero_tail16_kernel<<<256, 256, 0, st>>>(s.off + nb, nnz_b_max, capp, kpad, s.Wg16,
                                                   s.C16);
        OTM_CHECK_LAUNCH();
        te_v16_kernel<<<(unsigned)k, 128, 0, st>>>(V, (int)k, kpad, s.V16);
        OTM_CHECK_LAUNCH();
        // U = W_g V^T (tcgen05, BF16 operands, FP32 accumulation) over every row held
        if (capp > 0)
          OTM_TRY(gemm_bf16_nt(s.Wg16, s.V16, capp, k, kpad, 1, kpad, kpad, 0, 0, 0, 1.f, nullptr,
                               s.U, k, 0, nullptr, 0, 0, s.flag + 1, st));
      } else {
        te_gather_kernel<false><<<gg, 256, 0, st>>>(X->row_ptr, X->col, X->val, s.doc, nb, W,
                                                    (int)k, kpad, s.off, nnz_b_max, s.Wg,
                                                    nullptr, s.cnt, s.Ypp, s.lenp);
        OTM_CHECK_LAUNCH();
        te_zero_tail_kernel<<<256, 256, 0, st>>>(s.off + nb, nnz_b_max, (int)k, s.Wg);
        OTM_CHECK_LAUNCH();
        // U = W_g V^T over every row the workspace holds (a minibatch past the
        // capacity has set the flag; its occurrences beyond it are not read)
        if (nnz_b_max > 0)
          OTM_TRY(gemm_nn_small(s.Wg, nnz_b_max, k, s.Vt, k, s.U, nullptr, nullptr, 0.0, st));
      }
      OTM_CHECK_CUDA(cudaMemsetAsync(s.esum, 0, sizeof(double) * k, st));
      if (bf)
        te_coef_kernel<true><<<(unsigned)nb, TE_KMAX, 0, st>>>(
            s.off, nnz_b_max, s.cnt, s.Ypp, s.lenp, s.Yp, V, s.mu, (int)k, kpad, c1, c2, s.U,
            s.C16, s.A, s.esum);
      else
        te_coef_kernel<false><<<(unsigned)nb, TE_KMAX, 0, st>>>(
            s.off, nnz_b_max, s.cnt, s.Ypp, s.lenp, s.Yp, V, s.mu, (int)k, kpad, c1, c2, s.U,
            nullptr, s.A, s.esum);
      OTM_CHECK_LAUNCH();
      OTM_TRY(bf ? te_products16(s, k, nb, nnz_b_max, st) : te_products(s, k, nb, nnz_b_max, st));
      te_finish_kernel<<<(unsigned)k, TE_KMAX, 0, st>>>(V, (int)k, s.Gd, s.m, s.mu, s.esum,
                                                        1.0 / (double)nb, c3, kappa, beta, s.Vn);
      OTM_CHECK_LAUNCH();
      OTM_CHECK_CUDA(cudaMemcpyAsync(V, s.Vn, sizeof(float) * k * k, cudaMemcpyDeviceToDevice, st));
      if (snapshot_every > 0 && t % snapshot_every == 0)
        OTM_CHECK_CUDA(cudaMemcpyAsync(V_snap + (t / snapshot_every - 1) * k * k, V,
                                       sizeof(float) * k * k, cudaMemcpyDeviceToDevice, st));
    }
  int h[2] = {0, 0};
  OTM_CHECK_CUDA(cudaMemcpyAsync(h, s.flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h[1])
    return set_error(OTM_ETIMEOUT, "otm_sgd_run_topic_exact: a tensor-core product's wait timed out");
  if (h[0])
    return set_error(OTM_EINVAL, "otm_sgd_run_topic_exact: a minibatch holds more than "
                                 "nnz_b_max = %lld word occurrences", (long long)nnz_b_max);
  return OTM_OK;
}

}  // extern "C"
