// Sparse kernels over CSR count data: per-document statistics and first
// moments (Section 2.1 Eq. (1), the diagonal term of Eq. (2); Section 2.2
// Eq. (9)), and the two sparse-dense products the method is built from:
//   gather  SpMM  out = diag(s) X B        (projection y_t = W^T c_t, Section 3.1;
//                                            the X S half of M2 S, Section 4.2)
//   scatter SpMM  out += X^T diag(s) P     (the X^T half of M2 S and Pairs S)
// One warp per CSR row; the dense rows move as float4 (coalesced 16-byte
// loads), the row's (col, val) pairs are loaded once per warp and broadcast
// with shuffles.
//
// The topic whitening instead transposes the counts once (the CSR of X^T:
// per-word counts, an exclusive scan, a scatter of (document, count) pairs)
// and forms X^T P as a gather over that transpose: each warp takes a fixed
// run of nonzeros in word order (so a word of 300,000 documents is spread over
// many warps), sums the P rows of each word's documents in registers, and
// writes a word it holds whole with plain stores, a word it shares with
// another warp with vector atomics.  That replaces one vector atomic per
// nonzero by at most two per warp.  The first moments become per-word sums in
// FP64 over the same transpose, without atomics.
#include "otm_internal.cuh"

namespace otm {
namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Nonzeros per warp of the gather over the transpose.
constexpr int kCscChunk = 256;

// l_t, 1/l_t, 1/(l_t(l_t-1)) and the FP64 first-moment scatters.
__global__ void topic_stats_kernel(const int32_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ col,
                                   const float* __restrict__ val, int64_t rows, double inv_n,
                                   float* __restrict__ row_invlen, float* __restrict__ row_w,
                                   double* __restrict__ M1, double* __restrict__ delta) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= rows) return;
  const int32_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
  float l = 0.f;
  for (int32_t e = e0 + lane; e < e1; e += 32) l += val[e];
  l = warp_sum(l);
  // counts are integers: l is exact in float32 below 2^24
  const double ld = (double)l;
  const double invl = ld > 0.0 ? 1.0 / ld : 0.0;
  const double w = ld >= 2.0 ? 1.0 / (ld * (ld - 1.0)) : 0.0;
  if (lane == 0) {
    row_invlen[r] = (float)invl;
    row_w[r] = (float)w;
  }
  const double a = invl * inv_n, b = w * inv_n;
  for (int32_t e = e0 + lane; e < e1; e += 32) {
    const double v = (double)val[e];
    const int32_t c = col[e];
    if (a != 0.0) atomicAdd(&M1[c], v * a);
    if (b != 0.0) atomicAdd(&delta[c], v * b);
  }
}

__global__ void column_sums_kernel(const int32_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ col,
                                   const float* __restrict__ val, int64_t rows, double scale,
                                   double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= rows) return;
  for (int32_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32)
    atomicAdd(&out[col[e]], scale * (double)val[e]);
}

// Gather SpMM, float4 path: m % 4 == 0, NV float4 per lane (m <= 128 * NV).
template <int NV>
__global__ void __launch_bounds__(256) spmm_gather_v4_kernel(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, int64_t rows, const float4* __restrict__ B, int m4,
    const float* __restrict__ row_scale, float4* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= rows) return;
  float4 acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int32_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
  for (int32_t base = e0; base < e1; base += 32) {
    const int cnt = min(32, e1 - base);
    int32_t my_c = 0;
    float my_v = 0.f;
    if (lane < cnt) {
      my_c = col[base + lane];
      my_v = val[base + lane];
    }
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
      const int32_t c = __shfl_sync(0xffffffffu, my_c, j);
      const float v = __shfl_sync(0xffffffffu, my_v, j);
      const float4* brow = B + (int64_t)c * m4;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int idx = lane + 32 * q;
        if (idx < m4) {
          const float4 b = __ldg(brow + idx);
          acc[q].x = fmaf(v, b.x, acc[q].x);
          acc[q].y = fmaf(v, b.y, acc[q].y);
          acc[q].z = fmaf(v, b.z, acc[q].z);
          acc[q].w = fmaf(v, b.w, acc[q].w);
        }
      }
    }
  }
  const float s = row_scale ? row_scale[r] : 1.f;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int idx = lane + 32 * q;
    if (idx < m4) {
      float4 a = acc[q];
      a.x *= s; a.y *= s; a.z *= s; a.w *= s;
      out[r * m4 + idx] = a;
    }
  }
}

// Gather SpMM, scalar path (any m): lanes stride over columns.
__global__ void __launch_bounds__(256) spmm_gather_scalar_kernel(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, int64_t rows, const float* __restrict__ B, int64_t m,
    const float* __restrict__ row_scale, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= rows) return;
  const float s = row_scale ? row_scale[r] : 1.f;
  const int32_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
  for (int64_t c0 = 0; c0 < m; c0 += 32) {
    const int64_t cc = c0 + lane;
    float acc = 0.f;
    for (int32_t e = e0; e < e1; ++e) {
      if (cc < m) acc = fmaf(val[e], __ldg(B + (int64_t)col[e] * m + cc), acc);
    }
    if (cc < m) out[r * m + cc] = acc * s;
  }
}

// Scatter SpMM, float4 path: out[col, :] += coef * P[r, :], vector atomics.
template <int NV>
__global__ void __launch_bounds__(256) spmm_scatter_v4_kernel(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, int64_t rows, const float4* __restrict__ P, int m4,
    const float* __restrict__ row_scale, float alpha, float4* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= rows) return;
  const float s = alpha * (row_scale ? row_scale[r] : 1.f);
  if (s == 0.f) return;
  float4 p[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int idx = lane + 32 * q;
    p[q] = idx < m4 ? P[r * m4 + idx] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int32_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
  for (int32_t base = e0; base < e1; base += 32) {
    const int cnt = min(32, e1 - base);
    int32_t my_c = 0;
    float my_v = 0.f;
    if (lane < cnt) {
      my_c = col[base + lane];
      my_v = val[base + lane];
    }
    for (int j = 0; j < cnt; ++j) {
      const int32_t c = __shfl_sync(0xffffffffu, my_c, j);
      const float v = s * __shfl_sync(0xffffffffu, my_v, j);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int idx = lane + 32 * q;
        if (idx < m4) {
          float4 a = p[q];
          a.x *= v; a.y *= v; a.z *= v; a.w *= v;
          atomicAdd(out + (int64_t)c * m4 + idx, a);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(256) spmm_scatter_scalar_kernel(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, int64_t rows, const float* __restrict__ P, int64_t m,
    const float* __restrict__ row_scale, float alpha, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= rows) return;
  const float s = alpha * (row_scale ? row_scale[r] : 1.f);
  if (s == 0.f) return;
  for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
    const float v = s * val[e];
    float* orow = out + (int64_t)col[e] * m;
    for (int64_t cc = lane; cc < m; cc += 32) atomicAdd(orow + cc, v * P[r * m + cc]);
  }
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---- transpose of the counts and the products over it ----

__global__ void csc_count_kernel(const int32_t* __restrict__ col, int64_t nnz,
                                 int32_t* __restrict__ cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[e]], 1);
}

// ptr[0..d] = exclusive prefix sums of cnt[0..d-1] (ptr[d] = total), cursor = ptr[0..d-1].
// One block: warp w takes the w-th contiguous share of the entries, read in
// batches of 256 (eight coalesced loads in flight per lane); the warps' sums are
// scanned, and each warp then writes its share's prefix sums, one warp-wide
// scan of 32 entries at a time.
// cnt and cursor may be the same array (each lane reads an entry before writing it).
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(const int32_t* cnt, int64_t d,
                                                              int32_t* __restrict__ ptr,
                                                              int32_t* cursor) {
  __shared__ int64_t wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t share = ((d + 31) / 32 + 255) & ~(int64_t)255;
  const int64_t b = warp * share, e = b + share < d ? b + share : d;
  int64_t sum = 0;
  for (int64_t base = b; base < e; base += 256) {
    int32_t c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t i = base + 32 * j + lane;
      c[j] = i < e ? cnt[i] : 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) sum += c[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) wsum[warp] = sum;
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the 32 warp sums
    const int64_t v = wsum[lane];
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    wsum[lane] = x - v;
    if (lane == 31) ptr[d] = (int32_t)x;
  }
  __syncthreads();
  int64_t run = wsum[warp];
  for (int64_t base = b; base < e; base += 256) {
    int32_t c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t i = base + 32 * j + lane;
      c[j] = i < e ? cnt[i] : 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int64_t x = c[j];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const int64_t i = base + 32 * j + lane;
      if (i < e) {
        ptr[i] = (int32_t)(run + x - c[j]);
        cursor[i] = (int32_t)(run + x - c[j]);
      }
      run += __shfl_sync(0xffffffffu, x, 31);
    }
  }
}

// Scatter of (row, value) pairs into the transpose (one warp per CSR row).
__global__ void __launch_bounds__(256) csc_fill_kernel(const int32_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col,
                                                       const float* __restrict__ val, int64_t rows,
                                                       int32_t* __restrict__ cursor,
                                                       int32_t* __restrict__ rowT,
                                                       float* __restrict__ valT) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= rows) return;
  for (int32_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
    const int32_t pos = atomicAdd(&cursor[col[e]], 1);
    rowT[pos] = (int32_t)r;
    valT[pos] = val[e];
  }
}

// Document lengths l_t (exact in float32), 1/l_t and 1/(l_t(l_t-1)) in float32
// and, scaled by 1/n, in FP64 (wa, wb) for the first-moment sums.
__global__ void __launch_bounds__(256) topic_rows_kernel(const int32_t* __restrict__ row_ptr,
                                                         const float* __restrict__ val,
                                                         int64_t rows, double inv_n,
                                                         double* __restrict__ wa,
                                                         double* __restrict__ wb,
                                                         float* __restrict__ row_invlen,
                                                         float* __restrict__ row_w) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= rows) return;
  float l = 0.f;
  for (int32_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) l += val[e];
  l = warp_sum(l);
  if (lane == 0) {
    const double ld = (double)l;
    const double a = ld > 0.0 ? 1.0 / ld : 0.0, b = ld >= 2.0 ? 1.0 / (ld * (ld - 1.0)) : 0.0;
    wa[r] = a * inv_n;
    wb[r] = b * inv_n;
    row_invlen[r] = (float)a;
    row_w[r] = (float)b;
  }
}

// M1[c] += sum_t X[t, c] wa[t] and delta[c] += sum_t X[t, c] wb[t] over the
// transpose (M1, delta pre-zeroed), FP64.  Each warp takes kCscChunk nonzeros in
// column order; a column it holds whole is stored, a shared one added atomically.
__global__ void __launch_bounds__(256) topic_cols_kernel(const int32_t* __restrict__ colptr,
                                                         const int32_t* __restrict__ rowT,
                                                         const float* __restrict__ valT,
                                                         int64_t d, int64_t nnz,
                                                         const double* __restrict__ wa,
                                                         const double* __restrict__ wb,
                                                         double* __restrict__ M1,
                                                         double* __restrict__ delta) {
  const int lane = threadIdx.x & 31;
  const int64_t e0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * kCscChunk;
  if (e0 >= nnz) return;
  const int64_t e1 = e0 + kCscChunk < nnz ? e0 + kCscChunk : nnz;
  int64_t lo = 0, hi = d - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (colptr[mid] <= e0) lo = mid; else hi = mid - 1;
  }
  int64_t c = lo, e = e0;
  while (e < e1) {
    const int64_t cb = colptr[c], ce = colptr[c + 1];
    const int64_t se = ce < e1 ? ce : e1;
    double a = 0.0, b = 0.0;
    for (int64_t x = e + lane; x < se; x += 32) {
      const int32_t r = rowT[x];
      const double v = (double)valT[x];
      a = fma(v, wa[r], a);
      b = fma(v, wb[r], b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      if (cb >= e0 && ce <= e1) {
        M1[c] = a;
        delta[c] = b;
      } else {
        atomicAdd(&M1[c], a);
        atomicAdd(&delta[c], b);
      }
    }
    e = se;
    ++c;
    while (c < d && colptr[c + 1] <= e) ++c;
  }
}

// ---- blocked transpose: counting sort by word, one row block per CTA ----
// Row block b = rows [b R, (b + 1) R), R <= 65535, so a word's count within a
// block fits 16 bits: the CTA keeps one 16-bit counter per word in shared
// memory (two per 32-bit word), d <= 2 x (shared memory / 4).  Pass 1 writes
// the block's counts to bc[b][w]; a scan over blocks turns them into the
// block's offsets within each word; pass 2 places the entries at
// colptr[w] + bc[b][w] + (rank within the block).
__global__ void __launch_bounds__(1024) csc_block_count_kernel(const int32_t* __restrict__ row_ptr,
                                                               const int32_t* __restrict__ col,
                                                               int64_t rows, int64_t R, int64_t d,
                                                               int32_t* __restrict__ bc) {
  extern __shared__ uint32_t cnt2[];
  const int64_t dh = (d + 1) >> 1;
  for (int64_t i = threadIdx.x; i < dh; i += blockDim.x) cnt2[i] = 0u;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r1 = r0 + R < rows ? r0 + R : rows;
  const int64_t e0 = row_ptr[r0], e1 = row_ptr[r1];
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int32_t w = col[e];
    atomicAdd(&cnt2[w >> 1], 1u << ((w & 1) * 16));
  }
  __syncthreads();
  int32_t* out = bc + (int64_t)blockIdx.x * d;
  for (int64_t w = threadIdx.x; w < d; w += blockDim.x)
    out[w] = (int32_t)((cnt2[w >> 1] >> ((w & 1) * 16)) & 0xFFFFu);
}

// For each word: bc[b][w] <- sum_{b' < b} bc[b'][w] (in place), total[w] = the sum over all b.
// Eight blocks' counts are loaded before any is used, so that a thread keeps
// eight loads in flight instead of one.
__global__ void csc_block_scan_kernel(int32_t* __restrict__ bc, int64_t nblocks, int64_t d,
                                      int32_t* __restrict__ total) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= d) return;
  int32_t run = 0;
  for (int64_t b0 = 0; b0 < nblocks; b0 += 8) {
    int32_t c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j] = b0 + j < nblocks ? bc[(b0 + j) * d + w] : 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (b0 + j < nblocks) bc[(b0 + j) * d + w] = run;
      run += c[j];
    }
  }
  total[w] = run;
}

// Pass 2 in phases over ranges of consecutive words [wl, wh), each holding at
// most `quota` entries (or one word) and at most W words: in a phase the CTA
// keeps one 32-bit cursor per word of the range, colptr[w] + bc[b][w], and
// places the block's entries of those words at the cursor (atomic increment).
// Every CTA derives the same ranges from colptr and runs them in the same
// order, so the output being written at a time is the one contiguous slice
// colptr[wl] .. colptr[wh]: small enough for L2 to hold its partly written
// sectors until they are complete, instead of evicting them half written (a
// read-modify-write in DRAM for each) as one pass over all words does.  The
// ranges follow the entry counts, not the word indices: under Zipf-skewed word
// frequencies the first eighth of the words holds three quarters of the
// entries.  The block's column indices are read once per phase, streamed:
// where col is 16-byte aligned, warp w takes the w-th contiguous share of the
// block's 128-entry slabs (one int4 per lane per slab, four slabs in flight),
// and each lane follows the row of its entries with a cursor that only moves
// forward (one binary search per warp and phase); the few unaligned entries at
// the ends, or all of them otherwise, are placed one by one with a search each.
__global__ void __launch_bounds__(1024) csc_block_fill_kernel(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, int64_t rows, int64_t R, int64_t d,
    const int32_t* __restrict__ colptr, const int32_t* __restrict__ bc, int64_t nnz, int64_t W,
    int64_t quota, int vec, int32_t* __restrict__ rowT, float* __restrict__ valT) {
  extern __shared__ int32_t cur[];
  __shared__ int64_t s_wh;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r1 = r0 + R < rows ? r0 + R : rows;
  const int32_t* off = bc + (int64_t)blockIdx.x * d;
  const int64_t E0 = row_ptr[r0], E1 = row_ptr[r1];
  // aligned body [A0, A1) read as int4, the head and the tail one by one
  int64_t A0 = vec ? (E0 + 3) & ~(int64_t)3 : E1, A1 = vec ? E1 & ~(int64_t)3 : E1;
  if (A0 > A1) A0 = A1 = E1;
  auto row_of = [&](int64_t e) {  // the largest r in [r0, r1) with row_ptr[r] <= e
    int64_t lo = r0, hi = r1 - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if ((int64_t)row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t nslab = (A1 - A0 + 127) >> 7;
  const int64_t s0 = nslab * warp / nw, s1 = nslab * (warp + 1) / nw;
  const int64_t rstart = s0 < s1 ? row_of(A0 + (s0 << 7)) : r0;
  auto place = [&](int64_t e, int32_t w, int64_t wl) {
    const int64_t lo = row_of(e);
    const int32_t pos = atomicAdd(&cur[w - wl], 1);
    if (pos >= 0 && pos < nnz) {  // always, for distinct columns within each row
      rowT[pos] = (int32_t)lo;
      valT[pos] = val[e];
    }
  };
  for (int64_t wl = 0; wl < d;) {
    __syncthreads();  // the previous phase's cursors and s_wh are no longer used
    if (threadIdx.x == 0) {
      // the largest wh <= min(wl + W, d) with colptr[wh] - colptr[wl] <= quota, at least wl + 1
      int64_t lo = wl + 1, hi = wl + W < d ? wl + W : d;
      const int64_t lim = (int64_t)colptr[wl] + quota;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)colptr[mid] <= lim) lo = mid; else hi = mid - 1;
      }
      s_wh = lo;
    }
    __syncthreads();
    const int64_t wh = s_wh;
    for (int64_t w = wl + threadIdx.x; w < wh; w += blockDim.x) cur[w - wl] = colptr[w] + off[w];
    __syncthreads();
    for (int64_t e = E0 + threadIdx.x; e < A0; e += blockDim.x) {
      const int32_t w = __ldcs(col + e);
      if (w >= wl && w < wh) place(e, w, wl);
    }
    for (int64_t e = A1 + threadIdx.x; e < E1; e += blockDim.x) {
      const int32_t w = __ldcs(col + e);
      if (w >= wl && w < wh) place(e, w, wl);
    }
    if (s0 < s1) {
      const int4* c4p = reinterpret_cast<const int4*>(col) + (A0 >> 2);
      const int64_t q1 = (A1 - A0) >> 2;  // int4 of the body
      int64_t r = rstart;                 // row cursor of this lane
      for (int64_t sl = s0; sl < s1; sl += 4) {
        int4 c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t q = (sl + u) * 32 + lane;
          c[u] = (sl + u < s1 && q < q1) ? __ldcs(c4p + q) : make_int4(-1, -1, -1, -1);
        }
        // the values of the matching entries, all loads issued before any is used
        float v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t e = A0 + 4 * ((sl + u) * 32 + lane);
          const int32_t cw[4] = {c[u].x, c[u].y, c[u].z, c[u].w};
#pragma unroll
          for (int j = 0; j < 4; ++j)
            v[u][j] = (cw[j] >= wl && cw[j] < wh) ? __ldcs(val + e + j) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t e = A0 + 4 * ((sl + u) * 32 + lane);
          const int32_t cw[4] = {c[u].x, c[u].y, c[u].z, c[u].w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (cw[j] >= wl && cw[j] < wh) {
              while ((int64_t)row_ptr[r + 1] <= e + j) ++r;
              const int32_t pos = atomicAdd(&cur[cw[j] - wl], 1);
              if (pos >= 0 && pos < nnz) {
                rowT[pos] = (int32_t)r;
                valT[pos] = v[u][j];
              }
            }
          }
        }
      }
    }
    wl = wh;
  }
}

// out[c, :] += alpha * sum_{e in column c} valT[e] * P[rowT[e], :]  (out pre-zeroed),
// P and out with a row stride of ld4 float4, m4 float4 columns.  Warp w takes the
// nonzeros [w kCscChunk, (w + 1) kCscChunk) in column order.
template <int NV>
__global__ void __launch_bounds__(256) spmm_csc_v4_kernel(
    const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowT,
    const float* __restrict__ valT, int64_t d, int64_t nnz, const float4* __restrict__ P,
    int m4, int64_t ld4, float alpha, float4* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t e0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * kCscChunk;
  if (e0 >= nnz) return;
  const int64_t e1 = e0 + kCscChunk < nnz ? e0 + kCscChunk : nnz;
  // the column holding e0: the largest c with colptr[c] <= e0 (it is not empty)
  int64_t lo = 0, hi = d - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (colptr[mid] <= e0) lo = mid; else hi = mid - 1;
  }
  int64_t c = lo, e = e0;
  while (e < e1) {
    const int64_t cb = colptr[c], ce = colptr[c + 1];
    const int64_t se = ce < e1 ? ce : e1;
    float4 acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t base = e; base < se; base += 32) {
      const int cnt = se - base < 32 ? (int)(se - base) : 32;
      int32_t my_r = 0;
      float my_v = 0.f;
      if (lane < cnt) {
        my_r = rowT[base + lane];
        my_v = valT[base + lane];
      }
      // 16 row loads in flight per warp: the P rows (n x m, larger than L2 for the
      // topic whitening) come partly from HBM
#pragma unroll 16
      for (int j = 0; j < cnt; ++j) {
        const int32_t r = __shfl_sync(0xffffffffu, my_r, j);
        const float v = __shfl_sync(0xffffffffu, my_v, j);
        const float4* prow = P + (int64_t)r * ld4;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const int idx = lane + 32 * q;
          if (idx < m4) {
            const float4 b = __ldg(prow + idx);
            acc[q].x = fmaf(v, b.x, acc[q].x);
            acc[q].y = fmaf(v, b.y, acc[q].y);
            acc[q].z = fmaf(v, b.z, acc[q].z);
            acc[q].w = fmaf(v, b.w, acc[q].w);
          }
        }
      }
    }
    const bool whole = cb >= e0 && ce <= e1;  // no other warp touches column c
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int idx = lane + 32 * q;
      if (idx < m4) {
        float4 a = acc[q];
        a.x *= alpha; a.y *= alpha; a.z *= alpha; a.w *= alpha;
        if (whole)
          out[c * ld4 + idx] = a;
        else
          atomicAdd(out + c * ld4 + idx, a);
      }
    }
    e = se;
    ++c;
    while (c < d && colptr[c + 1] <= e) ++c;  // skip empty columns
  }
}

// The same over scalar columns (any m <= 32 NV): lane j holds columns j, j + 32, ...
template <int NV>
__global__ void __launch_bounds__(256) spmm_csc_scalar_kernel(
    const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowT,
    const float* __restrict__ valT, int64_t d, int64_t nnz, const float* __restrict__ P,
    int m, float alpha, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t e0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * kCscChunk;
  if (e0 >= nnz) return;
  const int64_t e1 = e0 + kCscChunk < nnz ? e0 + kCscChunk : nnz;
  int64_t lo = 0, hi = d - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (colptr[mid] <= e0) lo = mid; else hi = mid - 1;
  }
  int64_t c = lo, e = e0;
  while (e < e1) {
    const int64_t cb = colptr[c], ce = colptr[c + 1];
    const int64_t se = ce < e1 ? ce : e1;
    float acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.f;
    for (int64_t base = e; base < se; base += 32) {
      const int cnt = se - base < 32 ? (int)(se - base) : 32;
      int32_t my_r = 0;
      float my_v = 0.f;
      if (lane < cnt) {
        my_r = rowT[base + lane];
        my_v = valT[base + lane];
      }
      for (int j = 0; j < cnt; ++j) {
        const int32_t r = __shfl_sync(0xffffffffu, my_r, j);
        const float v = __shfl_sync(0xffffffffu, my_v, j);
        const float* prow = P + (int64_t)r * m;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const int idx = lane + 32 * q;
          if (idx < m) acc[q] = fmaf(v, __ldg(prow + idx), acc[q]);
        }
      }
    }
    const bool whole = cb >= e0 && ce <= e1;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int idx = lane + 32 * q;
      if (idx < m) {
        if (whole)
          out[c * m + idx] = alpha * acc[q];
        else
          atomicAdd(out + c * m + idx, alpha * acc[q]);
      }
    }
    e = se;
    ++c;
    while (c < d && colptr[c + 1] <= e) ++c;
  }
}

inline unsigned row_blocks(int64_t rows) {
  return (unsigned)((rows + kWarpsPerBlock - 1) / kWarpsPerBlock);
}

}  // namespace

otm_status check_csr(const otm_csr* X, const char* name) {
  if (X == nullptr) return set_error(OTM_EINVAL, "%s: null CSR descriptor", name);
  if (X->rows < 0 || X->cols < 0 || X->nnz < 0)
    return set_error(OTM_EINVAL, "%s: negative size", name);
  if (X->nnz > INT32_MAX) return set_error(OTM_EINVAL, "%s: nnz exceeds int32 range", name);
  if (X->rows > 0 && X->row_ptr == nullptr)
    return set_error(OTM_EINVAL, "%s: null row_ptr", name);
  if (X->nnz > 0 && (X->col == nullptr || X->val == nullptr))
    return set_error(OTM_EINVAL, "%s: null col/val", name);
  if (X->rows >= ((int64_t)1 << 31) / kWarpsPerBlock * kWarpsPerBlock)
    return set_error(OTM_EINVAL, "%s: too many rows", name);
  return OTM_OK;
}

otm_status topic_moments(const otm_csr* X, float* row_invlen, float* row_w, double* M1,
                         double* delta, cudaStream_t st) {
  OTM_CHECK_CUDA(cudaMemsetAsync(M1, 0, sizeof(double) * X->cols, st));
  OTM_CHECK_CUDA(cudaMemsetAsync(delta, 0, sizeof(double) * X->cols, st));
  if (X->rows == 0) return OTM_OK;
  topic_stats_kernel<<<row_blocks(X->rows), 32 * kWarpsPerBlock, 0, st>>>(
      X->row_ptr, X->col, X->val, X->rows, 1.0 / (double)X->rows, row_invlen, row_w, M1, delta);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status column_sums_scaled(const otm_csr* X, double scale, double* out, cudaStream_t st) {
  OTM_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * X->cols, st));
  if (X->rows == 0) return OTM_OK;
  column_sums_kernel<<<row_blocks(X->rows), 32 * kWarpsPerBlock, 0, st>>>(
      X->row_ptr, X->col, X->val, X->rows, scale, out);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status spmm_gather(const otm_csr* X, const float* B, int64_t m, const float* row_scale,
                       float* out, cudaStream_t st) {
  if (X->rows == 0 || m == 0) return OTM_OK;
  const unsigned g = row_blocks(X->rows);
  const int T = 32 * kWarpsPerBlock;
  if (m % 4 == 0 && m <= 384 && aligned16(B) && aligned16(out)) {
    const int m4 = (int)(m / 4);
    auto* B4 = reinterpret_cast<const float4*>(B);
    auto* O4 = reinterpret_cast<float4*>(out);
    if (m4 <= 32)
      spmm_gather_v4_kernel<1><<<g, T, 0, st>>>(X->row_ptr, X->col, X->val, X->rows, B4, m4,
                                                row_scale, O4);
    else if (m4 <= 64)
      spmm_gather_v4_kernel<2><<<g, T, 0, st>>>(X->row_ptr, X->col, X->val, X->rows, B4, m4,
                                                row_scale, O4);
    else
      spmm_gather_v4_kernel<3><<<g, T, 0, st>>>(X->row_ptr, X->col, X->val, X->rows, B4, m4,
                                                row_scale, O4);
  } else {
    spmm_gather_scalar_kernel<<<g, T, 0, st>>>(X->row_ptr, X->col, X->val, X->rows, B, m,
                                               row_scale, out);
  }
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

otm_status spmm_scatter(const otm_csr* X, const float* P, int64_t m, const float* row_scale,
                        float alpha, float* out, cudaStream_t st) {
  if (X->rows == 0 || m == 0) return OTM_OK;
  const unsigned g = row_blocks(X->rows);
  const int T = 32 * kWarpsPerBlock;
  if (m % 4 == 0 && m <= 384 && aligned16(P) && aligned16(out)) {
    const int m4 = (int)(m / 4);
    auto* P4 = reinterpret_cast<const float4*>(P);
    auto* O4 = reinterpret_cast<float4*>(out);
    if (m4 <= 32)
      spmm_scatter_v4_kernel<1><<<g, T, 0, st>>>(X->row_ptr, X->col, X->val, X->rows, P4, m4,
                                                 row_scale, alpha, O4);
    else if (m4 <= 64)
      spmm_scatter_v4_kernel<2><<<g, T, 0, st>>>(X->row_ptr, X->col, X->val, X->rows, P4, m4,
                                                 row_scale, alpha, O4);
    else
      spmm_scatter_v4_kernel<3><<<g, T, 0, st>>>(X->row_ptr, X->col, X->val, X->rows, P4, m4,
                                                 row_scale, alpha, O4);
  } else {
    spmm_scatter_scalar_kernel<<<g, T, 0, st>>>(X->row_ptr, X->col, X->val, X->rows, P, m,
                                                row_scale, alpha, out);
  }
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

int smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

int64_t csc_block_rows(int64_t n) {
  const int64_t r = (n + 1023) / 1024;  // at most 1,024 row blocks
  return r < 2048 ? 2048 : (r > 65535 ? 65535 : r);
}

bool csc_blocked_fits(int64_t n, int64_t d) {
  if (n > 1024 * 65535) return false;
  return (size_t)((d + 1) / 2) * 4 + 1024 <= (size_t)smem_optin();
}

size_t csr_transpose_workspace(int64_t n, int64_t d) {
  WorkspaceSize w;
  w.add<int32_t>(d > 0 ? d : 1);
  if (csc_blocked_fits(n, d)) w.add<int32_t>(((n + csc_block_rows(n) - 1) / csc_block_rows(n)) * d);
  return w.bytes();
}

otm_status csr_transpose(const otm_csr* X, int32_t* colptr, int32_t* rowT, float* valT,
                         void* scratch, cudaStream_t st) {
  const int64_t d = X->cols, nnz = X->nnz, n = X->rows;
  int32_t* cursor = static_cast<int32_t*>(scratch);
  int32_t* bc = reinterpret_cast<int32_t*>(static_cast<uint8_t*>(scratch) +
                                           ((sizeof(int32_t) * (d > 0 ? d : 1) + 255) & ~size_t(255)));
  if (n > 0 && d > 0 && nnz > 0 && csc_blocked_fits(n, d)) {
    const int64_t R = csc_block_rows(n), nb = (n + R - 1) / R;
    const size_t smem = (size_t)((d + 1) / 2) * 4;
    OTM_CHECK_CUDA(cudaFuncSetAttribute(csc_block_count_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    csc_block_count_kernel<<<(unsigned)nb, 1024, smem, st>>>(X->row_ptr, X->col, n, R, d, bc);
    OTM_CHECK_LAUNCH();
    csc_block_scan_kernel<<<(unsigned)((d + 255) / 256), 256, 0, st>>>(bc, nb, d, cursor);
    OTM_CHECK_LAUNCH();
    exclusive_scan_kernel<<<1, 1024, 0, st>>>(cursor, d, colptr, cursor);
    OTM_CHECK_LAUNCH();
    // word ranges of at most 96 MB of output (8 bytes per entry) and 49,152 cursors
    const int64_t W = d < 49152 ? d : 49152, quota = (96ll << 20) / 8;
    const int vec = (reinterpret_cast<uintptr_t>(X->col) & 15) == 0;
    const size_t fsmem = (size_t)W * sizeof(int32_t);
    OTM_CHECK_CUDA(cudaFuncSetAttribute(csc_block_fill_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    csc_block_fill_kernel<<<(unsigned)nb, 1024, fsmem, st>>>(X->row_ptr, X->col, X->val, n, R, d,
                                                             colptr, bc, nnz, W, quota, vec,
                                                             rowT, valT);
    OTM_CHECK_LAUNCH();
    return OTM_OK;
  }
  OTM_CHECK_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (d > 0 ? d : 1), st));
  if (nnz > 0) {
    const int64_t g = (nnz + 255) / 256 < 4096 ? (nnz + 255) / 256 : 4096;
    csc_count_kernel<<<(unsigned)g, 256, 0, st>>>(X->col, nnz, cursor);
    OTM_CHECK_LAUNCH();
  }
  exclusive_scan_kernel<<<1, 1024, 0, st>>>(cursor, d, colptr, cursor);
  OTM_CHECK_LAUNCH();
  if (X->rows > 0 && nnz > 0) {
    csc_fill_kernel<<<row_blocks(X->rows), 32 * kWarpsPerBlock, 0, st>>>(
        X->row_ptr, X->col, X->val, X->rows, cursor, rowT, valT);
    OTM_CHECK_LAUNCH();
  }
  return OTM_OK;
}

otm_status topic_moments_csc(const otm_csr* X, const int32_t* colptr, const int32_t* rowT,
                             const float* valT, double* wa, double* wb, float* row_invlen,
                             float* row_w, double* M1, double* delta, cudaStream_t st) {
  OTM_CHECK_CUDA(cudaMemsetAsync(M1, 0, sizeof(double) * X->cols, st));
  OTM_CHECK_CUDA(cudaMemsetAsync(delta, 0, sizeof(double) * X->cols, st));
  if (X->rows == 0) return OTM_OK;
  topic_rows_kernel<<<row_blocks(X->rows), 32 * kWarpsPerBlock, 0, st>>>(
      X->row_ptr, X->val, X->rows, 1.0 / (double)X->rows, wa, wb, row_invlen, row_w);
  OTM_CHECK_LAUNCH();
  if (X->cols > 0 && X->nnz > 0) {
    const int64_t warps = (X->nnz + kCscChunk - 1) / kCscChunk;
    topic_cols_kernel<<<(unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock),
                        32 * kWarpsPerBlock, 0, st>>>(colptr, rowT, valT, X->cols, X->nnz, wa,
                                                      wb, M1, delta);
    OTM_CHECK_LAUNCH();
  }
  return OTM_OK;
}

otm_status spmm_csc(const int32_t* colptr, const int32_t* rowT, const float* valT, int64_t d,
                    int64_t nnz, const float* P, int64_t m, float alpha, float* out,
                    cudaStream_t st) {
  OTM_REQUIRE(m <= 384, "spmm_csc: m=%lld > 384", (long long)m);
  if (nnz == 0 || m == 0 || d == 0) return OTM_OK;
  const int64_t warps = (nnz + kCscChunk - 1) / kCscChunk;
  const unsigned g = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
  const int T = 32 * kWarpsPerBlock;
  if (m % 4 != 0 || !aligned16(P) || !aligned16(out)) {
    const int mi = (int)m;
    if (m <= 32)
      spmm_csc_scalar_kernel<1><<<g, T, 0, st>>>(colptr, rowT, valT, d, nnz, P, mi, alpha, out);
    else if (m <= 64)
      spmm_csc_scalar_kernel<2><<<g, T, 0, st>>>(colptr, rowT, valT, d, nnz, P, mi, alpha, out);
    else if (m <= 128)
      spmm_csc_scalar_kernel<4><<<g, T, 0, st>>>(colptr, rowT, valT, d, nnz, P, mi, alpha, out);
    else
      spmm_csc_scalar_kernel<12><<<g, T, 0, st>>>(colptr, rowT, valT, d, nnz, P, mi, alpha, out);
    OTM_CHECK_LAUNCH();
    return OTM_OK;
  }
  const int m4 = (int)(m / 4);
  auto* P4 = reinterpret_cast<const float4*>(P);
  auto* O4 = reinterpret_cast<float4*>(out);
  if (m4 <= 32)
    spmm_csc_v4_kernel<1><<<g, T, 0, st>>>(colptr, rowT, valT, d, nnz, P4, m4, m4, alpha, O4);
  else if (m4 <= 64)
    spmm_csc_v4_kernel<2><<<g, T, 0, st>>>(colptr, rowT, valT, d, nnz, P4, m4, m4, alpha, O4);
  else
    spmm_csc_v4_kernel<3><<<g, T, 0, st>>>(colptr, rowT, valT, d, nnz, P4, m4, m4, alpha, O4);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

}  // namespace otm
