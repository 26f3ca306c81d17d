// Sparse kernels over CSR count data: per-document statistics and first
// moments (Section 2.1 Eq. (1), the diagonal term of Eq. (2); Section 2.2
// Eq. (9)), and the two sparse-dense products the method is built from:
//   gather  SpMM  out = diag(s) X B        (projection y_t = W^T c_t, Section 3.1;
//                                            the X S half of M2 S, Section 4.2)
//   scatter SpMM  out += X^T diag(s) P     (the X^T half of M2 S and Pairs S)
// One warp per CSR row; the dense rows move as float4 (coalesced 16-byte
// loads), the row's (col, val) pairs are loaded once per warp and broadcast
// with shuffles.
#include "otm_internal.cuh"

namespace otm {
namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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

}  // namespace otm
