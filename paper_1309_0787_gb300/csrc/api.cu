// C ABI: error reporting, argument validation and the thin entry points that
// forward to one kernel family (moments, projection, means, QR, eigensolver).
#include <stdarg.h>
#include <stdio.h>

#include <atomic>

#include "otm_internal.cuh"

namespace otm {
namespace {

thread_local char g_err[512] = {0};
std::atomic<uint64_t> g_launches{0};

// ybar[j] = (1/n) sum_t Y[t, j]; row blocks of 512, per column a compensated
// float32 sum (Knuth's TwoSum: the rounding error of every addition kept in a
// second float, about 2^-48 relative on the FP32 units), added in FP64 with
// FP64 atomics.
__global__ void column_mean_kernel(const float* __restrict__ Y, int64_t n, int64_t k,
                                   double inv_n, double* __restrict__ ybar) {
  const int64_t r0 = (int64_t)blockIdx.x * 512, r1 = min(n, r0 + 512);
  for (int64_t j = threadIdx.x; j < k; j += blockDim.x) {
    float h = 0.f, l = 0.f;
#pragma unroll 8
    for (int64_t r = r0; r < r1; ++r) {
      const float y = Y[r * k + j];
      const float s = __fadd_rn(h, y);
      const float bv = __fsub_rn(s, h);
      l = __fadd_rn(l, __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(y, bv)));
      h = s;
    }
    atomicAdd(&ybar[j], ((double)h + (double)l) * inv_n);
  }
}

}  // namespace

otm_status set_error(otm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

void clear_error() { g_err[0] = 0; }

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace otm

using namespace otm;

extern "C" {

int otm_version(void) { return 100; }

const char* otm_last_error(void) { return g_err; }

uint64_t otm_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

otm_status otm_topic_moments(const otm_csr* X, float* row_invlen, float* row_w, double* M1,
                             double* delta, void* stream) {
  clear_error();
  OTM_TRY(check_csr(X, "otm_topic_moments"));
  OTM_REQUIRE(X->rows == 0 || (row_invlen && row_w), "otm_topic_moments: null row outputs");
  OTM_REQUIRE(X->cols == 0 || (M1 && delta), "otm_topic_moments: null column outputs");
  return topic_moments(X, row_invlen, row_w, M1, delta, as_stream(stream));
}

otm_status otm_project(const otm_csr* X, const float* W, int64_t k, const float* row_scale,
                       float* Y, void* stream) {
  clear_error();
  OTM_TRY(check_csr(X, "otm_project"));
  OTM_REQUIRE(k >= 1, "otm_project: k must be >= 1");
  OTM_REQUIRE(X->rows == 0 || (W && Y), "otm_project: null W or Y");
  return spmm_gather(X, W, k, row_scale, Y, as_stream(stream));
}

otm_status otm_column_mean(const float* Y, int64_t n, int64_t k, double* ybar, void* stream) {
  clear_error();
  OTM_REQUIRE(n >= 1 && k >= 1 && Y && ybar, "otm_column_mean: bad arguments");
  cudaStream_t st = as_stream(stream);
  OTM_CHECK_CUDA(cudaMemsetAsync(ybar, 0, sizeof(double) * k, st));
  column_mean_kernel<<<(unsigned)((n + 511) / 512), 128, 0, st>>>(Y, n, k, 1.0 / (double)n, ybar);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

size_t otm_orth_workspace(int64_t m) { return orth_workspace(m) + 256; }

otm_status otm_orthonormalize(float* A, int64_t rows, int64_t m, void* ws, size_t ws_bytes,
                              void* stream) {
  clear_error();
  OTM_REQUIRE(A && m >= 1 && m <= 160 && rows >= m,
              "otm_orthonormalize: need A != NULL, 1 <= m <= 160, rows >= m");
  OTM_REQUIRE(ws_bytes >= otm_orth_workspace(m), "otm_orthonormalize: workspace too small");
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  int* flag = w.take<int>(1);
  OTM_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  OTM_TRY(orthonormalize(A, rows, m, w, st, flag));
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h) return set_error(OTM_ENOTCONVERGED, "otm_orthonormalize: non-finite Gram matrix");
  return OTM_OK;
}

size_t otm_syev_workspace(int64_t n) { return syev_workspace(n) + 256; }

otm_status otm_syev(const double* A, int64_t n, double* evals, double* evecs, void* ws,
                    size_t ws_bytes, void* stream) {
  clear_error();
  OTM_REQUIRE(A && evals && evecs && n >= 1 && n <= 160,
              "otm_syev: need non-null arguments and 1 <= n <= 160");
  OTM_REQUIRE(ws_bytes >= otm_syev_workspace(n), "otm_syev: workspace too small");
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  int* flag = w.take<int>(1);
  OTM_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  OTM_TRY(syev(A, n, evals, evecs, w, st, flag));
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h)
    return set_error(OTM_ENOTCONVERGED, "otm_syev: non-finite eigenvalues or refinement failure");
  return OTM_OK;
}

}  // extern "C"
