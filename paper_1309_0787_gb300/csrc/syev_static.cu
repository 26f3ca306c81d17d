// otm_syev_noalloc: the FP64 symmetric eigendecomposition of otm_syev for
// callers that cannot allocate device memory.
//
// Some callers have no way to hand the library a workspace: a host that runs
// inside another framework whose memory pool already owns the GPU's memory, a
// plugin interface that passes only input and output pointers, or a
// latency-critical loop that must not call cudaMalloc / cudaFree because both
// synchronise the whole device.  This entry point takes its scratch from a
// fixed array compiled into the library instead: the caller passes only A and
// the outputs, and the call allocates nothing (no cudaMalloc, no cudaFree, no
// allocating library routine).
//
// The array is a file-scope __device__ variable, so every GPU on which the
// library is loaded holds its SCRATCH_BYTES until the process exits, and every
// call on that GPU uses the same bytes.
#include <mutex>

#include "otm_internal.cuh"

namespace otm {
namespace {

constexpr int64_t NOALLOC_MAX_N = 160;
constexpr size_t SCRATCH_BYTES = size_t(2) << 20;  // 2 MiB; n = 160 needs about 1.88 MB
constexpr int MAX_DEVICES = 64;

// Device scratch of otm_syev_noalloc.  In host code this name only stands for
// the device variable: its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_syev_scratch[SCRATCH_BYTES];

std::mutex g_setup_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
otm_status scratch_address(void** out) {
  int dev = -1;
  OTM_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES)
    return set_error(OTM_EINVAL, "otm_syev_noalloc: device %d outside [0, %d)", dev, MAX_DEVICES);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_syev_scratch);
    if (e != cudaSuccess || !p)
      return set_error(OTM_ECUDA, "otm_syev_noalloc: cudaGetSymbolAddress failed on device %d: %s",
                       dev, cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return OTM_OK;
}

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

otm_status otm_syev_noalloc(const double* A, int64_t n, double* evals, double* evecs,
                            void* stream) {
  clear_error();
  OTM_REQUIRE(A && evals && evecs, "otm_syev_noalloc: null pointer");
  OTM_REQUIRE(n >= 1 && n <= NOALLOC_MAX_N,
              "otm_syev_noalloc: n=%lld outside [1, %lld] (the fixed scratch array holds the "
              "workspace of n <= %lld; use otm_syev with a caller workspace for larger n)",
              (long long)n, (long long)NOALLOC_MAX_N, (long long)NOALLOC_MAX_N);
  const size_t need = otm_syev_workspace(n);
  OTM_REQUIRE(need <= SCRATCH_BYTES, "otm_syev_noalloc: n=%lld needs %zu scratch bytes > %zu",
              (long long)n, need, SCRATCH_BYTES);
  void* base = nullptr;
  OTM_TRY(scratch_address(&base));
  cudaStream_t st = as_stream(stream);
  Workspace w(base, SCRATCH_BYTES);
  // the array keeps the previous call's bytes: the failure flag must start at
  // zero; every other scratch value is written before it is read
  int* flag = w.take<int>(1);
  OTM_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  OTM_TRY(syev(A, n, evals, evecs, w, st, flag));
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h)
    return set_error(OTM_ENOTCONVERGED, "otm_syev_noalloc: non-finite eigenvalues or refinement failure");
  return OTM_OK;
}

}  // extern "C"
