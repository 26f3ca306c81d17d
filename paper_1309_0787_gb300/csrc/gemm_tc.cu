// Batched BF16 GEMM on the fifth-generation tensor cores:
//   C[z] = alpha * A[z] B[z]^T   (A: M x K, B: N x K, both row-major = K-major)
// with FP32 accumulation in tensor memory and a fused epilogue (bias, GELU).
// It serves the dense products of the learned warm start (the MLP's forward
// and backward passes).
//
// One CTA computes a 128 x 128 tile of C.  Warp 0 streams 128 x 64 tiles of A
// and B into a four-stage shared-memory ring with TMA (cp.async.bulk.tensor);
// warp 1 issues tcgen05.mma (M = 128, N = 128, K = 16) into a 128-column TMEM
// accumulator and releases each stage with tcgen05.commit; warps 2-5 (one per
// 32-lane TMEM quarter) wait for the final commit, read the accumulator with
// tcgen05.ld and apply the epilogue.
//
// Shared-memory layout of a 128 x 64 operand tile: eight K-chunks of 8
// elements; chunk c holds the 128 rows x 16 bytes at c * 2048, i.e. core
// matrices (8 rows x 16 B) 128 B apart along M and 2048 B apart along K.  One
// TMA box of 8 x 128 elements fills one chunk.
#include <cudaTypedefs.h>

#include <mutex>

#include "otm_internal.cuh"
#include "tc_ptx.cuh"

namespace otm {
namespace {

using namespace tc;

constexpr int GM = 128, GN = 128, GK = 64, GSTAGES = 4;
constexpr int GEMM_THREADS = 192;
constexpr uint32_t G_TILE_BYTES = GM * GK * 2;  // 16 KiB per operand per stage
constexpr uint32_t G_STAGE_BYTES = 2 * G_TILE_BYTES;
constexpr size_t G_SMEM = (size_t)GSTAGES * G_STAGE_BYTES + 1024;

struct GemmEpi {
  int mode;
  float alpha;
  const float* bias;
  float* C;
  int64_t ldc, strideC;
  __nv_bfloat16* H;
  int64_t ldh, strideH;
};

__device__ __forceinline__ float gelu_exact(float z) {
  return 0.5f * z * (1.f + erff(z * 0.70710678118654752f));
}

__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gemm_bf16_nt_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                        int M, int N, int K, GemmEpi ep, int* err) {
  extern __shared__ __align__(1024) uint8_t gsm_raw[];
  uint8_t* gsm = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[GSTAGES];
  __shared__ __align__(8) uint64_t empty[GSTAGES];
  __shared__ __align__(8) uint64_t accb;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  __shared__ int s_issued, s_consumed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN, z = blockIdx.z;
  const int nk = (K + GK - 1) / GK;

  if (warp == 1) tmem_alloc(&tmem_base, GN);
  if (tid == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accb, 1);
    mbar_fence_init();
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
    tma_prefetch_desc(&ta);
    tma_prefetch_desc(&tb);
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      int kb = 0;
      for (; kb < nk; ++kb) {
        const int s = kb % GSTAGES;
        if (kb >= GSTAGES &&
            !mbar_wait_or_abort(&empty[s], ((kb / GSTAGES) - 1) & 1, &s_abort)) {
          s_abort = 1;
          break;
        }
        uint8_t* As = gsm + (size_t)s * G_STAGE_BYTES;
        uint8_t* Bs = As + G_TILE_BYTES;
        mbar_expect_tx(&full[s], G_STAGE_BYTES);
#pragma unroll
        for (int c = 0; c < GK / 8; ++c) {
          tma_load_3d(As + c * 2048, &ta, &full[s], kb * GK + c * 8, m0, z);
          tma_load_3d(Bs + c * 2048, &tb, &full[s], kb * GK + c * 8, n0, z);
        }
      }
      s_issued = kb;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(1, 0, 0, GM, GN);
      int kb = 0;
      for (; kb < nk; ++kb) {
        const int s = kb % GSTAGES;
        if (!mbar_wait_or_abort(&full[s], (kb / GSTAGES) & 1, &s_abort)) {
          s_abort = 1;
          break;
        }
        tc_after();
        const uint8_t* As = gsm + (size_t)s * G_STAGE_BYTES;
        const uint8_t* Bs = As + G_TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < GK / 16; ++kk) {
          const uint64_t ad = sdesc(As + kk * 2 * 2048, 2048, 128);
          const uint64_t bd = sdesc(Bs + kk * 2 * 2048, 2048, 128);
          mma<false>(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&empty[s]);
      }
      s_consumed = kb;
      mma_commit(&accb);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = tile rows
    const int quarter = warp & 3;
    const int row = m0 + quarter * 32 + lane;
    const bool ok = mbar_wait_or_abort(&accb, 0, &s_abort);
    if (!ok && lane == 0) s_abort = 1;
    tc_after();
    if (ok) {
      float* crow = ep.C ? ep.C + (int64_t)z * ep.strideC + (int64_t)row * ep.ldc : nullptr;
      __nv_bfloat16* hrow =
          ep.H ? ep.H + (int64_t)z * ep.strideH + (int64_t)row * ep.ldh : nullptr;
      for (int cb = 0; cb < GN; cb += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb, v);
        if (row < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = n0 + cb + j;
            if (col < N) {
              float x = v[j] * ep.alpha;
              if (ep.mode >= 1 && ep.bias) x += ep.bias[col];
              if (ep.mode == 2) {
                if (crow) crow[col] = x;
                hrow[col] = __float2bfloat16_rn(gelu_exact(x));
              } else {
                if (crow) crow[col] = x;
                if (hrow) hrow[col] = __float2bfloat16_rn(x);
              }
            }
          }
        }
      }
    }
  }
  tc_before();
  __syncthreads();
  if (tid == 0 && s_abort) {
    atomicExch(err, 1);
    // wait (bounded) for TMA copies that were issued but never consumed
    for (int kb = s_consumed; kb < s_issued; ++kb)
      mbar_wait(&full[kb % GSTAGES], (kb / GSTAGES) & 1);
  }
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, GN);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

otm_status get_encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  });
  if (!g_encode) return set_error(OTM_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  *out = g_encode;
  return OTM_OK;
}

// 3-D map over a batch of row-major BF16 matrices (rows x K, leading dimension
// ld elements, batch stride bs elements) with an 8 x 128 x 1 box.
otm_status make_map(CUtensorMap* map, const void* base, int64_t K, int64_t rows, int64_t batch,
                    int64_t ld, int64_t bs) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  OTM_TRY(get_encoder(&enc));
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)(batch > 1 ? bs : rows * ld) * 2};
  const cuuint32_t box[3] = {8, 128, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(OTM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return OTM_OK;
}

// Sets the kernel's shared-memory limit once per device.
otm_status configure_gemm() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  OTM_CHECK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return OTM_OK;
  OTM_CHECK_CUDA(cudaFuncSetAttribute(gemm_bf16_nt_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G_SMEM));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return OTM_OK;
}

}  // namespace

otm_status gemm_bf16_nt(const void* A, const void* B, int64_t M, int64_t N, int64_t K,
                        int64_t batch, int64_t lda, int64_t ldb, int64_t sA, int64_t sB, int mode,
                        float alpha, const float* bias, float* C, int64_t ldc, int64_t sC, void* H,
                        int64_t ldh, int64_t sH, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return OTM_OK;
  if (K <= 0 || (K % 8) != 0 || (lda % 8) != 0 || (ldb % 8) != 0 || lda < K || ldb < K ||
      (batch > 1 && ((sA % 8) != 0 || (sB % 8) != 0)))
    return set_error(OTM_EINVAL,
                     "gemm_bf16: K, lda, ldb (and batch strides) must be multiples of 8, lda, ldb >= K");
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
    return set_error(OTM_EINVAL, "gemm_bf16: A and B must be 16-byte aligned");
  if (M > (int64_t)1 << 30 || N > (int64_t)1 << 30 || K > (int64_t)1 << 30 || batch > 65535)
    return set_error(OTM_EINVAL, "gemm_bf16: size too large");
  if (mode < 0 || mode > 2 || (mode == 2 && !H) || (!C && !H))
    return set_error(OTM_EINVAL, "gemm_bf16: bad epilogue");
  CUtensorMap ta, tb;
  OTM_TRY(make_map(&ta, A, K, M, batch, lda, sA));
  OTM_TRY(make_map(&tb, B, K, N, batch, ldb, sB));
  OTM_TRY(configure_gemm());
  GemmEpi ep;
  ep.mode = mode;
  ep.alpha = alpha;
  ep.bias = bias;
  ep.C = C;
  ep.ldc = ldc;
  ep.strideC = sC;
  ep.H = static_cast<__nv_bfloat16*>(H);
  ep.ldh = ldh;
  ep.strideH = sH;
  const dim3 grid((unsigned)((M + GM - 1) / GM), (unsigned)((N + GN - 1) / GN), (unsigned)batch);
  gemm_bf16_nt_kernel<<<grid, GEMM_THREADS, G_SMEM, st>>>(ta, tb, (int)M, (int)N, (int)K, ep, err);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

}  // namespace otm

using namespace otm;

extern "C" {

size_t otm_gemm_bf16_workspace(void) { return 256; }

otm_status otm_gemm_bf16(const void* A, const void* B, int64_t M, int64_t N, int64_t K,
                         int64_t batch, int64_t lda, int64_t ldb, int64_t strideA, int64_t strideB,
                         int epilogue, float alpha, const float* bias, float* C, int64_t ldc,
                         int64_t strideC, void* H, int64_t ldh, int64_t strideH, void* ws,
                         size_t ws_bytes, void* stream) {
  clear_error();
  OTM_REQUIRE(A && B, "otm_gemm_bf16: null operand");
  OTM_REQUIRE(ws && ws_bytes >= otm_gemm_bf16_workspace(), "otm_gemm_bf16: workspace too small");
  cudaStream_t st = as_stream(stream);
  int* err = static_cast<int*>(ws);
  OTM_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  return gemm_bf16_nt(A, B, M, N, K, batch, lda, ldb, strideA, strideB, epilogue, alpha, bias, C,
                      ldc, strideC, H, ldh, strideH, err, st);
}

}  // extern "C"
