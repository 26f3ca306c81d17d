// Post-processing (Section 3.3, Lemma 4) and the reconstruction error used to
// measure convergence, both in FP64.
//   lambda_i = kappa ||v_i||^3,  mu_i = lambda_i (W^T)^+ v_i / ||v_i||,
//   (W^T)^+ = Q Cp kept in factored form, so mu = Q (Cp U diag(lambda)).
//   alpha_hat_i = lambda_i^-2 / sum_j lambda_j^-2.
// Error: || kappa sum v_i^(x)3 - sum lam_j u_j^(x)3 ||_F / || sum lam_j u_j^(x)3 ||_F
// from Gram matrices, using <x^(x)3, y^(x)3> = <x, y>^3.
#include "otm_internal.cuh"

namespace otm {
namespace {

__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)((blockDim.x + 31) / 32); ++i) t += red[i];
  return t;  // valid in thread 0
}

// Block i: norm of v_i, lambda_i, and column i of M = Cp U diag(lambda) (kt x k).
__global__ void unwhiten_cols_kernel(const float* __restrict__ V, int64_t k,
                                     const double* __restrict__ Cp, int64_t kt, double kappa,
                                     double* __restrict__ M, double* __restrict__ lambda) {
  __shared__ double red[32];
  __shared__ double s_scale;
  const int64_t i = blockIdx.x;
  double nn = 0.0;
  for (int64_t r = threadIdx.x; r < k; r += blockDim.x) {
    const double v = V[i * k + r];
    nn += v * v;
  }
  const double tot = block_sum(nn, red);
  if (threadIdx.x == 0) {
    const double norm = sqrt(tot);
    const double lam = kappa * norm * norm * norm;
    lambda[i] = lam;
    s_scale = norm > 0.0 ? lam / norm : 0.0;
  }
  __syncthreads();
  const double sc = s_scale;
  for (int64_t j = threadIdx.x; j < kt; j += blockDim.x) {
    double acc = 0.0;
    for (int64_t r = 0; r < k; ++r) acc = fma(Cp[j * k + r], (double)V[i * k + r], acc);
    M[j * k + i] = sc * acc;
  }
}

__global__ void alpha_hat_kernel(const double* __restrict__ lambda, int64_t k,
                                 double* __restrict__ alpha_hat) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) s += 1.0 / (lambda[i] * lambda[i]);
  const double tot = block_sum(s, red);
  __shared__ double s_tot;
  if (threadIdx.x == 0) s_tot = tot;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x)
    alpha_hat[i] = 1.0 / (lambda[i] * lambda[i]) / s_tot;
}

__global__ void colsum_f64_kernel(const double* __restrict__ A, int64_t rows, int64_t k,
                                  double* __restrict__ out) {
  const int64_t r0 = (int64_t)blockIdx.x * 64, r1 = min(rows, r0 + 64);
  for (int64_t j = threadIdx.x; j < k; j += blockDim.x) {
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) acc += A[r * k + j];
    atomicAdd(&out[j], acc);
  }
}

// A[:, j] /= s[j] (s[j] = 0: unchanged), as a multiply by the reciprocal (one
// FP64 division per column and block, not per entry); blocks take 64 rows at a
// time, so that the column of an entry is a 32-bit remainder.
__global__ void __launch_bounds__(256) divide_cols_kernel(double* __restrict__ A, int64_t rows,
                                                          int64_t k, const double* __restrict__ s) {
  extern __shared__ double rinv[];
  for (int64_t j = threadIdx.x; j < k; j += blockDim.x) rinv[j] = s[j] != 0.0 ? 1.0 / s[j] : 1.0;
  __syncthreads();
  const int kk = (int)k;
  for (int64_t r0 = (int64_t)blockIdx.x * 64; r0 < rows; r0 += (int64_t)gridDim.x * 64) {
    const int64_t r1 = r0 + 64 < rows ? r0 + 64 : rows;
    const int cnt = (int)((r1 - r0) * k);
    double* base = A + r0 * k;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) base[e] *= rinv[e % kk];
  }
}

// Block i: row i of the three Gram matrices -> partial sums of the error terms.
__global__ void recon_rows_kernel(const float* __restrict__ V, int64_t k,
                                  const double* __restrict__ U, const double* __restrict__ lam,
                                  double* __restrict__ part) {
  __shared__ double red[32];
  const int64_t i = blockIdx.x;
  double hh = 0.0, ht = 0.0, tt = 0.0;
  for (int64_t j = threadIdx.x; j < k; j += blockDim.x) {
    double vv = 0.0, vu = 0.0, uu = 0.0;
    for (int64_t r = 0; r < k; ++r) {
      const double vi = V[i * k + r];
      vv = fma(vi, (double)V[j * k + r], vv);
      vu = fma(vi, U[j * k + r], vu);
      uu = fma(U[i * k + r], U[j * k + r], uu);
    }
    hh += vv * vv * vv;
    ht += vu * vu * vu * lam[j];
    tt += uu * uu * uu * lam[i] * lam[j];
  }
  const double a = block_sum(hh, red);
  const double b = block_sum(ht, red);
  const double c = block_sum(tt, red);
  if (threadIdx.x == 0) {
    part[3 * i] = a;
    part[3 * i + 1] = b;
    part[3 * i + 2] = c;
  }
}

__global__ void recon_final_kernel(const double* __restrict__ part, int64_t k, double kappa,
                                   double* __restrict__ err) {
  if (threadIdx.x != 0) return;
  double hh = 0.0, ht = 0.0, tt = 0.0;
  for (int64_t i = 0; i < k; ++i) {
    hh += part[3 * i];
    ht += part[3 * i + 1];
    tt += part[3 * i + 2];
  }
  const double num = kappa * kappa * hh - 2.0 * kappa * ht + tt;
  // a rounding-negative num is zero; a non-finite V (a diverged run) gives NaN
  *err = isfinite(hh) && isfinite(ht) ? sqrt((num < 0.0 ? 0.0 : num) / tt) : nan("");
}

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

size_t otm_unwhiten_workspace(int64_t d, int64_t k, int64_t kt) {
  (void)d;
  WorkspaceSize w;
  w.add<double>(kt * k).add<double>(k);
  return w.bytes();
}

otm_status otm_unwhiten(const float* V, int64_t k, const float* Q, int64_t d, int64_t kt,
                        const double* Cp, double theta, int normalize, double* comps,
                        double* lambda, double* alpha_hat, void* ws, size_t ws_bytes,
                        void* stream) {
  clear_error();
  OTM_REQUIRE(V && Q && Cp && comps && lambda && alpha_hat, "otm_unwhiten: null pointer");
  OTM_REQUIRE(k >= 1 && kt >= k && d >= 1, "otm_unwhiten: need 1 <= k <= kt, d >= 1");
  OTM_REQUIRE(ws_bytes >= otm_unwhiten_workspace(d, k, kt), "otm_unwhiten: workspace too small");
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  double* M = w.take<double>(kt * k);
  double* csum = w.take<double>(k);
  const double kappa = 0.5 * (1.0 + theta);
  unwhiten_cols_kernel<<<(unsigned)k, 128, 0, st>>>(V, k, Cp, kt, kappa, M, lambda);
  OTM_CHECK_LAUNCH();
  alpha_hat_kernel<<<1, 256, 0, st>>>(lambda, k, alpha_hat);
  OTM_CHECK_LAUNCH();
  OTM_TRY(gemm_nn_f64(Q, d, kt, M, k, comps, st));
  if (normalize) {
    OTM_CHECK_CUDA(cudaMemsetAsync(csum, 0, sizeof(double) * k, st));
    colsum_f64_kernel<<<(unsigned)((d + 63) / 64), 128, 0, st>>>(comps, d, k, csum);
    OTM_CHECK_LAUNCH();
    const int64_t rb = (d + 63) / 64;
    divide_cols_kernel<<<(unsigned)(rb < 152 * 4 ? rb : 152 * 4), 256, sizeof(double) * k, st>>>(
        comps, d, k, csum);
    OTM_CHECK_LAUNCH();
  }
  return OTM_OK;
}

size_t otm_recon_error_workspace(int64_t k) {
  WorkspaceSize w;
  w.add<double>(3 * k);
  return w.bytes();
}

otm_status otm_recon_error(const float* V, int64_t k, double theta, const double* U_true,
                           const double* lam_true, double* err, void* ws, size_t ws_bytes,
                           void* stream) {
  clear_error();
  OTM_REQUIRE(V && U_true && lam_true && err && k >= 1, "otm_recon_error: bad arguments");
  OTM_REQUIRE(ws_bytes >= otm_recon_error_workspace(k), "otm_recon_error: workspace too small");
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  double* part = w.take<double>(3 * k);
  recon_rows_kernel<<<(unsigned)k, 128, 0, st>>>(V, k, U_true, lam_true, part);
  OTM_CHECK_LAUNCH();
  recon_final_kernel<<<1, 32, 0, st>>>(part, k, 0.5 * (1.0 + theta), err);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

}  // extern "C"
