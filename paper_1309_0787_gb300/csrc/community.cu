// Community membership (Section 3.3 Lemma 4, community case) and its
// validation by p-value testing (the paper's "Validation methods": Pearson
// correlation, Student-t right p-values, the bipartite graph of significant
// pairs, recovery ratio and average error).
//
// Membership: Pi_hat[i, x] = gamma^{1/3} / lambda_i * <u_i, y_x>, with
// u_i = v_i / ||v_i||, lambda_i = kappa ||v_i||^3, gamma = (sum_i lambda_i^-2)^{-1/2}
// and y_x the whitened view-A row of node x (Phi^T W^T G_{A,x} = (Y_A Phi)^T);
// entries below tau are set to zero.  An NT product of the k x k component
// matrix with the n x k sample rows: FP32 products and sums, FP64 scale.
//
// Validation: for every estimated row i and ground-truth row j,
//   rho = sum_x (a_x - mean a)(b_x - mean b) / sqrt(ss_a ss_b)  (0 for a constant row),
//   T = rho sqrt(n-2) / sqrt(1 - rho^2),  p = P(t_{n-2} > T),
//   l1 = (1/n) sum_x |a_x - b_x|,
// all in FP64; then R = (1/k) #{j : some i has p(i,j) <= threshold} and
// E = (1/k) sum over those pairs of l1.
#include <math.h>

#include "otm_internal.cuh"

namespace otm {
namespace {

constexpr int kMaxK = 1024;  // largest k of otm_membership

// ---- membership ---------------------------------------------------------

// One warp per component: norm[i] = ||v_i|| (FP64), eight components per CTA.
__global__ void component_norms_kernel(const float* __restrict__ V, int k,
                                       double* __restrict__ norm) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= k) return;
  double acc = 0.0;
#pragma unroll 4
  for (int r = lane; r < k; r += 32) {
    const double v = V[(int64_t)i * k + r];
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) norm[i] = sqrt(acc);
}

// Pi_hat (k x n) = diag(scale) Vr Y^T with Vr[i][j] = V[i * k + j] (row i = v_i)
// and scale[i] = gamma^{1/3} / (lambda_i ||v_i||) = gamma^{1/3} / (kappa ||v_i||^4):
// a 64 x 64 output tile per CTA, 256 threads with 4 x 4 outputs each, the
// contraction index staged 32 at a time in shared memory (transposed so that a
// thread's four rows / four nodes are contiguous), the next chunk loaded into
// registers while the current one is multiplied.  Every CTA sums
// sum_i lambda_i^-2 in the same fixed order, so all use the same gamma.
constexpr int MT = 64, NT = 64, KT = 32;
constexpr int LD = (MT * KT) / 256;  // elements of each tile a thread loads

__global__ void __launch_bounds__(256)
membership_kernel(const float* __restrict__ Y, int64_t n, int k, const float* __restrict__ V,
                  const double* __restrict__ norm, double kappa, double tau,
                  float* __restrict__ Pi_hat) {
  __shared__ __align__(16) float sA[KT][MT + 4];
  __shared__ __align__(16) float sB[KT][NT + 4];
  __shared__ double s_red[8];
  __shared__ double s_scale[MT];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.y * MT;
  const int64_t x0 = (int64_t)blockIdx.x * NT;
  const int ty = tid >> 4, tx = tid & 15;  // rows i0 + 4 ty .. +3, nodes x0 + 4 tx .. +3

  float ra[LD], rb[LD];
  auto load = [&](int j0) {
#pragma unroll
    for (int e = 0; e < LD; ++e) {
      const int idx = tid + e * 256;
      const int r = idx / KT, c = idx % KT;  // consecutive threads: consecutive j
      const int j = j0 + c;
      const int i = i0 + r;
      const int64_t x = x0 + r;
      ra[e] = (i < k && j < k) ? V[(int64_t)i * k + j] : 0.0f;
      rb[e] = (x < n && j < k) ? Y[x * k + j] : 0.0f;
    }
  };
  load(0);

  // gamma^{1/3} and this tile's row scales
  double part = 0.0;
  for (int i = tid; i < k; i += 256) {
    const double nv = norm[i];
    const double lam = kappa * nv * nv * nv;
    part += 1.0 / (lam * lam);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = part;
  __syncthreads();
  if (tid < MT && i0 + tid < k) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += s_red[w];
    const double g13 = cbrt(1.0 / sqrt(tot));
    const double nv = norm[i0 + tid];
    s_scale[tid] = g13 / (kappa * nv * nv * nv * nv);
  }

  float acc[4][4] = {};
  for (int j0 = 0; j0 < k; j0 += KT) {
#pragma unroll
    for (int e = 0; e < LD; ++e) {
      const int idx = tid + e * 256;
      const int r = idx / KT, c = idx % KT;
      sA[c][r] = ra[e];
      sB[c][r] = rb[e];
    }
    __syncthreads();
    if (j0 + KT < k) load(j0 + KT);
#pragma unroll
    for (int c = 0; c < KT; ++c) {
      const float4 a = *reinterpret_cast<const float4*>(&sA[c][4 * ty]);
      const float4 b = *reinterpret_cast<const float4*>(&sB[c][4 * tx]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int r = 4 * ty + p;
    if (i0 + r >= k) continue;
    const double s = s_scale[r];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t x = x0 + 4 * tx + q;
      if (x >= n) continue;
      const double v = s * (double)acc[p][q];
      Pi_hat[(int64_t)(i0 + r) * n + x] = v >= tau ? (float)v : 0.0f;
    }
  }
}

// ---- validation ---------------------------------------------------------

// Block r: mean of row r of A (rows x n, float32), in FP64.
__global__ void row_mean_kernel(const float* __restrict__ A, int64_t n,
                                double* __restrict__ mean) {
  __shared__ double s_red[32];
  const float* row = A + (int64_t)blockIdx.x * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  double acc = 0.0;
  for (int64_t x = threadIdx.x; x < n; x += blockDim.x) acc += (double)row[x];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) s_red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < nwarps; ++w) tot += s_red[w];
    mean[blockIdx.x] = tot / (double)n;
  }
}

// Regularised incomplete beta I_x(a, b) for x below (a+1)/(a+b+2), from its
// continued fraction (DLMF 8.17.22)
//   I_x(a,b) = x^a (1-x)^b / (a B(a,b)) * 1 / (1 + d_1 / (1 + d_2 / (1 + ...))),
//   d_{2m+1} = -(a+m)(a+b+m) x / ((a+2m)(a+2m+1)),  d_{2m} = m(b-m) x / ((a+2m-1)(a+2m)),
// evaluated with the modified Lentz method (Thompson and Barnett, J. Comput.
// Phys. 64, 1986).  y = 1 - x is passed separately so that it carries no
// cancellation.  At most 20,000 terms (the fraction needs O(sqrt(a)) here).
__device__ double betainc_cf(double a, double b, double x, double y) {
  const double tiny = 1e-300, eps = 1e-16;
  double f = 1.0, C = 1.0, D = 0.0;
  for (int t = 1; t <= 20000; ++t) {
    const int m = t >> 1;
    double d;
    if (t & 1)
      d = -(a + m) * (a + b + m) * x / ((a + 2 * m) * (a + 2 * m + 1));
    else
      d = m * (b - m) * x / ((a + 2 * m - 1) * (a + 2 * m));
    D = 1.0 + d * D;
    if (fabs(D) < tiny) D = tiny;
    C = 1.0 + d / C;
    if (fabs(C) < tiny) C = tiny;
    D = 1.0 / D;
    const double delta = C * D;
    f *= delta;
    if (fabs(delta - 1.0) < eps) break;
  }
  const double lbeta = lgamma(a) + lgamma(b) - lgamma(a + b);
  return exp(a * log(x) + b * log(y) - lbeta) / (a * f);
}

// Right tail P(t_nu > T) of Student's t: for T >= 0 it is I_x(nu/2, 1/2) / 2
// with x = nu / (nu + T^2); for T < 0 it is one minus the tail at -T.
__device__ double t_right_tail(double T, double nu) {
  if (T == INFINITY) return 0.0;
  if (T == -INFINITY) return 1.0;
  const double T2 = T * T;
  if (T2 == 0.0) return 0.5;
  const double x = nu / (nu + T2), y = T2 / (nu + T2);
  const double a = 0.5 * nu, b = 0.5;
  const double I = (x < (a + 1.0) / (a + b + 2.0)) ? betainc_cf(a, b, x, y)
                                                   : 1.0 - betainc_cf(b, a, y, x);
  const double tail = 0.5 * I;
  return T > 0.0 ? tail : 1.0 - tail;
}

// 16 estimated rows x 16 ground-truth rows per CTA (one pair per thread), the
// nodes staged 64 at a time, centred in FP64 and raw in float32 (raw rows
// padded by one word against bank conflicts).  Each thread sums the centred
// cross product and both centred squares in the same order, so that a row
// paired with an exact copy (or its negation) gets rho = 1 (-1) exactly.
// Epilogue: rho, T, the right p-value and the mean l1 distance.
constexpr int PT = 16, XT = 64;

__global__ void __launch_bounds__(256)
pair_kernel(const float* __restrict__ Pi_hat, int k_hat, const float* __restrict__ Pi, int k,
            int64_t n, const double* __restrict__ mean_hat, const double* __restrict__ mean_true,
            double* __restrict__ pvals, double* __restrict__ l1) {
  __shared__ double s_hc[PT][XT];      // centred estimated rows
  __shared__ double s_tc[PT][XT + 1];  // centred ground-truth rows
  __shared__ float s_h[PT][XT + 1];    // raw estimated rows
  __shared__ float s_t[PT][XT + 1];    // raw ground-truth rows
  const int tid = threadIdx.x;
  const int ti = tid >> 4, tj = tid & 15;
  const int i0 = blockIdx.y * PT, j0 = blockIdx.x * PT;
  double cross = 0.0, saa = 0.0, sbb = 0.0, dist = 0.0;
  for (int64_t xb = 0; xb < n; xb += XT) {
    for (int idx = tid; idx < PT * XT; idx += 256) {
      const int r = idx / XT, c = idx % XT;
      const int64_t x = xb + c;
      const int ih = i0 + r, jt = j0 + r;
      const bool in = x < n;
      const bool hin = in && ih < k_hat, tin = in && jt < k;
      const float h = hin ? Pi_hat[(int64_t)ih * n + x] : 0.0f;
      const float t = tin ? Pi[(int64_t)jt * n + x] : 0.0f;
      s_h[r][c] = h;
      s_t[r][c] = t;
      s_hc[r][c] = hin ? (double)h - mean_hat[ih] : 0.0;
      s_tc[r][c] = tin ? (double)t - mean_true[jt] : 0.0;
    }
    __syncthreads();
    const int cnt = (n - xb < (int64_t)XT) ? (int)(n - xb) : XT;
    for (int c = 0; c < cnt; ++c) {
      const double a = s_hc[ti][c], b = s_tc[tj][c];
      cross = fma(a, b, cross);
      saa = fma(a, a, saa);
      sbb = fma(b, b, sbb);
      dist += fabs((double)s_h[ti][c] - (double)s_t[tj][c]);
    }
    __syncthreads();
  }
  const int i = i0 + ti, j = j0 + tj;
  if (i >= k_hat || j >= k) return;
  const double rho = (saa > 0.0 && sbb > 0.0) ? cross / sqrt(saa * sbb) : 0.0;
  double T;
  if (rho >= 1.0)
    T = INFINITY;
  else if (rho <= -1.0)
    T = -INFINITY;
  else
    T = rho * sqrt((double)n - 2.0) / sqrt(1.0 - rho * rho);
  pvals[(int64_t)i * k + j] = t_right_tail(T, (double)n - 2.0);
  l1[(int64_t)i * k + j] = dist / (double)n;
}

// One CTA: degree of each ground-truth community in the p-value graph, the
// recovery ratio R and the average error E (sums in a fixed order).
__global__ void match_scores_kernel(const double* __restrict__ pvals,
                                    const double* __restrict__ l1, int k_hat, int k,
                                    double threshold, double* __restrict__ scores) {
  __shared__ double s_err[1024];
  __shared__ int s_hit[1024];
  double err = 0.0;
  int hit = 0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    int deg = 0;
    for (int i = 0; i < k_hat; ++i) {
      if (pvals[(int64_t)i * k + j] <= threshold) {
        ++deg;
        err += l1[(int64_t)i * k + j];
      }
    }
    hit += deg > 0;
  }
  s_err[threadIdx.x] = err;
  s_hit[threadIdx.x] = hit;
  __syncthreads();
  if (threadIdx.x == 0) {
    double e = 0.0;
    int h = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      e += s_err[t];
      h += s_hit[t];
    }
    scores[0] = (double)h / (double)k;
    scores[1] = e / (double)k;
  }
}

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

size_t otm_membership_workspace(int64_t k) {
  return WorkspaceSize().add<double>(k > 0 ? (size_t)k : 1).bytes();
}

otm_status otm_membership(const float* Y, int64_t n, int64_t k, const float* V, double theta,
                          double tau, float* Pi_hat, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_REQUIRE(k >= 1 && k <= kMaxK, "otm_membership: k = %lld outside [1, %d]", (long long)k,
              kMaxK);
  OTM_REQUIRE(n >= 0, "otm_membership: n = %lld < 0", (long long)n);
  OTM_REQUIRE(V && (n == 0 || (Y && Pi_hat)), "otm_membership: null pointer");
  OTM_REQUIRE(n <= (int64_t)65535 * NT * 1024, "otm_membership: n = %lld too large",
              (long long)n);
  OTM_REQUIRE(ws_bytes >= otm_membership_workspace(k), "otm_membership: workspace too small");
  if (n == 0) return OTM_OK;
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  double* norm = w.take<double>(k);
  component_norms_kernel<<<(unsigned)((k + 7) / 8), 256, 0, st>>>(V, (int)k, norm);
  OTM_CHECK_LAUNCH();
  const dim3 grid((unsigned)((n + NT - 1) / NT), (unsigned)((k + MT - 1) / MT));
  membership_kernel<<<grid, 256, 0, st>>>(Y, n, (int)k, V, norm, 0.5 * (1.0 + theta), tau,
                                          Pi_hat);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

size_t otm_pvalue_match_workspace(int64_t k_hat, int64_t k) {
  const size_t a = k_hat > 0 ? (size_t)k_hat : 1, b = k > 0 ? (size_t)k : 1;
  return WorkspaceSize().add<double>(a).add<double>(b).bytes();
}

otm_status otm_pvalue_match(const float* Pi_hat, int64_t k_hat, const float* Pi, int64_t k,
                            int64_t n, double threshold, double* pvals, double* l1,
                            double* scores, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_REQUIRE(k_hat >= 1 && k_hat <= 65535 * PT && k >= 1 && k <= 1024,
              "otm_pvalue_match: k_hat = %lld, k = %lld (need k_hat >= 1, 1 <= k <= 1024)",
              (long long)k_hat, (long long)k);
  OTM_REQUIRE(n >= 3, "otm_pvalue_match: n = %lld nodes (the t statistic needs n >= 3)",
              (long long)n);
  OTM_REQUIRE(Pi_hat && Pi && pvals && l1 && scores, "otm_pvalue_match: null pointer");
  OTM_REQUIRE(ws_bytes >= otm_pvalue_match_workspace(k_hat, k),
              "otm_pvalue_match: workspace too small");
  cudaStream_t st = as_stream(stream);
  Workspace w(ws, ws_bytes);
  double* mean_hat = w.take<double>(k_hat);
  double* mean_true = w.take<double>(k);
  row_mean_kernel<<<(unsigned)k_hat, 256, 0, st>>>(Pi_hat, n, mean_hat);
  OTM_CHECK_LAUNCH();
  row_mean_kernel<<<(unsigned)k, 256, 0, st>>>(Pi, n, mean_true);
  OTM_CHECK_LAUNCH();
  const dim3 grid((unsigned)((k + PT - 1) / PT), (unsigned)((k_hat + PT - 1) / PT));
  pair_kernel<<<grid, 256, 0, st>>>(Pi_hat, (int)k_hat, Pi, (int)k, n, mean_hat, mean_true,
                                    pvals, l1);
  OTM_CHECK_LAUNCH();
  match_scores_kernel<<<1, 1024, 0, st>>>(pvals, l1, (int)k_hat, (int)k, threshold, scores);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

}  // extern "C"
