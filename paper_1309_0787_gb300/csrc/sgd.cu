// Stochastic tensor gradient descent on the implicit whitened tensor
// (Section 3.2, Lemma 3 / Eq. (16), Appendix A), fused into one kernel.
//
// Per step, for the minibatch Y_b (b samples, three views) and V (k x k):
//   A_A = V^T Y_A^T, A_B = V^T Y_B^T                         (k x b)
//   a_A = V^T ybar_A, a_B = V^T ybar_B                        (k)
//   B   = c1 A_A o A_B - c2 (a_B o A_A + a_A o A_B)           (column-broadcast a)
//   s   = (1/b) sum_t (A_A o A_B)[:, t]
//   G_data = (1/b) Y_C^T B^T + ybar_C (c3 a_A o a_B - c2 s)^T  (column i = T_b(v_i, v_i, I))
//   G_gram = V ((V^T V) o (V^T V))
//   V <- V - beta_t (kappa G_gram - G_data)
// This is the stacked ("BLAS III", Section 4.3) form of the per-component
// update of Lemma 3; the k x k x k tensor is never formed.
//
// GB300 mapping: one thread-block cluster runs the whole loop of steps (the
// "device interface" of Section 4.3: V never leaves the chip).  Each CTA of
// the cluster holds a full copy of V in shared memory and processes a slice
// of the minibatch in chunks of 32 samples (register-tiled FP32 FMAs for both
// products; the next chunk arrives by cp.async while one is computed, and the
// next step's row indices are fetched a step ahead).  Partial Y_C^T B^T are reduced column-wise through distributed
// shared memory: CTA q owns columns [q*cpq, (q+1)*cpq), sums them over the
// cluster, adds the Gram and mean terms and broadcasts the new columns into
// every CTA's next-V buffer together with their means a_A, a_B.  Two cluster
// barriers per step; no global memory traffic besides the samples.
#include <algorithm>
#include <atomic>

#include <cooperative_groups.h>

#include "otm_internal.cuh"
#include "tc_ptx.cuh"

namespace cg = cooperative_groups;

namespace otm {
namespace {

using tc::cp_async16;
using tc::cp_async_commit;
using tc::cp_async_wait;

constexpr int TC = 32;        // samples per chunk
constexpr int THREADS = 256;  // 8 warps
constexpr int KMAX = 128;
constexpr int RB = 4 * THREADS;  // staged row indices per CTA and step

struct SgdArgs {
  const float* YA;
  const float* YB;
  const float* YC;
  const int32_t* perm;
  const double* ybar3;
  float* V;
  float* V_snap;
  int64_t n, b, spe, total_steps, snapshot_every;
  int k;
  double beta0;
  float c1, c2, c3, kappa;
};

struct Layout {
  int kp, ldk, cpq, nview;
  int64_t bq;  // samples of a minibatch per CTA
  int nrows;   // of which the row indices are staged in shared memory
  int nbuf;    // sample-chunk buffers: 2 (load the next chunk during this one) or 1
  size_t off_v0, off_v1, off_u, off_p6, off_small, off_rows, total_floats;
};

// Shared memory (floats): V twice (current / next), the sample chunks (nbuf
// buffers of nview x TC samples; two where they fit) and B, the owner buffers, the means (a_A, a_B
// double-buffered by step parity), and the row indices of this CTA's slice of
// the current and the next minibatch (the first RB of them; a longer slice reads
// the rest of its indices from the permutation as it goes).
__host__ __device__ inline Layout make_layout(int k, int CL, bool sym, int64_t b, int nbuf) {
  Layout L;
  L.kp = (k + 3) & ~3;
  L.ldk = L.kp;
  L.cpq = (k + CL - 1) / CL;
  L.nview = sym ? 1 : 3;
  L.bq = (b + CL - 1) / CL;
  L.nrows = (int)(L.bq < RB ? L.bq : RB);
  const size_t vsz = (size_t)L.kp * L.ldk;
  L.nbuf = nbuf;
  size_t u1 = (size_t)(nbuf * L.nview + 1) * TC * L.ldk;
  const size_t u = u1 > vsz ? u1 : vsz;
  L.off_v0 = 0;
  L.off_v1 = vsz;
  L.off_u = 2 * vsz;
  L.off_p6 = L.off_u + u;
  L.off_small = L.off_p6 + (size_t)3 * L.cpq * L.ldk;
  L.off_rows = L.off_small + 8 * (size_t)L.ldk + (size_t)L.cpq + 8;
  L.total_floats = L.off_rows + 2 * (size_t)L.nrows + 4;
  return L;
}

template <bool SYM, int MT, int CL>
__global__ void __launch_bounds__(THREADS, 1) sgd_cluster_kernel(SgdArgs a, int nbuf) {
  extern __shared__ __align__(16) float sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k;
  const Layout L = make_layout(k, CL, SYM, a.b, nbuf);
  const int ldk = L.ldk, kp = L.kp, cpq = L.cpq;
  float* V0 = sm + L.off_v0;
  float* V1 = sm + L.off_v1;
  float* U = sm + L.off_u;
  float* Bt = U + nbuf * L.nview * TC * ldk;
  float* Gp = U;  // k x ldk partial Y_C^T B^T (after the chunk loop)
  float* gd = sm + L.off_p6;              // cpq x ldk
  float* Hm = gd + cpq * ldk;             // cpq x ldk
  float* vn = Hm + cpq * ldk;             // cpq x ldk
  float* aAb = sm + L.off_small;          // [2][ldk] by step parity
  float* aBb = aAb + 2 * ldk;             // [2][ldk]
  float* ybA = aBb + 2 * ldk;
  float* ybB = ybA + ldk;
  float* ybC = ybB + ldk;
  float* spart = ybC + ldk;
  float* sown = spart + ldk;
  int* srow = reinterpret_cast<int*>(sm + L.off_rows);  // [2][nrows] by step parity

  // ---- initial state: V (zero padded) and the means ----
  for (int idx = tid; idx < kp * ldk; idx += THREADS) {
    const int i = idx / ldk, r = idx % ldk;
    V0[idx] = (i < k && r < k) ? a.V[(int64_t)i * k + r] : 0.f;
    V1[idx] = 0.f;  // padding rows stay zero; owners fill the rest
  }
  for (int r = tid; r < 4 * ldk; r += THREADS) aAb[r] = 0.f;  // a_A, a_B, both parities
  for (int r = tid; r < ldk; r += THREADS) {
    ybA[r] = r < k ? (float)a.ybar3[r] : 0.f;
    ybB[r] = r < k ? (float)a.ybar3[k + r] : 0.f;
    ybC[r] = r < k ? (float)a.ybar3[2 * k + r] : 0.f;
  }
  const int own_lo = q * cpq, own_hi = min(k, own_lo + cpq);
  const int64_t bq = L.bq;
  // row index of sample p of this CTA's slice of step s (-1 outside the minibatch)
  auto row_of = [&](int64_t s, int64_t p) -> int {
    const int64_t e = s / a.spe, pos0 = (s % a.spe) * a.b;
    const int64_t lo = (int64_t)q * bq + p;
    if (lo >= min(a.b, a.n - pos0) || p >= bq) return -1;
    return a.perm ? a.perm[e * a.n + pos0 + lo] : (int)(pos0 + lo);
  };
  const int nrows = L.nrows;
  for (int p = tid; p < nrows; p += THREADS) srow[p] = a.total_steps > 0 ? row_of(0, p) : -1;
  cluster.sync();  // zeroed buffers before any remote write
  // a_A, a_B of the initial V (later steps receive them from the owners)
  for (int i = warp; i < kp; i += THREADS / 32) {
    float x = 0.f, y = 0.f;
    for (int r = lane; r < ldk; r += 32) {
      const float v = V0[i * ldk + r];
      x = fmaf(v, ybA[r], x);
      y = fmaf(v, ybB[r], y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) {
      aAb[i] = x;
      aBb[i] = y;
    }
  }
  __syncthreads();
  // rows 16-byte aligned: chunks arrive by cp.async while the previous one is used
  const bool vec_rows = (k & 3) == 0 && ((reinterpret_cast<uintptr_t>(a.YA) |
                                          reinterpret_cast<uintptr_t>(a.YB) |
                                          reinterpret_cast<uintptr_t>(a.YC)) & 15) == 0;

  // GEMM1 thread mapping: warp w covers components 16w..16w+15 as i = 16w + il + 4j,
  // lane covers samples t = tl + 8j'.
  const int tl = lane & 7, il = lane >> 3;
  const int ibase = 16 * warp + il;

  for (int64_t s = 0; s < a.total_steps; ++s) {
    float* Vc = (s & 1) ? V1 : V0;
    float* Vn = (s & 1) ? V0 : V1;
    const int64_t pos0 = (s % a.spe) * a.b;
    const int64_t beff = min(a.b, a.n - pos0);
    const float beta = (float)a.beta0 / sqrtf((float)(s + 1));
    const float inv_b = 1.f / (float)beff;
    const int par = (int)(s & 1);
    const float* aA = aAb + par * ldk;  // means of this step's V, from the owners
    const float* aB = aBb + par * ldk;
    const int* rows = srow + par * nrows;
    // the next step's row indices: loaded now, stored at the end of the step
    int pre[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = tid + THREADS * j;
      pre[j] = (s + 1 < a.total_steps && p < nrows) ? row_of(s + 1, p) : -1;
    }
    for (int i = tid; i < kp; i += THREADS) spart[i] = 0.f;
    float gacc[MT][4][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) gacc[m][x][y] = 0.f;

    const int64_t my_lo = (int64_t)q * bq;
    const int64_t nmy = max((int64_t)0, min(beff, my_lo + bq) - my_lo);
    const int nchunk = (int)((nmy + TC - 1) / TC);
    // chunk c of the slice into buffer `buf` (rows beyond the slice are zero; an
    // index outside [0, n), i.e. an invalid permutation, reads as a zero sample)
    auto load_chunk = [&](int c, int buf) {
      float* Yd = U + (size_t)buf * L.nview * TC * ldk;
      const int c0 = c * TC;
      const int nv4 = ldk / 4;
      if (vec_rows) {
        for (int idx = tid; idx < TC * nv4; idx += THREADS) {
          const int tt = idx / nv4, r4 = idx % nv4;
          const int p = c0 + tt;
          const int row = p < nmy ? (p < nrows ? rows[p] : row_of(s, p)) : -1;
          const bool ok = row >= 0 && row < a.n;
          for (int v = 0; v < L.nview; ++v) {
            const float* Yg = v == 0 ? a.YA : (v == 1 ? a.YB : a.YC);
            cp_async16(Yd + ((size_t)v * TC + tt) * ldk + 4 * r4,
                       ok ? Yg + (int64_t)row * k + 4 * r4 : Yg, ok ? 16u : 0u);
          }
        }
        cp_async_commit();
      } else {
        for (int idx = tid; idx < TC * nv4; idx += THREADS) {
          const int tt = idx / nv4, r4 = idx % nv4;
          const int p = c0 + tt;
          const int row = p < nmy ? (p < nrows ? rows[p] : row_of(s, p)) : -1;
          for (int v = 0; v < L.nview; ++v) {
            const float* Yg = v == 0 ? a.YA : (v == 1 ? a.YB : a.YC);
            float t4[4] = {0.f, 0.f, 0.f, 0.f};
            if (row >= 0 && row < a.n) {
              const int r = 4 * r4;
#pragma unroll
              for (int z = 0; z < 4; ++z) t4[z] = (r + z < k) ? Yg[(int64_t)row * k + r + z] : 0.f;
            }
            reinterpret_cast<float4*>(Yd + ((size_t)v * TC + tt) * ldk)[r4] =
                make_float4(t4[0], t4[1], t4[2], t4[3]);
          }
        }
      }
    };
    if (nbuf == 2 && nchunk > 0) load_chunk(0, 0);
    for (int ch = 0; ch < nchunk; ++ch) {
      const int buf = nbuf == 2 ? (ch & 1) : 0;
      const bool ahead = nbuf == 2 && ch + 1 < nchunk;
      if (ahead) load_chunk(ch + 1, buf ^ 1);
      if (nbuf == 1) load_chunk(ch, 0);
      if (vec_rows) cp_async_wait(ahead ? 1 : 0);
      __syncthreads();
      const float* Ya = U + (size_t)buf * L.nview * TC * ldk;
      const float* Yb = SYM ? Ya : Ya + TC * ldk;
      const float* Yc = SYM ? Ya : Ya + 2 * TC * ldk;

      // GEMM1: A_A, A_B for 4 components x 4 samples per thread, then B
      if (16 * warp < kp) {
        float accA[4][4], accB[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            accA[x][y] = 0.f;
            accB[x][y] = 0.f;
          }
#pragma unroll 2
        for (int r = 0; r < ldk; r += 4) {
          float4 v[4], ya[4], yb[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int i = ibase + 4 * j;
            v[j] = i < kp ? *reinterpret_cast<const float4*>(Vc + i * ldk + r)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
            ya[j] = *reinterpret_cast<const float4*>(Ya + (tl + 8 * j) * ldk + r);
            if (!SYM) yb[j] = *reinterpret_cast<const float4*>(Yb + (tl + 8 * j) * ldk + r);
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
              float t = accA[x][y];
              t = fmaf(v[x].x, ya[y].x, t);
              t = fmaf(v[x].y, ya[y].y, t);
              t = fmaf(v[x].z, ya[y].z, t);
              t = fmaf(v[x].w, ya[y].w, t);
              accA[x][y] = t;
              if (!SYM) {
                float u = accB[x][y];
                u = fmaf(v[x].x, yb[y].x, u);
                u = fmaf(v[x].y, yb[y].y, u);
                u = fmaf(v[x].z, yb[y].z, u);
                u = fmaf(v[x].w, yb[y].w, u);
                accB[x][y] = u;
              }
            }
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int i = ibase + 4 * x;
          const float ai = i < kp ? aA[i] : 0.f, bi = i < kp ? aB[i] : 0.f;
          float ssum = 0.f;
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const float xa = accA[x][y];
            const float xb = SYM ? xa : accB[x][y];
            const float pr = xa * xb;
            ssum += pr;
            const float bv = a.c1 * pr - a.c2 * (bi * xa + ai * xb);
            if (i < kp) Bt[(tl + 8 * y) * ldk + i] = bv;
          }
          // sum over the 8 sample lanes sharing this component (lane bits 0..2)
          ssum += __shfl_xor_sync(0xffffffffu, ssum, 1);
          ssum += __shfl_xor_sync(0xffffffffu, ssum, 2);
          ssum += __shfl_xor_sync(0xffffffffu, ssum, 4);
          if (tl == 0 && i < kp) spart[i] += ssum;
        }
      }
      __syncthreads();

      // GEMM2: Gp[r][i] += sum_t Y_C[t][r] B[t][i]; 4 x 4 tiles, MT tiles per thread
      {
        const int nt = kp / 4;
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          const int g = tid + THREADS * m;
          if (g < nt * nt) {
            const int r0 = 4 * (g % nt), i0 = 4 * (g / nt);
#pragma unroll 8
            for (int tt = 0; tt < TC; ++tt) {
              const float4 yc = *reinterpret_cast<const float4*>(Yc + tt * ldk + r0);
              const float4 bt = *reinterpret_cast<const float4*>(Bt + tt * ldk + i0);
              const float ycv[4] = {yc.x, yc.y, yc.z, yc.w};
              const float btv[4] = {bt.x, bt.y, bt.z, bt.w};
#pragma unroll
              for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) gacc[m][x][y] = fmaf(ycv[x], btv[y], gacc[m][x][y]);
            }
          }
        }
      }
      __syncthreads();
    }

    // partial results to shared memory: Gp[i][r] (column i contiguous)
    {
      const int nt = kp / 4;
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        const int g = tid + THREADS * m;
        if (g < nt * nt) {
          const int r0 = 4 * (g % nt), i0 = 4 * (g / nt);
#pragma unroll
          for (int y = 0; y < 4; ++y)
            *reinterpret_cast<float4*>(Gp + (i0 + y) * ldk + r0) =
                make_float4(gacc[m][0][y], gacc[m][1][y], gacc[m][2][y], gacc[m][3][y]);
        }
      }
    }
    cluster.sync();  // partials of every CTA visible cluster-wide

    // phase 6: owned columns -- reduce over the cluster, Gram term, update, broadcast
    const int nown = own_hi - own_lo;
    if (tid < nown) {
      float part[CL];
#pragma unroll
      for (int c = 0; c < CL; ++c) part[c] = cluster.map_shared_rank(spart, c)[own_lo + tid];
      float ss = 0.f;
#pragma unroll
      for (int c = 0; c < CL; ++c) ss += part[c];
      sown[tid] = ss;
    }
    for (int idx = tid; idx < nown * kp; idx += THREADS) {
      const int jj = idx / kp, r = idx % kp;
      const int i = own_lo + jj;
      float part[CL];
#pragma unroll
      for (int c = 0; c < CL; ++c) part[c] = cluster.map_shared_rank(Gp, c)[i * ldk + r];
      float g = 0.f;
#pragma unroll
      for (int c = 0; c < CL; ++c) g += part[c];
      gd[jj * ldk + r] = g;
    }
    // H[jj][j] = (v_i . v_j)^2 (thread per entry, four partial sums)
    for (int idx = tid; idx < nown * kp; idx += THREADS) {
      const int jj = idx / kp, j = idx % kp;
      const float* vi = Vc + (own_lo + jj) * ldk;
      const float* vj = Vc + j * ldk;
      float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f;
#pragma unroll 5
      for (int r = 0; r < ldk; r += 4) {
        const float4 x = *reinterpret_cast<const float4*>(vi + r);
        const float4 y = *reinterpret_cast<const float4*>(vj + r);
        h0 = fmaf(x.x, y.x, h0);
        h1 = fmaf(x.y, y.y, h1);
        h2 = fmaf(x.z, y.z, h2);
        h3 = fmaf(x.w, y.w, h3);
      }
      const float h = (h0 + h1) + (h2 + h3);
      Hm[jj * ldk + j] = h * h;
    }
    __syncthreads();
    // Gram term G = V (H o H) and the update: thread per (column, 4 coordinates)
    for (int idx = tid; idx < nown * (kp / 4); idx += THREADS) {
      const int jj = idx / (kp / 4), r = 4 * (idx % (kp / 4));
      const int i = own_lo + jj;
      float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
      int j = 0;
#pragma unroll 4
      for (; j + 1 < k; j += 2) {
        const float ha = Hm[jj * ldk + j], hb = Hm[jj * ldk + j + 1];
        const float4 va = *reinterpret_cast<const float4*>(Vc + j * ldk + r);
        const float4 vb = *reinterpret_cast<const float4*>(Vc + (j + 1) * ldk + r);
        g0.x = fmaf(ha, va.x, g0.x);
        g0.y = fmaf(ha, va.y, g0.y);
        g0.z = fmaf(ha, va.z, g0.z);
        g0.w = fmaf(ha, va.w, g0.w);
        g1.x = fmaf(hb, vb.x, g1.x);
        g1.y = fmaf(hb, vb.y, g1.y);
        g1.z = fmaf(hb, vb.z, g1.z);
        g1.w = fmaf(hb, vb.w, g1.w);
      }
      if (j < k) {
        const float ha = Hm[jj * ldk + j];
        const float4 va = *reinterpret_cast<const float4*>(Vc + j * ldk + r);
        g0.x = fmaf(ha, va.x, g0.x);
        g0.y = fmaf(ha, va.y, g0.y);
        g0.z = fmaf(ha, va.z, g0.z);
        g0.w = fmaf(ha, va.w, g0.w);
      }
      const float gg[4] = {g0.x + g1.x, g0.y + g1.y, g0.z + g1.z, g0.w + g1.w};
      const float mean_term = a.c3 * aA[i] * aB[i] - a.c2 * sown[jj] * inv_b;
      float out[4];
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const float gdata = gd[jj * ldk + r + z] * inv_b + ybC[r + z] * mean_term;
        const float vnew = Vc[i * ldk + r + z] - beta * (a.kappa * gg[z] - gdata);
        out[z] = (r + z < k) ? vnew : 0.f;
      }
      *reinterpret_cast<float4*>(vn + jj * ldk + r) = make_float4(out[0], out[1], out[2], out[3]);
    }
    __syncthreads();
    for (int idx = tid; idx < nown * (kp / 4); idx += THREADS) {
      const int jj = idx / (kp / 4), r = 4 * (idx % (kp / 4));
      const float4 v = *reinterpret_cast<const float4*>(vn + jj * ldk + r);
#pragma unroll
      for (int c = 0; c < CL; ++c)
        *reinterpret_cast<float4*>(cluster.map_shared_rank(Vn, c) + (own_lo + jj) * ldk + r) = v;
    }
    // means of the new owned columns for the next step, to every CTA
    for (int jj = warp; jj < nown; jj += THREADS / 32) {
      float x = 0.f, y = 0.f;
      for (int r = lane; r < kp; r += 32) {
        x = fmaf(vn[jj * ldk + r], ybA[r], x);
        y = fmaf(vn[jj * ldk + r], ybB[r], y);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      if (lane < CL) {
        cluster.map_shared_rank(aAb, lane)[(par ^ 1) * ldk + own_lo + jj] = x;
        cluster.map_shared_rank(aBb, lane)[(par ^ 1) * ldk + own_lo + jj] = y;
      }
    }
    {
      int* rows_next = srow + (par ^ 1) * nrows;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int p = tid + THREADS * j;
        if (p < nrows) rows_next[p] = pre[j];
      }
    }
    cluster.sync();  // next V and means complete everywhere; partials may be overwritten

    if (a.snapshot_every > 0 && (s + 1) % a.snapshot_every == 0) {
      float* dst = a.V_snap + ((s + 1) / a.snapshot_every - 1) * (int64_t)k * k;
      for (int idx = tid; idx < nown * k; idx += THREADS) {
        const int jj = idx / k, r = idx % k;
        dst[(int64_t)(own_lo + jj) * k + r] = Vn[(own_lo + jj) * ldk + r];
      }
    }
  }
  const float* Vf = (a.total_steps & 1) ? V1 : V0;
  for (int idx = tid; idx < (own_hi - own_lo) * k; idx += THREADS) {
    const int jj = idx / k, r = idx % k;
    a.V[(int64_t)(own_lo + jj) * k + r] = Vf[(own_lo + jj) * ldk + r];
  }
}

template <bool SYM, int MT, int CL>
otm_status launch_cl(const SgdArgs& args, int nbuf, cudaStream_t st) {
  const Layout L = make_layout(args.k, CL, SYM, args.b, nbuf);
  const size_t smem = L.total_floats * sizeof(float);
  auto kern = sgd_cluster_kernel<SYM, MT, CL>;
  OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (CL > 8)
    OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  OTM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, args, nbuf));
  count_launch();
  return OTM_OK;
}

template <bool SYM, int MT>
otm_status launch_mt(const SgdArgs& args, int CL, int nbuf, cudaStream_t st) {
  switch (CL) {
    case 16: return launch_cl<SYM, MT, 16>(args, nbuf, st);
    case 8: return launch_cl<SYM, MT, 8>(args, nbuf, st);
    case 4: return launch_cl<SYM, MT, 4>(args, nbuf, st);
    case 2: return launch_cl<SYM, MT, 2>(args, nbuf, st);
    default: return launch_cl<SYM, MT, 1>(args, nbuf, st);
  }
}

template <bool SYM>
otm_status launch_sym(const SgdArgs& args, int CL, int nbuf, cudaStream_t st) {
  const int nt = ((args.k + 3) & ~3) / 4;
  const int MT = (nt * nt + THREADS - 1) / THREADS;
  switch (MT) {
    case 1: return launch_mt<SYM, 1>(args, CL, nbuf, st);
    case 2: return launch_mt<SYM, 2>(args, CL, nbuf, st);
    case 3: return launch_mt<SYM, 3>(args, CL, nbuf, st);
    default: return launch_mt<SYM, 4>(args, CL, nbuf, st);
  }
}

// Largest supported cluster size whose shared-memory footprint fits (16, then
// 8, ...), with two sample-chunk buffers where they fit and one otherwise;
// *nbuf receives the buffer count.
int pick_cluster(int k, bool sym, int64_t b, int max_cl, int* nbuf) {
  static int max_smem = 0;
  if (max_smem == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (max_smem <= 0) max_smem = 227 * 1024;
  }
  for (int CL : {16, 8, 4, 2, 1})
    for (int nb : {2, 1}) {
      if (CL > max_cl) continue;
      const Layout L = make_layout(k, CL, sym, b, nb);
      if (L.total_floats * sizeof(float) <= (size_t)max_smem) {
        *nbuf = nb;
        return CL;
      }
    }
  return 0;
}

// Which form runs otm_sgd_step / otm_sgd_run: 0 = chosen by size, 1 = the
// cluster form (this file), 2 = the grid form (sgd_grid.cu), 3 = the split
// form (sgd_split.cu).
std::atomic<int> g_sgd_form{0};
// The grid and split forms are chosen for minibatches of at least this many samples.
constexpr int64_t GRID_AUTO_MIN_B = 256;

otm_status run(float* V, const float* YA, const float* YB, const float* YC, int64_t n, int64_t k,
               const double* ybar3, const int32_t* perm, int64_t epochs, int64_t b,
               double beta0, double theta, double alpha0, int64_t snapshot_every, float* V_snap,
               void* ws, size_t ws_bytes, cudaStream_t st) {
  const int form = g_sgd_form.load();
  const bool sym_views = (YA == YB) && (YB == YC);
  const bool grid_ok = sgd_grid_applicable(k, b);
  // auto: the grid form where it applies (the fastest per step at b = 1,024,
  // k = 100); beyond its minibatch limit the split form, which spreads a large
  // minibatch over all clusters instead of one
  if (form == 3 || (form == 0 && !grid_ok && b >= GRID_AUTO_MIN_B && ws &&
                    ws_bytes >= sgd_split_workspace(k))) {
    const bool split_ok = sgd_split_applicable(k, b, sym_views);
    if (form == 3 && !split_ok)
      return set_error(OTM_EINVAL, "sgd: the split form needs k <= 128 and all of its clusters "
                                   "resident at once");
    if (split_ok)
      return sgd_split_run(V, YA, YB, YC, n, k, ybar3, perm, epochs, b, beta0, theta, alpha0,
                           snapshot_every, V_snap, ws, ws_bytes, st);
  }
  if (form == 2 && !grid_ok)
    return set_error(OTM_EINVAL, "sgd: the grid form needs k <= 128 and 16 <= b <= 32 x SMs");
  // the auto choice takes the grid form only when the caller gave it its scratch
  const bool grid_ws_ok = ws && ws_bytes >= sgd_grid_workspace(k, b);
  if (form == 2 || (form == 0 && grid_ok && grid_ws_ok && b >= GRID_AUTO_MIN_B))
    return sgd_grid_run(V, YA, YB, YC, n, k, ybar3, perm, epochs, b, beta0, theta, alpha0,
                        snapshot_every, V_snap, ws, ws_bytes, st);
  SgdArgs args;
  const bool sym = (YA == YB) && (YB == YC);
  args.YA = YA;
  args.YB = YB;
  args.YC = YC;
  args.perm = perm;
  args.ybar3 = ybar3;
  args.V = V;
  args.V_snap = V_snap;
  args.n = n;
  args.b = b;
  args.spe = (n + b - 1) / b;
  args.total_steps = args.spe * epochs;
  args.snapshot_every = snapshot_every;
  args.k = (int)k;
  args.beta0 = beta0;
  const double a0 = alpha0;
  args.c1 = (float)((a0 + 1.0) * (a0 + 2.0) / 2.0);
  args.c2 = (float)(a0 * (a0 + 1.0) / 2.0);
  args.c3 = (float)(a0 * a0);
  args.kappa = (float)(0.5 * (1.0 + theta));
  int nbuf = 1;
  int CL = pick_cluster((int)k, sym, b, 16, &nbuf);
  if (CL == 0) return set_error(OTM_EINVAL, "sgd: k=%lld does not fit shared memory", (long long)k);
  // honour the device's limit on active clusters of this size
  static int cl16_ok = -1;
  if (CL == 16 && cl16_ok < 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = make_layout((int)k, 16, sym, b, nbuf).total_floats * sizeof(float);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto kern = sgd_cluster_kernel<false, 4, 16>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)cfg.dynamicSmemBytes);
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    cl16_ok = (e == cudaSuccess && nclusters > 0) ? 1 : 0;
    cudaGetLastError();
  }
  if (CL == 16 && cl16_ok == 0) CL = pick_cluster((int)k, sym, b, 8, &nbuf);
  if (CL == 0) return set_error(OTM_EINVAL, "sgd: k=%lld does not fit shared memory", (long long)k);
  return sym ? launch_sym<true>(args, CL, nbuf, st) : launch_sym<false>(args, CL, nbuf, st);
}

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

size_t otm_sgd_workspace(int64_t k, int64_t b) {
  return std::max(sgd_grid_workspace(k, b), sgd_split_workspace(k));
}

otm_status otm_sgd_step(float* V, const float* YA, const float* YB, const float* YC, int64_t b,
                        int64_t k, const double* ybar3, double theta, double beta,
                        double alpha0, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  OTM_REQUIRE(V && YA && YB && YC && ybar3, "otm_sgd_step: null pointer");
  OTM_REQUIRE(k >= 1 && k <= KMAX, "otm_sgd_step: k=%lld outside [1, %d]", (long long)k, KMAX);
  OTM_REQUIRE(b >= 1, "otm_sgd_step: b must be >= 1");
  return run(V, YA, YB, YC, b, k, ybar3, nullptr, 1, b, beta, theta, alpha0, 0, nullptr, ws,
             ws_bytes, as_stream(stream));
}

otm_status otm_sgd_set_form(int form) {
  clear_error();
  OTM_REQUIRE(form >= 0 && form <= 3, "otm_sgd_set_form: form must be 0, 1, 2 or 3");
  g_sgd_form.store(form);
  return OTM_OK;
}

otm_status otm_sgd_run(float* V, const float* YA, const float* YB, const float* YC, int64_t n,
                       int64_t k, const double* ybar3, const int32_t* perm, int64_t epochs,
                       int64_t b, double beta0, double theta, double alpha0,
                       int64_t snapshot_every, float* V_snap, void* ws, size_t ws_bytes,
                       void* stream) {
  clear_error();
  OTM_REQUIRE(V && YA && YB && YC && ybar3, "otm_sgd_run: null pointer");
  OTM_REQUIRE(k >= 1 && k <= KMAX, "otm_sgd_run: k=%lld outside [1, %d]", (long long)k, KMAX);
  OTM_REQUIRE(n >= 1 && b >= 1 && epochs >= 0, "otm_sgd_run: need n >= 1, b >= 1, epochs >= 0");
  OTM_REQUIRE(snapshot_every >= 0, "otm_sgd_run: snapshot_every must be >= 0");
  OTM_REQUIRE(snapshot_every == 0 || V_snap, "otm_sgd_run: V_snap required for snapshots");
  if (epochs == 0) return OTM_OK;
  return run(V, YA, YB, YC, n, k, ybar3, perm, epochs, b, beta0, theta, alpha0, snapshot_every,
             V_snap, ws, ws_bytes, as_stream(stream));
}

}  // extern "C"
