// Precision form of the fused STGD step (Section 3.2, Lemma 3) on the
// fifth-generation tensor cores.  The two products of the stacked update,
//   A = Y_b V        (samples x components, K = coordinates; views A and B)
//   G = Y_C^T B      (coordinates x components, K = samples)
// run as tcgen05.mma in BF16 (kind::f16) or FP8 e4m3 (kind::f8f6f4) with
// FP32 accumulators in tensor memory; B = c1 A_A o A_B - c2 (a_B o A_A +
// a_A o A_B) is formed in registers between them.  The FP32 master V, the
// Gram term V((V^T V) o (V^T V)), the mean terms and the update stay in FP32
// as in the FP32 kernel (sgd.cu), and so does the organisation: one
// thread-block cluster runs all steps, the minibatch is split over its CTAs,
// partial G are summed column-wise through distributed shared memory, and V
// never leaves the chip.
//
// Scaling: samples are stored quantised with one scale per sample (FP8; BF16
// stores scale 1); V is re-quantised every step with one scale per component;
// B with one scale per component per 128-sample tile.  Every scale is applied
// to the FP32 accumulator in the epilogues:
//   A[t][i] = s_t sigma_i D1[t][i],   G[r][i] = sum over tiles of beta_i D2[r][i].
//
// Operand layouts in shared memory (no swizzle; 8-row x 16-byte core
// matrices; LBO = stride between cores along K, SBO = along M/N):
//   sample tile: core (tg, rg) = 8 samples x 16 B of coordinates at
//                (tg * CR + rg) * 128 with CR = KP * esize / 16; read K-major
//                (M = samples, K = coordinates) by the first product and
//                MN-major (M = coordinates, K = samples) by the second;
//   V image:     core (ng, rg) = 8 components x 16 B of coordinates, K-major;
//   B image:     core (tg, ng) = 8 samples x 16 B of components, MN-major.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "otm_internal.cuh"
#include "tc_ptx.cuh"

namespace cg = cooperative_groups;

namespace otm {
namespace {

constexpr int TILE = 128;        // samples per MMA tile (M of the first product)
constexpr int KP = 128;          // padded coordinates (M of the second product)
constexpr int TC_THREADS = 256;  // 8 warps: 2 warps per 32-lane TMEM quarter
constexpr uint32_t TMEM_COLS = 512;
constexpr int TC_KMAX = 128;

using namespace tc;

struct TcArgs {
  const uint8_t* YA;  // quantised samples, row stride ldq elements
  const uint8_t* YB;
  const uint8_t* YC;
  const float* sA;    // per-sample scales (null = 1)
  const float* sB;
  const float* sC;
  const int32_t* perm;
  const double* ybar3;
  float* V;
  float* V_snap;
  int* err;
  int64_t n, b, spe, total_steps, snapshot_every;
  int k, ldq;
  double beta0;
  float c1, c2, c3, kappa;
};

struct TcLayout {
  int np, ldk, cpq, nview, esize, cr, cb;
  size_t y_bytes, b_bytes, v_bytes;
  size_t off_b, off_v, off_f;
  // float offsets inside the FP32 region
  size_t vm, gd, hm, vn, aA, aB, ybA, ybB, ybC, vsc, bsc, spw, spart, sown, sAt, sBt, sCt,
      amax, nfloat;
  size_t total;
};

__host__ __device__ inline TcLayout tc_layout(int k, int CL, bool sym, int esize) {
  TcLayout L;
  L.np = (k + 15) & ~15;
  L.ldk = (k + 3) & ~3;
  L.cpq = (k + CL - 1) / CL;
  L.nview = sym ? 1 : 3;
  L.esize = esize;
  L.cr = KP * esize / 16;
  L.cb = L.np * esize / 16;
  L.y_bytes = (size_t)TILE * KP * esize;
  L.b_bytes = (size_t)TILE * L.np * esize;
  L.v_bytes = (size_t)L.np * KP * esize;
  L.off_b = L.y_bytes * L.nview;
  size_t region = L.off_b + L.b_bytes;
  const size_t gp = (size_t)L.np * KP * 4;  // partial G (FP32) reuses the sample images
  if (region < gp) region = gp;
  L.off_v = (region + 1023) & ~(size_t)1023;
  L.off_f = (L.off_v + L.v_bytes + 1023) & ~(size_t)1023;
  size_t f = 0;
  L.vm = f; f += (size_t)k * L.ldk;
  L.gd = f; f += (size_t)L.cpq * L.ldk;
  L.hm = f; f += (size_t)L.cpq * L.ldk;
  L.vn = f; f += (size_t)L.cpq * L.ldk;
  L.aA = f; f += L.np;
  L.aB = f; f += L.np;
  L.ybA = f; f += L.ldk;
  L.ybB = f; f += L.ldk;
  L.ybC = f; f += L.ldk;
  L.vsc = f; f += L.np;
  L.bsc = f; f += L.np;
  L.spw = f; f += 4 * (size_t)L.np;
  L.spart = f; f += L.np;
  L.sown = f; f += L.cpq + 4;
  L.sAt = f; f += TILE;
  L.sBt = f; f += TILE;
  L.sCt = f; f += TILE;
  L.amax = f; f += L.np;
  L.nfloat = f;
  L.total = L.off_f + f * 4 + 64;
  return L;
}

struct TcCtx {
  uint64_t* mbar;
  int* abort;
  uint32_t tmem;
  uint32_t phase;
};

// One STGD chain (one decomposition) with V on-chip, run by one cluster.
// TMEM and the mbarrier are set up by the caller; the chain ends with a
// cluster barrier so that the caller may reuse shared memory afterwards.
template <bool FP8, bool SYM, int CL>
__device__ __forceinline__ void tc_chain(const TcArgs& a, uint8_t* smem, TcCtx& cx) {
  constexpr int ES = FP8 ? 1 : 2;
  constexpr int KSTEP = FP8 ? 32 : 16;            // K of one MMA
  constexpr uint32_t FMT = FP8 ? 0u : 1u;         // E4M3 / BF16
  constexpr float QMAX = FP8 ? 448.f : 1.f;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quad = warp & 3, half = warp >> 2;
  const int k = a.k;
  const TcLayout L = tc_layout(k, CL, SYM, ES);
  const int np = L.np, ldk = L.ldk, cpq = L.cpq, CR = L.cr, CB = L.cb;
  uint8_t* Yimg = smem;                        // nview x y_bytes
  uint8_t* Bimg = smem + L.off_b;
  uint8_t* Vimg = smem + L.off_v;
  float* Gp = reinterpret_cast<float*>(smem);  // np x KP, after the last product
  float* F = reinterpret_cast<float*>(smem + L.off_f);
  float* Vm = F + L.vm;
  float* gd = F + L.gd;
  float* Hm = F + L.hm;
  float* vn = F + L.vn;
  float* aA = F + L.aA;
  float* aB = F + L.aB;
  float* ybA = F + L.ybA;
  float* ybB = F + L.ybB;
  float* ybC = F + L.ybC;
  float* vsc = F + L.vsc;
  float* bsc = F + L.bsc;
  float* spw = F + L.spw;
  float* spart = F + L.spart;
  float* sown = F + L.sown;
  float* sAt = F + L.sAt;
  float* sBt = F + L.sBt;
  float* sCt = F + L.sCt;
  unsigned* amax = reinterpret_cast<unsigned*>(F + L.amax);
  uint64_t& mbar = *cx.mbar;
  int& s_abort = *cx.abort;

  for (int idx = tid; idx < k * ldk; idx += TC_THREADS) {
    const int i = idx / ldk, r = idx % ldk;
    Vm[idx] = r < k ? a.V[(int64_t)i * k + r] : 0.f;
  }
  for (int r = tid; r < ldk; r += TC_THREADS) {
    ybA[r] = r < k ? (float)a.ybar3[r] : 0.f;
    ybB[r] = r < k ? (float)a.ybar3[k + r] : 0.f;
    ybC[r] = r < k ? (float)a.ybar3[2 * k + r] : 0.f;
  }
  __syncthreads();
  const uint32_t tmem = cx.tmem;
  const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
  const uint32_t colA = 0, colB = SYM ? 0 : 128, colG = 256;
  const int own_lo = q * cpq, own_hi = min(k, own_lo + cpq);
  const int64_t bq = (a.b + CL - 1) / CL;
  const int nchunk = np / 16;
  uint32_t phase = cx.phase;

  for (int64_t s = 0; s < a.total_steps; ++s) {
    const int64_t e = s / a.spe, jb = s % a.spe;
    const int64_t pos0 = jb * a.b;
    const int64_t beff = min(a.b, a.n - pos0);
    const float beta = (float)(a.beta0 / sqrt((double)(s + 1)));
    const float inv_b = 1.f / (float)beff;

    // -- per-step: a_A, a_B, V scales, V image --
    for (int i = warp; i < np; i += TC_THREADS / 32) {
      float x = 0.f, y = 0.f, m = 0.f;
      if (i < k)
        for (int r = lane; r < k; r += 32) {
          const float v = Vm[i * ldk + r];
          x = fmaf(v, ybA[r], x);
          y = fmaf(v, ybB[r], y);
          m = fmaxf(m, fabsf(v));
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      }
      if (lane == 0) {
        aA[i] = x;
        aB[i] = y;
        vsc[i] = FP8 ? (m > 0.f ? m / QMAX : 1.f) : 1.f;
        spart[i] = 0.f;
      }
      if (lane < 4) spw[lane * np + i] = 0.f;
    }
    __syncthreads();
    // V image: 16-byte core rows of (component i, coordinate group rg)
    for (int idx = tid; idx < np * CR; idx += TC_THREADS) {
      const int i = idx / CR, rg = idx % CR;
      const int r0 = rg * (16 / ES);
      const float inv = 1.f / vsc[i];
      float v[16];
#pragma unroll
      for (int z = 0; z < 16 / ES; ++z) {
        const int r = r0 + z;
        v[z] = (i < k && r < k) ? Vm[i * ldk + r] * inv : 0.f;
      }
      uint4 w;
      if constexpr (FP8) {
        w.x = pack_e4m3(v[0], v[1], v[2], v[3]);
        w.y = pack_e4m3(v[4], v[5], v[6], v[7]);
        w.z = pack_e4m3(v[8], v[9], v[10], v[11]);
        w.w = pack_e4m3(v[12], v[13], v[14], v[15]);
      } else {
        w.x = pack_bf16(v[0], v[1]);
        w.y = pack_bf16(v[2], v[3]);
        w.z = pack_bf16(v[4], v[5]);
        w.w = pack_bf16(v[6], v[7]);
      }
      *reinterpret_cast<uint4*>(Vimg + ((size_t)((i >> 3) * CR + rg) << 7) + ((i & 7) << 4)) = w;
    }

    // per-thread accumulators of the second product (this thread's TMEM lane,
    // chunks c = half, half + 2, ...)
    float gacc[4][16];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int j = 0; j < 16; ++j) gacc[c][j] = 0.f;

    const int64_t my_lo = (int64_t)q * bq, my_hi = min(beff, my_lo + bq);
    for (int64_t t0 = my_lo; t0 < my_hi; t0 += TILE) {
      // -- sample tile(s) into the operand images --
      for (int idx = tid; idx < TILE * CR; idx += TC_THREADS) {
        const int t = idx / CR, rg = idx % CR;
        const int64_t p = t0 + t;
        int64_t row = p < my_hi ? (a.perm ? (int64_t)a.perm[e * a.n + pos0 + p] : pos0 + p) : -1;
        if (row >= a.n) row = -1;
        const int c0 = rg * (16 / ES);
        const size_t off = ((size_t)((t >> 3) * CR + rg) << 7) + ((t & 7) << 4);
        const bool in = row >= 0 && c0 < a.ldq;
        const size_t goff = (size_t)row * a.ldq * ES + (size_t)c0 * ES;
        const uint4 z4 = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(Yimg + off) =
            in ? *reinterpret_cast<const uint4*>(a.YA + goff) : z4;
        if (!SYM) {
          *reinterpret_cast<uint4*>(Yimg + L.y_bytes + off) =
              in ? *reinterpret_cast<const uint4*>(a.YB + goff) : z4;
          *reinterpret_cast<uint4*>(Yimg + 2 * L.y_bytes + off) =
              in ? *reinterpret_cast<const uint4*>(a.YC + goff) : z4;
        }
        if (rg == 0) {
          sAt[t] = row >= 0 ? (a.sA ? a.sA[row] : 1.f) : 0.f;
          sBt[t] = row >= 0 ? (a.sB ? a.sB[row] : 1.f) : 0.f;
          sCt[t] = row >= 0 ? (a.sC ? a.sC[row] : 1.f) : 0.f;
        }
        if (FP8 && idx < np) amax[idx] = 0u;
      }
      fence_async_smem();
      tc_before();
      __syncthreads();
      tc_after();
      // -- first product: D1 = Y_tile V^T (K-major operands) --
      if (tid == 0 && !s_abort) {
        const uint32_t id1 = make_idesc(FMT, 0, 0, TILE, (uint32_t)np);
        for (int v = 0; v < (SYM ? 1 : 2); ++v) {
          const uint8_t* Y = Yimg + v * L.y_bytes;
          const uint32_t col = v == 0 ? colA : colB;
          for (int ks = 0; ks < KP / KSTEP; ++ks) {
            const uint64_t da = sdesc(Y + ks * 256, 128, (uint32_t)CR * 128);
            const uint64_t db = sdesc(Vimg + ks * 256, 128, (uint32_t)CR * 128);
            mma<FP8>(tmem + col, da, db, id1, ks > 0 ? 1u : 0u);
          }
        }
        mma_commit(&mbar);
      }
      if (!mbar_wait(&mbar, phase) && lane == 0) {
        s_abort = 1;
        atomicExch(a.err, 1);
      }
      phase ^= 1u;
      tc_after();
      // -- epilogue 1: B = c1 A_A o A_B - c2 (a_B o A_A + a_A o A_B), per-column s --
      {
        const int t = 32 * quad + lane;
        const float sa = sAt[t], sb = sBt[t], sc = sCt[t];
        float bv[4][16];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int ch = half + 2 * c;
          if (ch < nchunk) {
            float xa[16], xb[16];
            tmem_ld16(tmem + lane_base + colA + 16 * ch, xa);
            if (!SYM) tmem_ld16(tmem + lane_base + colB + 16 * ch, xb);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int i = 16 * ch + j;
              const float va = xa[j] * sa * vsc[i];
              const float vb = SYM ? va : xb[j] * sb * vsc[i];
              const float pr = va * vb;
              bv[c][j] = sc * (a.c1 * pr - a.c2 * (aB[i] * va + aA[i] * vb));
              float ps = pr;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
              if (lane == 0) spw[quad * np + i] += ps;
              if (FP8) {
                float m = fabsf(bv[c][j]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) atomicMax(&amax[i], __float_as_uint(m));
              }
            }
          }
        }
        if (FP8) {
          __syncthreads();
          if (tid < np) bsc[tid] = amax[tid] > 0u ? __uint_as_float(amax[tid]) / QMAX : 1.f;
          __syncthreads();
        }
        // B image (MN-major: core (tg, ng) = 8 samples x 16 B of components)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int ch = half + 2 * c;
          if (ch < nchunk) {
            float w[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = FP8 ? bv[c][j] / bsc[16 * ch + j] : bv[c][j];
            if constexpr (FP8) {
              uint4 u;
              u.x = pack_e4m3(w[0], w[1], w[2], w[3]);
              u.y = pack_e4m3(w[4], w[5], w[6], w[7]);
              u.z = pack_e4m3(w[8], w[9], w[10], w[11]);
              u.w = pack_e4m3(w[12], w[13], w[14], w[15]);
              *reinterpret_cast<uint4*>(Bimg + ((size_t)((t >> 3) * CB + ch) << 7) +
                                        ((t & 7) << 4)) = u;
            } else {
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                uint4 u;
                u.x = pack_bf16(w[8 * hh + 0], w[8 * hh + 1]);
                u.y = pack_bf16(w[8 * hh + 2], w[8 * hh + 3]);
                u.z = pack_bf16(w[8 * hh + 4], w[8 * hh + 5]);
                u.w = pack_bf16(w[8 * hh + 6], w[8 * hh + 7]);
                *reinterpret_cast<uint4*>(Bimg + ((size_t)((t >> 3) * CB + 2 * ch + hh) << 7) +
                                          ((t & 7) << 4)) = u;
              }
            }
          }
        }
      }
      fence_async_smem();
      tc_before();
      __syncthreads();
      tc_after();
      // -- second product: D2 = Y_C^T B (MN-major operands) --
      if (tid == 0 && !s_abort) {
        const uint32_t id2 = make_idesc(FMT, 1, 1, KP, (uint32_t)np);
        const uint8_t* YC = Yimg + (SYM ? 0 : 2 * L.y_bytes);
        for (int ks = 0; ks < TILE / KSTEP; ++ks) {
          const uint64_t da =
              sdesc(YC + (size_t)ks * (KSTEP / 8) * CR * 128, (uint32_t)CR * 128, 128);
          const uint64_t db =
              sdesc(Bimg + (size_t)ks * (KSTEP / 8) * CB * 128, (uint32_t)CB * 128, 128);
          mma<FP8>(tmem + colG, da, db, id2, ks > 0 ? 1u : 0u);
        }
        mma_commit(&mbar);
      }
      if (!mbar_wait(&mbar, phase) && lane == 0) {
        s_abort = 1;
        atomicExch(a.err, 1);
      }
      phase ^= 1u;
      tc_after();
      // -- epilogue 2: accumulate beta_i D2[r][i] for this thread's coordinate r --
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ch = half + 2 * c;
        if (ch < nchunk) {
          float x[16];
          tmem_ld16(tmem + lane_base + colG + 16 * ch, x);
#pragma unroll
          for (int j = 0; j < 16; ++j) gacc[c][j] = fmaf(x[j], FP8 ? bsc[16 * ch + j] : 1.f, gacc[c][j]);
        }
      }
      tc_before();
      __syncthreads();  // operand images free for the next tile
      tc_after();
    }
    // partial G to shared memory, column i contiguous: Gp[i * KP + r]
    {
      const int r = 32 * quad + lane;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ch = half + 2 * c;
        if (ch < nchunk) {
#pragma unroll
          for (int j = 0; j < 16; ++j) Gp[(16 * ch + j) * KP + r] = gacc[c][j];
        }
      }
      for (int i = tid; i < np; i += TC_THREADS)
        spart[i] = spw[i] + spw[np + i] + spw[2 * np + i] + spw[3 * np + i];
    }
    cluster.sync();  // partial products of every CTA visible

    // -- owned columns: cluster sums, Gram term, update (FP32) --
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
    for (int idx = tid; idx < nown * k; idx += TC_THREADS) {
      const int jj = idx / k, r = idx % k;
      float part[CL];
#pragma unroll
      for (int c = 0; c < CL; ++c) part[c] = cluster.map_shared_rank(Gp, c)[(own_lo + jj) * KP + r];
      float g = 0.f;
#pragma unroll
      for (int c = 0; c < CL; ++c) g += part[c];
      gd[jj * ldk + r] = g;
    }
    for (int idx = tid; idx < nown * k; idx += TC_THREADS) {
      const int jj = idx / k, j = idx % k;
      const float* vi = Vm + (own_lo + jj) * ldk;
      const float* vj = Vm + j * ldk;
      float h = 0.f;
      for (int r = 0; r < ldk; r += 4) {
        const float4 x = *reinterpret_cast<const float4*>(vi + r);
        const float4 y = *reinterpret_cast<const float4*>(vj + r);
        h = fmaf(x.x, y.x, h);
        h = fmaf(x.y, y.y, h);
        h = fmaf(x.z, y.z, h);
        h = fmaf(x.w, y.w, h);
      }
      Hm[jj * ldk + j] = h * h;
    }
    __syncthreads();
    for (int idx = tid; idx < nown * k; idx += TC_THREADS) {
      const int jj = idx / k, r = idx % k;
      const int i = own_lo + jj;
      float g = 0.f;
      for (int j = 0; j < k; ++j) g = fmaf(Hm[jj * ldk + j], Vm[j * ldk + r], g);
      const float gdata =
          gd[jj * ldk + r] * inv_b + ybC[r] * (a.c3 * aA[i] * aB[i] - a.c2 * sown[jj] * inv_b);
      vn[jj * ldk + r] = Vm[i * ldk + r] - beta * (a.kappa * g - gdata);
    }
    cluster.sync();  // every owner's new columns ready; all reads of V and Gp done
    // pull the new V from the owners
    for (int idx = tid; idx < k * k; idx += TC_THREADS) {
      const int i = idx / k, r = idx % k;
      const int owner = i / cpq, jj = i % cpq;
      Vm[i * ldk + r] = cluster.map_shared_rank(vn, owner)[jj * ldk + r];
    }
    __syncthreads();
    if (a.snapshot_every > 0 && (s + 1) % a.snapshot_every == 0) {
      float* dst = a.V_snap + ((s + 1) / a.snapshot_every - 1) * (int64_t)k * k;
      for (int idx = tid; idx < nown * k; idx += TC_THREADS) {
        const int jj = idx / k, r = idx % k;
        dst[(int64_t)(own_lo + jj) * k + r] = Vm[(own_lo + jj) * ldk + r];
      }
    }
  }
  for (int idx = tid; idx < (own_hi - own_lo) * k; idx += TC_THREADS) {
    const int jj = idx / k, r = idx % k;
    a.V[(int64_t)(own_lo + jj) * k + r] = Vm[(own_lo + jj) * ldk + r];
  }
  cx.phase = phase;
  // no CTA may leave (or reuse its shared memory) while others still read it
  cluster.sync();
}

template <bool FP8, bool SYM, int CL>
__device__ __forceinline__ void tc_setup(TcCtx& cx, uint64_t* mbar, uint32_t* tmem_base,
                                         int* s_abort) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    *s_abort = 0;
  }
  tc_before();
  __syncthreads();
  tc_after();
  cx.mbar = mbar;
  cx.abort = s_abort;
  cx.tmem = *tmem_base;
  cx.phase = 0;
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
  tc_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

template <bool FP8, bool SYM, int CL>
__global__ void __launch_bounds__(TC_THREADS, 1) sgd_tc_kernel(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  TcCtx cx;
  tc_setup<FP8, SYM, CL>(cx, &mbar, &tmem_base, &s_abort);
  tc_chain<FP8, SYM, CL>(a, smem, cx);
  tc_teardown(cx.tmem);
}

// Persistent batched form: every cluster takes (problem, restart) chains from
// a cost-ordered work list until it is exhausted.  Cluster rank 0 claims the
// next item with one atomic and broadcasts it through distributed shared memory.
template <bool FP8, bool SYM, int CL>
__global__ void __launch_bounds__(TC_THREADS, 1) sgd_tc_batched_kernel(const TcArgs* __restrict__ items,
                                                                       int nitems, int* counter) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  __shared__ int s_item;
  cg::cluster_group cluster = cg::this_cluster();
  TcCtx cx;
  tc_setup<FP8, SYM, CL>(cx, &mbar, &tmem_base, &s_abort);
  while (true) {
    if (cluster.block_rank() == 0 && threadIdx.x == 0) {
      const int it = atomicAdd(counter, 1);
#pragma unroll
      for (int c = 0; c < CL; ++c) *cluster.map_shared_rank(&s_item, c) = it;
    }
    cluster.sync();
    const int it = s_item;
    if (it >= nitems) break;
    const TcArgs a = items[it];
    tc_chain<FP8, SYM, CL>(a, smem, cx);
  }
  tc_teardown(cx.tmem);
}

// quantise rows: FP8 -> per-row scale amax/448; BF16 -> scale 1.  Output row
// stride ldq (zero padded).
template <bool FP8>
__global__ void quantize_rows_kernel(const float* __restrict__ Y, int64_t n, int k, int ldq,
                                     uint8_t* __restrict__ Yq, float* __restrict__ scale) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= n) return;
  const float* y = Y + r * k;
  float m = 0.f;
  for (int c = lane; c < k; c += 32) m = fmaxf(m, fabsf(y[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float sc = FP8 ? (m > 0.f ? m / 448.f : 1.f) : 1.f;
  const float inv = 1.f / sc;
  for (int c = lane; c < ldq; c += 32) {
    const float v = c < k ? y[c] * inv : 0.f;
    if constexpr (FP8) {
      const __nv_fp8_e4m3 q(v);
      Yq[r * ldq + c] = *reinterpret_cast<const uint8_t*>(&q);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      reinterpret_cast<__nv_bfloat16*>(Yq)[r * ldq + c] = h;
    }
  }
  if (lane == 0 && scale) scale[r] = sc;
}

template <bool FP8, bool SYM, int CL>
otm_status launch_tc(const TcArgs& args, cudaStream_t st) {
  const TcLayout L = tc_layout(args.k, CL, SYM, FP8 ? 1 : 2);
  auto kern = sgd_tc_kernel<FP8, SYM, CL>;
  OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  if (CL > 8)
    OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = L.total;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  OTM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, args));
  count_launch();
  return OTM_OK;
}

template <bool FP8, bool SYM>
otm_status launch_tc_cl(const TcArgs& args, int CL, cudaStream_t st) {
  switch (CL) {
    case 16: return launch_tc<FP8, SYM, 16>(args, st);
    case 8: return launch_tc<FP8, SYM, 8>(args, st);
    case 4: return launch_tc<FP8, SYM, 4>(args, st);
    case 2: return launch_tc<FP8, SYM, 2>(args, st);
    default: return launch_tc<FP8, SYM, 1>(args, st);
  }
}

// configure = set the kernel's shared-memory / cluster attributes first (done by
// the prepare call, so that the launch itself issues stream work only)
template <bool FP8, int CL>
otm_status launch_batched_cl(const TcArgs* items, int nitems, int* counter, size_t smem,
                             int nclusters, cudaStream_t st, bool configure) {
  auto kern = sgd_tc_batched_kernel<FP8, true, CL>;
  if (configure) {
    OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (CL > 8)
      OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  }
  if (nitems == 0) return OTM_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL * nclusters, 1, 1);
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  OTM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, items, nitems, counter));
  count_launch();
  return OTM_OK;
}

template <bool FP8>
otm_status launch_batched(int CL, const TcArgs* items, int nitems, int* counter, size_t smem,
                          int nclusters, cudaStream_t st, bool configure) {
  switch (CL) {
    case 16: return launch_batched_cl<FP8, 16>(items, nitems, counter, smem, nclusters, st, configure);
    case 8: return launch_batched_cl<FP8, 8>(items, nitems, counter, smem, nclusters, st, configure);
    case 4: return launch_batched_cl<FP8, 4>(items, nitems, counter, smem, nclusters, st, configure);
    case 2: return launch_batched_cl<FP8, 2>(items, nitems, counter, smem, nclusters, st, configure);
    default: return launch_batched_cl<FP8, 1>(items, nitems, counter, smem, nclusters, st, configure);
  }
}

// clusters of the batched kernel that can be resident at once (persistent grid)
template <bool FP8, int CL>
int resident_clusters_cl(size_t smem) {
  auto kern = sgd_tc_batched_kernel<FP8, true, CL>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = 0;
  }
  return n;
}

template <bool FP8>
int resident_clusters(int CL, size_t smem) {
  switch (CL) {
    case 16: return resident_clusters_cl<FP8, 16>(smem);
    case 8: return resident_clusters_cl<FP8, 8>(smem);
    case 4: return resident_clusters_cl<FP8, 4>(smem);
    case 2: return resident_clusters_cl<FP8, 2>(smem);
    default: return resident_clusters_cl<FP8, 1>(smem);
  }
}

int num_sms_tc() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 148;
  }
  return v;
}

// Persistent grid: as many clusters as are resident at once (the occupancy
// query; one CTA per SM if it is unavailable).  Call after the kernel's
// attributes are set.
int batched_clusters(bool fp8, int CL, size_t smem) {
  const int n = fp8 ? resident_clusters<true>(CL, smem) : resident_clusters<false>(CL, smem);
  return n > 0 ? n : std::max(1, num_sms_tc() / CL);
}

// autotuner cache: (precision, max k, cluster candidates tried) -> chosen size
std::mutex g_tune_mu;
std::map<long long, int> g_tune_cache;

int max_smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (v <= 0) v = 227 * 1024;
  }
  return v;
}

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

otm_status otm_quantize_samples(const float* Y, int64_t n, int64_t k, int precision, void* Yq,
                                float* scales, void* stream) {
  clear_error();
  OTM_REQUIRE(Y && Yq && n >= 1 && k >= 1 && k <= TC_KMAX, "otm_quantize_samples: bad arguments");
  OTM_REQUIRE(precision == OTM_PREC_BF16 || precision == OTM_PREC_FP8,
              "otm_quantize_samples: precision must be OTM_PREC_BF16 or OTM_PREC_FP8");
  OTM_REQUIRE(precision == OTM_PREC_BF16 || scales, "otm_quantize_samples: FP8 needs scales");
  const int ldq = (int)((k + 15) & ~15);
  cudaStream_t st = as_stream(stream);
  const unsigned grid = (unsigned)((n + 7) / 8);
  if (precision == OTM_PREC_FP8)
    quantize_rows_kernel<true><<<grid, 256, 0, st>>>(Y, n, (int)k, ldq, (uint8_t*)Yq, scales);
  else
    quantize_rows_kernel<false><<<grid, 256, 0, st>>>(Y, n, (int)k, ldq, (uint8_t*)Yq, scales);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

size_t otm_sgd_run_lp_workspace(void) { return 256; }

otm_status otm_sgd_run_lp(float* V, const void* YA, const void* YB, const void* YC,
                          const float* sA, const float* sB, const float* sC, int64_t n, int64_t k,
                          const double* ybar3, const int32_t* perm, int64_t epochs, int64_t b,
                          double beta0, double theta, double alpha0, int precision,
                          int64_t snapshot_every, float* V_snap, void* ws, size_t ws_bytes,
                          void* stream) {
  clear_error();
  OTM_REQUIRE(V && YA && YB && YC && ybar3, "otm_sgd_run_lp: null pointer");
  OTM_REQUIRE(k >= 1 && k <= TC_KMAX, "otm_sgd_run_lp: k=%lld outside [1, %d]", (long long)k,
              TC_KMAX);
  OTM_REQUIRE(n >= 1 && b >= 1 && epochs >= 0, "otm_sgd_run_lp: need n >= 1, b >= 1, epochs >= 0");
  OTM_REQUIRE(precision == OTM_PREC_BF16 || precision == OTM_PREC_FP8,
              "otm_sgd_run_lp: precision must be OTM_PREC_BF16 or OTM_PREC_FP8");
  OTM_REQUIRE(snapshot_every >= 0 && (snapshot_every == 0 || V_snap),
              "otm_sgd_run_lp: V_snap required for snapshots");
  OTM_REQUIRE(ws && ws_bytes >= otm_sgd_run_lp_workspace(), "otm_sgd_run_lp: workspace too small");
  if (epochs == 0) return OTM_OK;
  const bool fp8 = precision == OTM_PREC_FP8;
  const bool sym = (YA == YB) && (YB == YC);
  const int esize = fp8 ? 1 : 2;
  // largest cluster (16, 8, ...) whose CTAs each hold at most a few tiles and
  // whose shared-memory footprint fits
  int CL = 0;
  for (int c : {8, 16, 4, 2, 1}) {
    if (tc_layout((int)k, c, sym, esize).total <= (size_t)max_smem_optin()) {
      CL = c;
      break;
    }
  }
  OTM_REQUIRE(CL > 0, "otm_sgd_run_lp: k=%lld does not fit shared memory with %s views",
              (long long)k, sym ? "one" : "three");
  if (b > 8 * TILE && CL == 8 && tc_layout((int)k, 16, sym, esize).total <= (size_t)max_smem_optin())
    CL = 16;
  cudaStream_t st = as_stream(stream);
  int* err = static_cast<int*>(ws);
  OTM_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  TcArgs args;
  args.YA = static_cast<const uint8_t*>(YA);
  args.YB = static_cast<const uint8_t*>(YB);
  args.YC = static_cast<const uint8_t*>(YC);
  args.sA = sA;
  args.sB = sB;
  args.sC = sC;
  args.perm = perm;
  args.ybar3 = ybar3;
  args.V = V;
  args.V_snap = V_snap;
  args.err = err;
  args.n = n;
  args.b = b;
  args.spe = (n + b - 1) / b;
  args.total_steps = args.spe * epochs;
  args.snapshot_every = snapshot_every;
  args.k = (int)k;
  args.ldq = (int)((k + 15) & ~15);
  args.beta0 = beta0;
  args.c1 = (float)((alpha0 + 1.0) * (alpha0 + 2.0) / 2.0);
  args.c2 = (float)(alpha0 * (alpha0 + 1.0) / 2.0);
  args.c3 = (float)(alpha0 * alpha0);
  args.kappa = (float)(0.5 * (1.0 + theta));
  otm_status s_;
  if (fp8)
    s_ = sym ? launch_tc_cl<true, true>(args, CL, st) : launch_tc_cl<true, false>(args, CL, st);
  else
    s_ = sym ? launch_tc_cl<false, true>(args, CL, st) : launch_tc_cl<false, false>(args, CL, st);
  if (s_ != OTM_OK) return s_;
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h) return set_error(OTM_ETIMEOUT, "otm_sgd_run_lp: a tensor-core wait timed out");
  return OTM_OK;
}

size_t otm_sgd_batched_workspace(int64_t nitems) {
  WorkspaceSize w;
  w.add<int>(64).add<TcArgs>(nitems).add<TcArgs>(nitems).add<float>(
      (size_t)std::min<int64_t>(nitems, 512) * TC_KMAX * TC_KMAX);
  return w.bytes();
}

otm_status otm_sgd_batched_prepare(const otm_problem* probs, int nprob, int precision,
                                   int cluster, void* ws, size_t ws_bytes, otm_batch_plan* plan,
                                   void* stream) {
  clear_error();
  OTM_REQUIRE(probs && nprob >= 1 && plan, "otm_sgd_batched_prepare: bad arguments");
  OTM_REQUIRE(precision == OTM_PREC_BF16 || precision == OTM_PREC_FP8,
              "otm_sgd_batched_prepare: precision must be OTM_PREC_BF16 or OTM_PREC_FP8");
  OTM_REQUIRE(cluster == 0 || cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8 ||
                  cluster == 16,
              "otm_sgd_batched_prepare: cluster must be 0 (autotune), 1, 2, 4, 8 or 16");
  const bool fp8 = precision == OTM_PREC_FP8;
  std::vector<TcArgs> items;
  std::vector<double> cost;
  int max_k = 0;
  for (int p = 0; p < nprob; ++p) {
    const otm_problem& P = probs[p];
    OTM_REQUIRE(P.k >= 1 && P.k <= TC_KMAX && P.n >= 1 && P.b >= 1 && P.epochs >= 0 &&
                    P.restarts >= 1 && P.Yq && P.ybar3 && P.V,
                "otm_sgd_batched_prepare: problem %d invalid (need 1 <= k <= %d, n, b, "
                "restarts >= 1, non-null Yq, ybar3, V)", p, TC_KMAX);
    max_k = std::max(max_k, (int)P.k);
    for (int64_t r = 0; r < P.restarts; ++r) {
      TcArgs a;
      a.YA = a.YB = a.YC = static_cast<const uint8_t*>(P.Yq);
      a.sA = a.sB = a.sC = P.scales;
      a.perm = P.perm;
      a.ybar3 = P.ybar3;
      a.V = P.V + r * P.k * P.k;
      a.V_snap = nullptr;
      a.err = nullptr;
      a.n = P.n;
      a.b = P.b;
      a.spe = (P.n + P.b - 1) / P.b;
      a.total_steps = a.spe * P.epochs;
      a.snapshot_every = 0;
      a.k = (int)P.k;
      a.ldq = (int)((P.k + 15) & ~15);
      a.beta0 = P.beta0;
      a.c1 = (float)((P.alpha0 + 1.0) * (P.alpha0 + 2.0) / 2.0);
      a.c2 = (float)(P.alpha0 * (P.alpha0 + 1.0) / 2.0);
      a.c3 = (float)(P.alpha0 * P.alpha0);
      a.kappa = (float)(0.5 * (1.0 + P.theta));
      items.push_back(a);
      cost.push_back((double)a.total_steps * ((double)P.b * P.k * P.k + (double)P.k * P.k * P.k));
    }
  }
  const int nitems = (int)items.size();
  OTM_REQUIRE(ws_bytes >= otm_sgd_batched_workspace(nitems),
              "otm_sgd_batched_prepare: workspace too small (need %zu bytes)",
              otm_sgd_batched_workspace(nitems));
  // longest chains first: the tail of the persistent loop is then short ones
  std::vector<int> order(nitems);
  for (int i = 0; i < nitems; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<TcArgs> sorted(nitems);
  for (int i = 0; i < nitems; ++i) sorted[i] = items[order[i]];
  Workspace w(ws, ws_bytes);
  int* hdr = w.take<int>(64);
  TcArgs* dev_items = w.take<TcArgs>(nitems);
  TcArgs* trial_items = w.take<TcArgs>(nitems);
  float* scratchV = w.take<float>((size_t)std::min(nitems, 512) * TC_KMAX * TC_KMAX);
  cudaStream_t st = as_stream(stream);
  for (int i = 0; i < nitems; ++i) sorted[i].err = hdr + 1;
  OTM_CHECK_CUDA(cudaMemcpyAsync(dev_items, sorted.data(), sizeof(TcArgs) * nitems,
                                 cudaMemcpyHostToDevice, st));
  OTM_CHECK_CUDA(cudaMemsetAsync(hdr, 0, 64 * sizeof(int), st));
  // feasible cluster sizes: shared memory for the largest k
  std::vector<int> cands;
  for (int c : {1, 2, 4, 8, 16})
    if (tc_layout(max_k, c, true, fp8 ? 1 : 2).total + 1024 <= (size_t)max_smem_optin())
      cands.push_back(c);  // 1 KiB left for the kernel's static shared variables
  OTM_REQUIRE(!cands.empty(), "otm_sgd_batched_prepare: k=%d does not fit shared memory", max_k);
  int chosen = cluster;
  if (chosen != 0) {
    OTM_REQUIRE(std::find(cands.begin(), cands.end(), chosen) != cands.end(),
                "otm_sgd_batched_prepare: cluster %d does not fit k=%d", chosen, max_k);
  } else {
    // autotune: time a short trial (<= 4 steps per chain, on scratch V) for every
    // feasible cluster size; the choice is cached per (precision, max k, items)
    const long long key = ((long long)precision << 40) | ((long long)max_k << 24) | nitems;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto f = g_tune_cache.find(key);
      if (f != g_tune_cache.end()) chosen = f->second;
    }
    if (chosen == 0) {
      const int ntrial = std::min(nitems, 512);
      std::vector<TcArgs> trial(sorted.begin(), sorted.begin() + ntrial);
      for (int i = 0; i < ntrial; ++i) {
        trial[i].V = scratchV + (size_t)i * TC_KMAX * TC_KMAX;
        trial[i].total_steps = std::min<int64_t>(trial[i].total_steps, 4);
      }
      OTM_CHECK_CUDA(cudaMemsetAsync(scratchV, 0, sizeof(float) * ntrial * TC_KMAX * TC_KMAX, st));
      OTM_CHECK_CUDA(cudaMemcpyAsync(trial_items, trial.data(), sizeof(TcArgs) * ntrial,
                                     cudaMemcpyHostToDevice, st));
      cudaEvent_t e0, e1;
      OTM_CHECK_CUDA(cudaEventCreate(&e0));
      OTM_CHECK_CUDA(cudaEventCreate(&e1));
      float best = 3.0e38f;
      for (int c : cands) {
        const size_t smem = tc_layout(max_k, c, true, fp8 ? 1 : 2).total;
        float tot = 0.f;
        // set attributes (zero-item launch) before the occupancy query
        otm_status s1 = fp8 ? launch_batched<true>(c, trial_items, 0, hdr + 8, smem, 1, st, true)
                            : launch_batched<false>(c, trial_items, 0, hdr + 8, smem, 1, st, true);
        if (s1 != OTM_OK) return s1;
        const int ncl = std::min(batched_clusters(fp8, c, smem), ntrial);
        for (int rep = 0; rep < 2; ++rep) {
          OTM_CHECK_CUDA(cudaMemsetAsync(hdr + 8, 0, sizeof(int), st));
          OTM_CHECK_CUDA(cudaEventRecord(e0, st));
          otm_status s2 = fp8 ? launch_batched<true>(c, trial_items, ntrial, hdr + 8, smem, ncl,
                                                     st, false)
                              : launch_batched<false>(c, trial_items, ntrial, hdr + 8, smem, ncl,
                                                      st, false);
          if (s2 != OTM_OK) return s2;
          OTM_CHECK_CUDA(cudaEventRecord(e1, st));
          OTM_CHECK_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          OTM_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (rep == 1) tot = ms;  // second run: code and caches warm
        }
        if (tot < best) {
          best = tot;
          chosen = c;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = chosen;
    }
  }
  {
    const size_t smem = tc_layout(max_k, chosen, true, fp8 ? 1 : 2).total;
    otm_status s3 = fp8 ? launch_batched<true>(chosen, dev_items, 0, hdr, smem, 1, st, true)
                        : launch_batched<false>(chosen, dev_items, 0, hdr, smem, 1, st, true);
    if (s3 != OTM_OK) return s3;
  }
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  plan->nitems = nitems;
  plan->cluster = chosen;
  plan->precision = precision;
  plan->max_k = max_k;
  plan->smem_bytes = (int64_t)tc_layout(max_k, chosen, true, fp8 ? 1 : 2).total;
  plan->grid_clusters =
      std::min(batched_clusters(fp8, chosen, (size_t)plan->smem_bytes), nitems);
  plan->ws = ws;
  plan->ws_bytes = ws_bytes;
  return OTM_OK;
}

otm_status otm_sgd_batched_launch(const otm_batch_plan* plan, void* stream) {
  clear_error();
  OTM_REQUIRE(plan && plan->ws && plan->nitems >= 1 && plan->grid_clusters >= 1,
              "otm_sgd_batched_launch: invalid plan");
  cudaStream_t st = as_stream(stream);
  Workspace w(plan->ws, plan->ws_bytes);
  int* hdr = w.take<int>(64);
  TcArgs* dev_items = w.take<TcArgs>(plan->nitems);
  OTM_CHECK_CUDA(cudaMemsetAsync(hdr, 0, 2 * sizeof(int), st));
  const int c = plan->cluster;
  return plan->precision == OTM_PREC_FP8
             ? launch_batched<true>(c, dev_items, plan->nitems, hdr, (size_t)plan->smem_bytes,
                                    plan->grid_clusters, st, false)
             : launch_batched<false>(c, dev_items, plan->nitems, hdr, (size_t)plan->smem_bytes,
                                     plan->grid_clusters, st, false);
}

otm_status otm_sgd_batched_check(const otm_batch_plan* plan, void* stream) {
  clear_error();
  OTM_REQUIRE(plan && plan->ws, "otm_sgd_batched_check: invalid plan");
  cudaStream_t st = as_stream(stream);
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, static_cast<int*>(plan->ws) + 1, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h) return set_error(OTM_ETIMEOUT, "otm_sgd_batched: a tensor-core wait timed out");
  return OTM_OK;
}

}  // extern "C"
