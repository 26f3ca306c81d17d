// Stochastic tensor gradient descent on the implicit whitened tensor
// (Section 3.2, Lemma 3 / Eq. (16)), FP32, as ONE cooperative launch over
// many SMs -- the "grid" form of the fused step (the cluster form in sgd.cu
// is limited to the 16 SMs of one thread-block cluster).
//
// Per step, for the minibatch Y_b and V (k x k), exactly the quantities of
// the cluster form:
//   A_A = V^T Y_A^T, A_B = V^T Y_B^T; a_A = V^T ybar_A, a_B = V^T ybar_B
//   B   = c1 A_A o A_B - c2 (a_B o A_A + a_A o A_B)
//   s   = (1/b) sum_t (A_A o A_B)[:, t]
//   G_data = (1/b) Y_C^T B^T + ybar_C (c3 a_A o a_B - c2 s)^T
//   G_gram = V ((V^T V) o (V^T V))
//   V <- V - beta_t (kappa G_gram - G_data)
//
// Organisation: G CTAs (one per SM, up to the SM count); CTA g takes samples
// [g S, g S + S) of every minibatch (S = ceil(b / G)), holds a copy of V in
// shared memory, forms A, B and its partial Y_C^T B^T and sum of A_A o A_B,
// and writes the partials to global memory (L2).  Grid barrier.  CTA g then
// owns components i = g, g + G, ...: it sums the G partials of its columns,
// adds the Gram and mean terms, and writes the new column (and its means
// a_A, a_B) to the iterate buffer of the next step.  Grid barrier.  Every CTA
// reloads V from that buffer at the start of the next step (one bulk copy,
// completing on an mbarrier, where the buffers are 16-byte aligned).  Two grid
// barriers per step; the partial sums are added in a fixed order, so the
// result does not depend on timing.  The samples of step s + 1 do not depend
// on V: they are copied (cp.async) into a second buffer at the start of step
// s and land while step s computes and waits at its barriers.
#include "grid_sync.cuh"
#include "otm_internal.cuh"
#include "tc_ptx.cuh"

namespace otm {
namespace {

constexpr int GT = 256;       // threads per CTA
constexpr int G_SAMPLES = 8;  // target samples per CTA per step (k = 100, b = 1024: 128 CTAs)
constexpr int G_SMAX = 32;    // at most this many samples per CTA per step
constexpr int G_KMAX = 128;
constexpr int G_MAXGRID = 160;  // CTAs at most (the owners' sums load G / 8 partials at once)
constexpr int VQ = (G_KMAX * (G_KMAX + 4) / 4 + GT - 1) / GT;  // float4 of V per thread
constexpr int RQ = G_MAXGRID / 8;                              // partials per thread

struct GridArgs {
  const float* YA;
  const float* YB;
  const float* YC;
  const int32_t* perm;
  const double* ybar3;
  float* V;       // k x k, component-major (row i = v_i); initial and final iterate
  float* V_snap;
  float* Vg;      // 2 x kp x ld: the iterate of the next step, by step parity
  float* means;   // 2 x 2 x kp: a_A, a_B of that iterate, by step parity
  float* part;    // G x kp x ld: partial Y_C^T B^T of each CTA (row i = component i)
  float* spart;   // G x kp: partial sums of A_A o A_B
  unsigned* bar;  // grid barrier counter (zero on entry)
  int* flag;      // barrier time-out
  int64_t n, b, spe, total_steps, snapshot_every;
  int k, S;
  int vec;        // sample rows are 16-byte aligned (k % 4 == 0, aligned bases)
  int bulkv;      // Vg and means are 16-byte aligned: V and its means reload by bulk copy
  double beta0;
  float c1, c2, c3, kappa;
};

struct GLayout {
  int kp, ld, nview, S;
  size_t off_v, off_y, off_b, off_p, off_yb, off_a, off_red, off_h, total;
};

// Shared memory (floats).  Rows of V and of the samples have stride ld, an odd
// number of float4s, so that float4 reads of consecutive rows fall in
// different bank groups.
__host__ __device__ inline GLayout g_layout(int k, bool sym, int S) {
  GLayout L;
  L.kp = (k + 3) & ~3;
  L.ld = ((L.kp / 4) & 1) ? L.kp : L.kp + 4;
  L.nview = sym ? 1 : 3;
  L.S = S;
  size_t f = 0;
  L.off_v = f;   f += (size_t)L.kp * L.ld;          // V, component rows
  L.off_y = f;   f += 2 * (size_t)L.nview * S * L.ld;  // this CTA's samples [step parity][view][t]
  L.off_b = f;   f += (size_t)S * L.kp;             // B [t][i]
  L.off_p = f;   f += (size_t)S * L.kp;             // A_A o A_B [t][i]
  L.off_yb = f;  f += 3 * (size_t)L.ld;             // ybar_A, ybar_B, ybar_C
  L.off_a = f;   f += 2 * (size_t)L.kp;             // a_A, a_B
  L.off_red = f; f += 16 * (size_t)L.kp;            // 8 partial rows of Y_C^T B^T, 8 of G_gram
  L.off_h = f;   f += (size_t)L.kp;                 // (v_i . v_j)^2 of an owned column i
  L.total = f;
  return L;
}

__device__ __forceinline__ void fma4(float4& acc, float s, const float4& v) {
  acc.x = fmaf(s, v.x, acc.x);
  acc.y = fmaf(s, v.y, acc.y);
  acc.z = fmaf(s, v.z, acc.z);
  acc.w = fmaf(s, v.w, acc.w);
}
__device__ __forceinline__ float dot4(const float4& a, const float4& b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}

template <bool SYM>
__global__ void __launch_bounds__(GT, 1) sgd_grid_kernel(GridArgs a) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float s_red[2][GT / 32];
  __shared__ float s_si;
  __shared__ int s_row[2][G_SMAX];  // sample rows of this CTA, by step parity (-1: none)
  __shared__ __align__(8) uint64_t s_vb;  // completion of the bulk reload of V and its means
  const int g = blockIdx.x, G = gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k;
  const GLayout L = g_layout(k, SYM, a.S);
  const int kp = L.kp, ld = L.ld, S = L.S, kq = kp / 4;
  float* Vs = sm + L.off_v;
  float* Ys = sm + L.off_y;
  float* Bs = sm + L.off_b;
  float* Ps = sm + L.off_p;
  float* ybA = sm + L.off_yb;
  float* ybB = ybA + ld;
  float* ybC = ybB + ld;
  float* aA = sm + L.off_a;
  float* aB = aA + kp;
  float* red = sm + L.off_red;
  float* redg = red + 8 * kp;
  float* hs = sm + L.off_h;
  // on a barrier time-out the owned columns of V are set to NaN (the caller
  // sees the failure in the result) and the CTA returns
  auto fail = [&]() {
    tc::cp_async_wait(0);  // no copy into shared memory outlives the CTA
    for (int i = g; i < k; i += G)
      for (int r = tid; r < k; r += GT) a.V[(int64_t)i * k + r] = __int_as_float(0x7fc00000);
  };

  for (int r = tid; r < ld; r += GT) {
    ybA[r] = r < k ? (float)a.ybar3[r] : 0.f;
    ybB[r] = r < k ? (float)a.ybar3[k + r] : 0.f;
    ybC[r] = r < k ? (float)a.ybar3[2 * k + r] : 0.f;
  }
  for (int idx = tid; idx < kp * ld; idx += GT) {
    const int i = idx / ld, r = idx % ld;
    Vs[idx] = (i < k && r < k) ? a.V[(int64_t)i * k + r] : 0.f;
  }
  // padding rows of both iterate buffers and their means stay zero
  if (g == 0) {
    for (int idx = tid; idx < 2 * (kp - k) * ld; idx += GT) {
      const int bsel = idx / ((kp - k) * ld), rem = idx % ((kp - k) * ld);
      a.Vg[(size_t)bsel * kp * ld + (size_t)k * ld + rem] = 0.f;
    }
    for (int idx = tid; idx < 2 * 2 * (kp - k); idx += GT) {
      const int q = idx / (kp - k), i = k + idx % (kp - k);
      a.means[(size_t)q * kp + i] = 0.f;
    }
  }
  // row of sample t of this CTA in step s (-1 outside the minibatch or for an
  // index outside [0, n), which reads as a zero sample)
  auto row_of = [&](int64_t s, int t) -> int {
    if (s >= a.total_steps) return -1;
    const int64_t e = s / a.spe, pos0 = (s % a.spe) * a.b;
    const int64_t beff = min(a.b, a.n - pos0), p = (int64_t)g * S + t;
    if (p >= beff) return -1;
    const int64_t row = a.perm ? (int64_t)a.perm[e * a.n + pos0 + p] : pos0 + p;
    return (row >= 0 && row < a.n) ? (int)row : -1;
  };
  // copies of the samples of a step into buffer `buf` (zero rows outside the
  // minibatch); one cp.async group per call
  const size_t ybuf = (size_t)L.nview * S * ld;
  auto issue_samples = [&](int buf) {
    float* dstb = Ys + (size_t)buf * ybuf;
    const int ny = L.nview * S * kq;
#pragma unroll 1
    for (int idx = tid; idx < ny; idx += GT) {
      const int v = idx / (S * kq), rem = idx % (S * kq), t = rem / kq, r = 4 * (rem % kq);
      const float* Yg = v == 0 ? a.YA : (v == 1 ? a.YB : a.YC);
      const int row = s_row[buf][t];
      float* dst = dstb + ((size_t)v * S + t) * ld + r;
      const float* src = row >= 0 ? Yg + (int64_t)row * k + r : Yg;
      if (a.vec) {
        tc::cp_async16(dst, src, row >= 0 ? 16u : 0u);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          tc::cp_async4(dst + j, row >= 0 && r + j < k ? src + j : Yg,
                        row >= 0 && r + j < k ? 4u : 0u);
      }
    }
    tc::cp_async_commit();
  };
  if (tid < S) s_row[0][tid] = row_of(0, tid);
  if (tid == 0) {
    tc::mbar_init(&s_vb, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  issue_samples(0);
  uint32_t vph = 0;  // phase of s_vb
  const uint32_t vbytes = (uint32_t)(kp * ld * sizeof(float)), mbytes = (uint32_t)(2 * kp * sizeof(float));
  for (int i = warp; i < kp; i += GT / 32) {  // a_A, a_B of the initial V
    float x = 0.f, y = 0.f;
    for (int r = lane; r < kp; r += 32) {
      x = fmaf(Vs[i * ld + r], ybA[r], x);
      y = fmaf(Vs[i * ld + r], ybB[r], y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) {
      aA[i] = x;
      aB[i] = y;
    }
  }

  for (int64_t s = 0; s < a.total_steps; ++s) {
    const int par = (int)(s & 1);
    float* Vnext = a.Vg + (size_t)(par ^ 1) * kp * ld;
    float* Mnext = a.means + (size_t)(par ^ 1) * 2 * kp;
    const int64_t pos0 = (s % a.spe) * a.b;
    const int64_t beff = min(a.b, a.n - pos0);
    // rows of the next step's samples; the iterate the owners wrote in the
    // previous step and its means (every load issued before any store)
    if (tid < S) s_row[par ^ 1][tid] = row_of(s + 1, tid);
    if (a.bulkv) {
      // every generic access of Vs and aA of the last step is behind the grid
      // barrier's CTA barrier; the owners fenced their writes for the async proxy
      if (s > 0 && tid == 0) {
        tc::fence_async_smem();
        tc::mbar_expect_tx(&s_vb, vbytes + mbytes);
        tc::bulk_g2s(Vs, a.Vg + (size_t)par * kp * ld, vbytes, &s_vb);
        tc::bulk_g2s(aA, a.means + (size_t)par * 2 * kp, mbytes, &s_vb);
      }
    } else {
      float4 vv[VQ];
      const int nv4 = s > 0 ? kp * ld / 4 : 0;
      const float4* src = reinterpret_cast<const float4*>(a.Vg + (size_t)par * kp * ld);
#pragma unroll
      for (int c = 0; c < VQ; ++c) {
        const int idx = tid + c * GT;
        if (idx < nv4) vv[c] = __ldcg(src + idx);
      }
      if (s > 0) {
        const float* msrc = a.means + (size_t)par * 2 * kp;
        for (int idx = tid; idx < 2 * kp; idx += GT) aA[idx] = __ldcg(msrc + idx);  // aA, aB
      }
      float4* dst = reinterpret_cast<float4*>(Vs);
#pragma unroll
      for (int c = 0; c < VQ; ++c) {
        const int idx = tid + c * GT;
        if (idx < nv4) dst[idx] = vv[c];
      }
    }
    __syncthreads();  // s_row of the next step
    issue_samples(par ^ 1);
    if (a.bulkv && s > 0) {
      const bool ok = tc::mbar_wait(&s_vb, vph);
      vph ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(a.flag, 1);
        fail();
        return;
      }
    }
    tc::cp_async_wait(1);  // this step's samples (issued one step earlier) have landed
    __syncthreads();
    const float* Yst = Ys + (size_t)par * ybuf;

    // A_A, A_B for 4 components x 1 sample per item (consecutive threads take
    // consecutive samples), then B and A_A o A_B
    for (int item = tid; item < S * kq; item += GT) {
      const int t = item % S, i0 = 4 * (item / S);
      const float* ya = Yst + (size_t)t * ld;
      const float* yb = SYM ? ya : Yst + ((size_t)S + t) * ld;
      float xa[4] = {0.f, 0.f, 0.f, 0.f}, xb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
      for (int r = 0; r < kp; r += 4) {
        const float4 yA = *reinterpret_cast<const float4*>(ya + r);
        const float4 yB = SYM ? yA : *reinterpret_cast<const float4*>(yb + r);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 v = *reinterpret_cast<const float4*>(Vs + (i0 + j) * ld + r);
          xa[j] = dot4(v, yA, xa[j]);
          if (!SYM) xb[j] = dot4(v, yB, xb[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = i0 + j;
        const float xA = xa[j], xB = SYM ? xa[j] : xb[j];
        const float pr = xA * xB;
        Ps[t * kp + i] = pr;
        Bs[t * kp + i] = a.c1 * pr - a.c2 * (aB[i] * xA + aA[i] * xB);
      }
    }
    __syncthreads();
    // partial sums of A_A o A_B and partial Y_C^T B^T (4 x 4 tiles) to L2
    for (int i = tid; i < kp; i += GT) {
      float sum = 0.f;
      for (int t = 0; t < S; ++t) sum += Ps[t * kp + i];
      a.spart[(size_t)g * kp + i] = sum;
    }
    {
      float* pg = a.part + (size_t)g * kp * ld;
      const float* yc = SYM ? Yst : Yst + 2 * (size_t)S * ld;
      for (int tile = tid; tile < kq * kq; tile += GT) {
        const int r0 = 4 * (tile % kq), i0 = 4 * (tile / kq);
        float4 acc[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[x] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int t = 0; t < S; ++t) {
          const float4 bt = *reinterpret_cast<const float4*>(Bs + t * kp + i0);
          const float4 y4 = *reinterpret_cast<const float4*>(yc + (size_t)t * ld + r0);
          fma4(acc[0], bt.x, y4);
          fma4(acc[1], bt.y, y4);
          fma4(acc[2], bt.z, y4);
          fma4(acc[3], bt.w, y4);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
          *reinterpret_cast<float4*>(pg + (size_t)(i0 + x) * ld + r0) = acc[x];
      }
    }
    if (!grid_barrier(a.bar, a.flag, 1)) {
      fail();
      return;
    }

    // owned components: sum the partials, Gram term, update, means
    const float beta = (float)a.beta0 / sqrtf((float)(s + 1));
    const float inv_b = 1.f / (float)beff;
    for (int i = g; i < k; i += G) {
      // the partials of column i are loaded first; the Gram term, which needs
      // only V, is computed while they are in flight
      const int h = tid >> 5, q = tid & 31;  // 8 groups x 32 float4 columns (kq <= 32)
      float4 p[RQ];
      if (q < kq) {
#pragma unroll
        for (int c = 0; c < RQ; ++c) {
          const int gg = h + 8 * c;
          p[c] = gg < G ? __ldcg(reinterpret_cast<const float4*>(
                              a.part + ((size_t)gg * kp + i) * ld + 4 * q))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      float sv[G_MAXGRID / 32];
      if (warp == 0) {
#pragma unroll
        for (int c = 0; c < G_MAXGRID / 32; ++c) {
          const int gg = lane + 32 * c;
          sv[c] = gg < G ? __ldcg(a.spart + (size_t)gg * kp + i) : 0.f;
        }
      }
      for (int j = tid; j < kp; j += GT) {  // (v_i . v_j)^2
        const float* vi = Vs + (size_t)i * ld;
        const float* vj = Vs + (size_t)j * ld;
        float h0 = 0.f, h1 = 0.f;
        for (int r = 0; r < kp; r += 8) {
          h0 = dot4(*reinterpret_cast<const float4*>(vi + r),
                    *reinterpret_cast<const float4*>(vj + r), h0);
          if (r + 4 < kp)
            h1 = dot4(*reinterpret_cast<const float4*>(vi + r + 4),
                      *reinterpret_cast<const float4*>(vj + r + 4), h1);
        }
        const float hv = h0 + h1;
        hs[j] = hv * hv;
      }
      __syncthreads();
      if (q < kq) {  // Gram term, components j = h (mod 8)
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = h; j < k; j += 8)
          fma4(acc, hs[j], *reinterpret_cast<const float4*>(Vs + (size_t)j * ld + 4 * q));
        *reinterpret_cast<float4*>(redg + h * kp + 4 * q) = acc;
        float4 t = p[0];
#pragma unroll
        for (int c = 1; c < RQ; ++c) {
          t.x += p[c].x;
          t.y += p[c].y;
          t.z += p[c].z;
          t.w += p[c].w;
        }
        *reinterpret_cast<float4*>(red + h * kp + 4 * q) = t;
      }
      if (warp == 0) {
        float v = sv[0];
#pragma unroll
        for (int c = 1; c < G_MAXGRID / 32; ++c) v += sv[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_si = v;
      }
      __syncthreads();
      {
        const float si = s_si;
        const float mean_term = a.c3 * aA[i] * aB[i] - a.c2 * si * inv_b;
        float x = 0.f, y = 0.f;
        for (int r = tid; r < kp; r += GT) {
          float gg = 0.f, gdr = 0.f;
#pragma unroll
          for (int hh = 0; hh < 8; ++hh) {
            gg += redg[hh * kp + r];
            gdr += red[hh * kp + r];
          }
          const float gdata = gdr * inv_b + ybC[r] * mean_term;
          const float v = r < k ? Vs[(size_t)i * ld + r] - beta * (a.kappa * gg - gdata) : 0.f;
          Vnext[(size_t)i * ld + r] = v;
          x = fmaf(v, ybA[r], x);
          y = fmaf(v, ybB[r], y);
          if (r < k) {
            if (a.snapshot_every > 0 && (s + 1) % a.snapshot_every == 0)
              a.V_snap[((s + 1) / a.snapshot_every - 1) * (int64_t)k * k + (int64_t)i * k + r] = v;
            if (s + 1 == a.total_steps) a.V[(int64_t)i * k + r] = v;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          x += __shfl_xor_sync(0xffffffffu, x, o);
          y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (lane == 0) {
          s_red[0][warp] = x;
          s_red[1][warp] = y;
        }
        __syncthreads();
        if (tid == 0) {
          float tx = 0.f, ty = 0.f;
#pragma unroll
          for (int w = 0; w < GT / 32; ++w) {
            tx += s_red[0][w];
            ty += s_red[1][w];
          }
          Mnext[i] = tx;
          Mnext[kp + i] = ty;
        }
        __syncthreads();  // shared scratch is reused by the next owned column
      }
    }
    if (a.bulkv) tc::fence_async_global();  // the new columns are read by bulk copies
    if (!grid_barrier(a.bar, a.flag, 1)) {
      fail();
      return;
    }
  }
  tc::cp_async_wait(0);  // the last (empty) prefetch
}

unsigned grid_sms() {
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (sms[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? v : 1;
  }
  return (unsigned)sms[dev];
}

template <bool SYM>
otm_status launch_grid(GridArgs& args, int G, cudaStream_t st) {
  const GLayout L = g_layout(args.k, SYM, args.S);
  const size_t smem = L.total * sizeof(float);
  auto kern = sgd_grid_kernel<SYM>;
  OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  void* kargs[] = {&args};
  OTM_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(GT), kargs, smem, st));
  count_launch();
  return OTM_OK;
}

}  // namespace

// CTAs of the grid form for minibatch b: about G_SAMPLES samples each, at
// most one per SM.
static int grid_ctas(int64_t b) {
  const int64_t want = (b + G_SAMPLES - 1) / G_SAMPLES;
  return (int)std::min<int64_t>(std::min<int64_t>(grid_sms(), G_MAXGRID), want);
}

// Scratch of the grid form: the iterate by step parity and its means, the
// partial products and sums of every CTA, the barrier counter and a flag.
static WorkspaceSize grid_ws(int64_t k, int64_t b) {
  const GLayout L = g_layout((int)k, false, 1);  // kp and ld do not depend on the views
  const int G = grid_ctas(b);
  WorkspaceSize w;
  w.add<float>(2 * (size_t)L.kp * L.ld).add<float>(4 * (size_t)L.kp);
  w.add<float>((size_t)G * L.kp * L.ld).add<float>((size_t)G * L.kp);
  w.add<unsigned>(1).add<int>(1);
  return w;
}

size_t sgd_grid_workspace(int64_t k, int64_t b) {
  return sgd_grid_applicable(k, b) ? grid_ws(k, b).bytes() : 0;
}

bool sgd_grid_applicable(int64_t k, int64_t b) {
  const int64_t gmax = std::min<int64_t>(grid_sms(), G_MAXGRID);
  return k >= 1 && k <= G_KMAX && b >= 16 && b <= (int64_t)G_SMAX * gmax;
}

otm_status sgd_grid_run(float* V, const float* YA, const float* YB, const float* YC, int64_t n,
                        int64_t k, const double* ybar3, const int32_t* perm, int64_t epochs,
                        int64_t b, double beta0, double theta, double alpha0,
                        int64_t snapshot_every, float* V_snap, void* ws_ptr, size_t ws_bytes,
                        cudaStream_t st) {
  if (!sgd_grid_applicable(k, b)) return set_error(OTM_EINVAL, "sgd grid form: k or b out of range");
  const bool sym = (YA == YB) && (YB == YC);
  const int G = grid_ctas(b);
  const int S = (int)((b + G - 1) / G);
  if (S > G_SMAX) return set_error(OTM_EINVAL, "sgd grid form: minibatch too large for the grid");
  GridArgs args;
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
  args.S = S;
  args.vec = (k % 4 == 0) && ((reinterpret_cast<uintptr_t>(YA) | reinterpret_cast<uintptr_t>(YB) |
                                reinterpret_cast<uintptr_t>(YC)) & 15) == 0;
  args.beta0 = beta0;
  args.c1 = (float)((alpha0 + 1.0) * (alpha0 + 2.0) / 2.0);
  args.c2 = (float)(alpha0 * (alpha0 + 1.0) / 2.0);
  args.c3 = (float)(alpha0 * alpha0);
  args.kappa = (float)(0.5 * (1.0 + theta));
  const GLayout L = g_layout((int)k, sym, S);
  if (!ws_ptr || ws_bytes < grid_ws(k, b).bytes())
    return set_error(OTM_EINVAL, "sgd grid form: workspace too small (need %zu bytes)",
                     grid_ws(k, b).bytes());
  Workspace ws(ws_ptr, ws_bytes);
  args.Vg = ws.take<float>(2 * (size_t)L.kp * L.ld);
  args.means = ws.take<float>(4 * (size_t)L.kp);
  args.part = ws.take<float>((size_t)G * L.kp * L.ld);
  args.spart = ws.take<float>((size_t)G * L.kp);
  args.bar = ws.take<unsigned>(1);
  args.flag = ws.take<int>(1);
  args.bulkv = ((reinterpret_cast<uintptr_t>(args.Vg) | reinterpret_cast<uintptr_t>(args.means)) &
                15) == 0;
  OTM_CHECK_CUDA(cudaMemsetAsync(args.bar, 0, sizeof(unsigned), st));
  return sym ? launch_grid<true>(args, G, st) : launch_grid<false>(args, G, st);
}

}  // namespace otm
