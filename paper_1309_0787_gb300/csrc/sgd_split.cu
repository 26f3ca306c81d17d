// Stochastic tensor gradient descent on the implicit whitened tensor
// (Section 3.2, Lemma 3 / Eq. (16)), FP32, "split" form: ONE launch of C
// thread-block clusters of CL CTAs that runs every step of the schedule.
//
// The k components are cut into C blocks of Nc and every minibatch into CL
// slices of Sb samples.  Cluster c owns block c; CTA s of the cluster owns
// slice s and, for the update, components i = c Nc + s, c Nc + s + CL, ...
// (one or two).  C is the largest count whose clusters can all be resident.
// Per step:
//   every CTA, for its slice and its cluster's block (in chunks of SC samples):
//     A_A = Y_A V_c, A_B = Y_B V_c          (samples x block components)
//     B   = c1 A_A o A_B - c2 (a_B o A_A + a_A o A_B)
//     part[i] = sum_t y_C,t B[t, i],  part[i][kp] = sum_t (A_A o A_B)[t, i]
//   cluster barrier;
//   the owner of component i sums the CL partial columns of i through
//   distributed shared memory and forms
//     G_data = part / b + ybar_C (c3 a_A a_B - c2 s / b),
//     G_gram = sum_j <v_j, v_i>^2 v_j      (from its copy of all of V),
//     v_i   <- v_i - beta_t (kappa G_gram - G_data),
//   and writes v_i and its means a_A, a_B to the iterate buffer of the next
//   step in global memory;
//   grid barrier (hierarchical: cluster barrier, one arrival per cluster on a
//   global counter, cluster barrier), then every CTA copies the new V into
//   shared memory (cp.async through L2) while the samples of the next chunk are
//   already in flight.
// Compared with the grid form (sgd_grid.cu), which reduces one k x k partial
// per CTA through L2 and needs two grid barriers per step, each CTA here
// produces only k x Nc partial sums, the reduction stays inside the cluster,
// and a step has one grid barrier.  The partial sums are added in a fixed
// order, so the result does not depend on timing.
//
// Every wait is bounded: a global-counter wait that times out sets a flag,
// the decision is shared by the whole cluster through distributed shared
// memory, and every CTA of the cluster leaves the kernel at the same point;
// the owners then write NaN into their columns of V.
#include <algorithm>

#include <cooperative_groups.h>

#include "grid_sync.cuh"
#include "otm_internal.cuh"
#include "tc_ptx.cuh"

namespace cg = cooperative_groups;

namespace otm {
namespace {

constexpr int ST = 256;          // threads per CTA
constexpr int SP_KMAX = 128;
constexpr int SP_CLMAX = 16;
constexpr int SP_SCMAX = 64;     // samples per chunk at most

struct SplitArgs {
  const float* YA;
  const float* YB;
  const float* YC;
  const int32_t* perm;
  const double* ybar3;
  float* V;        // k x k, component-major (row i = v_i); initial and final iterate
  float* V_snap;
  float* Vg;       // 2 x kp x ld: the iterate of the next step, by step parity
  float* Mg;       // 2 x 2 x kp: its means a_A, a_B, by step parity
  unsigned* bar;   // global arrival counter (zero on entry)
  int* flag;       // wait time-out
  int64_t n, b, spe, total_steps, snapshot_every;
  int k, Nc, Sb, SC;
  int vec;         // sample rows are 16-byte aligned (k % 4 == 0, aligned bases)
  double beta0;
  float c1, c2, c3, kappa;
};

struct SLayout {
  int kp, ld, nview, Nc4, kpp, SC;
  size_t off_v, off_y, off_b, off_p, off_part, off_yb, off_a, off_h, off_g, off_red, total;
};

// Shared memory (floats).  Rows of V and of the samples have stride ld, an odd
// number of float4s, so that float4 reads of consecutive rows fall in
// different bank groups.
__host__ __device__ inline SLayout s_layout(int k, bool sym, int Nc, int SC) {
  SLayout L;
  L.kp = (k + 3) & ~3;
  L.ld = ((L.kp / 4) & 1) ? L.kp : L.kp + 4;
  L.nview = sym ? 1 : 3;
  L.Nc4 = (Nc + 3) & ~3;
  L.kpp = L.kp + 4;  // a partial column: kp coordinates, then the sum of A_A o A_B
  L.SC = SC;
  size_t f = 0;
  L.off_v = f;    f += (size_t)L.kp * L.ld;              // all of V, component rows
  L.off_y = f;    f += 2 * (size_t)L.nview * SC * L.ld;  // sample chunks [buf][view][t]
  L.off_b = f;    f += (size_t)SC * L.Nc4;               // B [t][i]
  L.off_p = f;    f += (size_t)L.Nc4;                    // sum_t (A_A o A_B)[t][i] of a step
  L.off_part = f; f += (size_t)L.Nc4 * L.kpp;            // partial columns [i][r]
  L.off_yb = f;   f += 3 * (size_t)L.ld;                 // ybar_A, ybar_B, ybar_C
  L.off_a = f;    f += 2 * (size_t)L.Nc4;                // a_A, a_B of the block
  L.off_h = f;    f += (size_t)L.kp;                     // <v_j, v_i>^2 of the owned i
  L.off_g = f;    f += 2 * (size_t)L.kp;                 // two half sums of a Gram column
  L.off_red = f;  f += 2 * (ST / 32) + 4;
  L.total = f;
  return L;
}

__device__ __forceinline__ float dot4(const float4& a, const float4& b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}
__device__ __forceinline__ void cp16(float* dst, const float* src, bool in) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(in ? 16u : 0u)
               : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src, bool in) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(in ? 4u : 0u)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_two() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }
// One-dimensional bulk copy (TMA) of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) from global to this CTA's shared memory, completing on mbar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
      : "memory");
}
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Grid-wide barrier of the cooperative cluster launch.  Every CTA of a cluster
// arrives at a cluster barrier; thread 0 of cluster rank 0 then arrives on the
// global counter (release) and waits (acquire, bounded) for the other
// clusters; a second cluster barrier releases the cluster, whose CTAs read the
// outcome from rank 0's shared memory, so that all of them leave or continue
// together.  Returns false on a time-out (*flag set).
__device__ __forceinline__ bool cluster_grid_barrier(cg::cluster_group& cluster, unsigned* count,
                                                     int* flag, int* s_ok) {
  cluster.sync();
  if (cluster.block_rank() == 0 && threadIdx.x == 0) {
    const unsigned nclusters = gridDim.x / cluster.num_blocks();
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (nclusters - 1) : 1u;
    unsigned old, v;
    int ok = 1;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(count), "r"(add) : "memory");
    const long long t0 = clock64();
    do {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (((v ^ old) & 0x80000000u) != 0u) break;
      if (clock64() - t0 > GRID_WAIT_CYCLES) {
        atomicExch(flag, 1);
        ok = 0;
        break;
      }
    } while (true);
    *s_ok = ok;
  }
  cluster.sync();
  return *cluster.map_shared_rank(s_ok, 0) != 0;
}

template <bool SYM>
__global__ void __launch_bounds__(ST, 1) sgd_split_kernel(SplitArgs a) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_ok;
  __shared__ int s_rows[2][SP_SCMAX];  // corpus rows of a chunk's samples, by chunk parity
  // bulk-copy completion (16-byte aligned rows): the two chunk buffers, the
  // block's rows of V, the other rows of V
  __shared__ __align__(8) uint64_t s_mb[4];
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int sl = (int)cluster.block_rank();       // sample slice of this CTA
  const int cb = (int)(blockIdx.x / CL);          // component block of its cluster
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k, Nc = a.Nc, Sb = a.Sb;
  const SLayout L = s_layout(k, SYM, Nc, a.SC);
  const int kp = L.kp, ld = L.ld, kq = kp / 4, SC = L.SC, Nc4 = L.Nc4, kpp = L.kpp;
  float* Vs = sm + L.off_v;
  float* Ysb = sm + L.off_y;
  float* Bs = sm + L.off_b;
  float* psum = sm + L.off_p;   // sum over the step's samples of A_A o A_B (Nc4)
  float* part = sm + L.off_part;
  float* ybA = sm + L.off_yb;
  float* ybB = ybA + ld;
  float* ybC = ybB + ld;
  float* aA = sm + L.off_a;
  float* aB = aA + Nc4;
  float* hs = sm + L.off_h;
  float* gpart = sm + L.off_g;  // two half sums of the Gram column (2 x kp)
  float* red = sm + L.off_red;
  const int c0 = cb * Nc;                          // first component of the block
  const int nchunk = (Sb + SC - 1) / SC;

  for (int r = tid; r < ld; r += ST) {
    ybA[r] = r < k ? (float)a.ybar3[r] : 0.f;
    ybB[r] = r < k ? (float)a.ybar3[k + r] : 0.f;
    ybC[r] = r < k ? (float)a.ybar3[2 * k + r] : 0.f;
  }
  for (int idx = tid; idx < kp * ld; idx += ST) {
    const int i = idx / ld, r = idx % ld;
    Vs[idx] = (i < k && r < k) ? a.V[(int64_t)i * k + r] : 0.f;
  }
  // padding rows and columns of both iterate buffers stay zero (the owners
  // write rows < k, columns < kp)
  if (blockIdx.x == 0) {
    for (int bsel = 0; bsel < 2; ++bsel) {
      float* Vb = a.Vg + (size_t)bsel * kp * ld;
      for (int idx = tid; idx < kp * ld; idx += ST) {
        const int i = idx / ld, r = idx % ld;
        if (i >= k || r >= kp) Vb[idx] = 0.f;
      }
    }
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(&s_mb[i], 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  // a_A, a_B of the block's components from the initial V
  for (int i = warp; i < Nc4; i += ST / 32) {
    float x = 0.f, y = 0.f;
    const int gi = c0 + i;
    if (i < Nc && gi < k)
      for (int r = lane; r < kp; r += 32) {
        x = fmaf(Vs[gi * ld + r], ybA[r], x);
        y = fmaf(Vs[gi * ld + r], ybB[r], y);
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

  // Position of the next chunk to issue (step, chunk within the step, epoch,
  // minibatch within the epoch), advanced without divisions.  The row of this
  // thread's sample (t = tid < SC) in the chunk after it is loaded one issue
  // ahead, so that the permutation's latency is hidden.
  int64_t is_s = 0, is_e = 0, is_jb = 0;
  int is_q = 0;
  auto row_at = [&](int64_t s, int64_t e, int64_t jb, int q, int t) -> int {
    if (s >= a.total_steps) return -1;
    const int64_t pos0 = jb * a.b;
    const int64_t beff = min(a.b, a.n - pos0);
    const int pl = q * SC + t;
    const int64_t p = (int64_t)sl * Sb + pl;
    if (pl >= Sb || p >= beff) return -1;
    const int64_t row = a.perm ? (int64_t)a.perm[e * a.n + pos0 + p] : pos0 + p;
    return (row >= 0 && row < a.n) ? (int)row : -1;
  };
  auto advance = [&](int64_t& s, int64_t& e, int64_t& jb, int& q) {
    if (++q == nchunk) {
      q = 0;
      ++s;
      if (++jb == a.spe) {
        jb = 0;
        ++e;
      }
    }
  };
  int pf_row = tid < SC ? row_at(0, 0, 0, 0, tid) : -1;
  // the next chunk into buffer gg & 1 (gg counts issues).  Every call commits
  // one cp.async group (an empty one past the last step).  One warp per sample
  // row, its lanes over the row's 16-byte (or 4-byte) pieces.
  // completion parities of the four barriers, an unwaited chunk, a failed wait
  uint32_t mph = 0;
  int64_t out_g = -1;
  bool bad = false;
  auto mwait = [&](int i) {
    if (!tc::mbar_wait(&s_mb[i], (mph >> i) & 1u)) {
      if (tid == 0) atomicExch(a.flag, 2);
      bad = true;
    }
    mph ^= 1u << i;
  };
  auto issue_chunk = [&](int64_t gg) {
    if (is_s >= a.total_steps) {
      if (!a.vec) cp_commit();
      return;
    }
    int* rows = s_rows[gg & 1];
    {
      int64_t ns = is_s, ne = is_e, njb = is_jb;
      int nq = is_q;
      advance(ns, ne, njb, nq);
      if (tid < SC) {
        rows[tid] = pf_row;
        pf_row = row_at(ns, ne, njb, nq, tid);
      }
      is_s = ns;
      is_e = ne;
      is_jb = njb;
      is_q = nq;
    }
    float* Yb = Ysb + (size_t)(gg & 1) * L.nview * SC * ld;
    if (a.vec) {
      // one bulk copy per sample row and view; rows outside the data are zeroed
      const int valid = __syncthreads_count(tid < SC && rows[tid] >= 0);
      if (tid == 0) tc::mbar_expect_tx(&s_mb[gg & 1], (uint32_t)(valid * L.nview * k * 4));
      __syncthreads();
      if (tid < SC) {
        const int row = rows[tid];
        tc::fence_async_smem();  // earlier reads of the buffer precede the copy
        for (int v = 0; v < L.nview; ++v) {
          const float* Yg = v == 0 ? a.YA : (v == 1 ? a.YB : a.YC);
          float* dst = Yb + ((size_t)v * SC + tid) * ld;
          if (row >= 0)
            bulk_g2s(dst, Yg + (int64_t)row * k, (uint32_t)(k * 4), &s_mb[gg & 1]);
          else
            for (int r = 0; r < kp; r += 4)
              *reinterpret_cast<float4*>(dst + r) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      out_g = gg;
      return;
    }
    __syncthreads();
    const int per_row = kp;
    for (int vt = warp; vt < L.nview * SC; vt += ST / 32) {
      const int v = vt / SC, t = vt - v * SC;
      const int64_t row = rows[t];
      const float* Yg = v == 0 ? a.YA : (v == 1 ? a.YB : a.YC);
      float* dst = Yb + ((size_t)v * SC + t) * ld;
      for (int u = lane; u < per_row; u += 32) {
        const bool in = row >= 0 && u < k;
        cp4(dst + u, in ? Yg + row * k + u : Yg, in);
      }
    }
    cp_commit();
  };
  // rows of V outside this cluster's block, from the iterate buffer src (the
  // block's rows were copied before the step's first product)
  auto issue_vrest = [&](const float* src) {
    const int r1 = min(c0 + Nc, kp);
    if (a.vec) {
      if (tid == 0) {
        tc::mbar_expect_tx(&s_mb[3], (uint32_t)((kp - (r1 - c0)) * ld * 4));
        if (c0 > 0) bulk_g2s(Vs, src, (uint32_t)(c0 * ld * 4), &s_mb[3]);
        if (r1 < kp)
          bulk_g2s(Vs + (size_t)r1 * ld, src + (size_t)r1 * ld, (uint32_t)((kp - r1) * ld * 4),
                   &s_mb[3]);
      }
      return;
    }
    const int b0 = c0 * ld / 4, b1 = r1 * ld / 4;
    for (int idx = tid; idx < kp * ld / 4; idx += ST)
      if (idx < b0 || idx >= b1) cp16(Vs + 4 * idx, src + 4 * idx, true);
    cp_commit();
  };

  int64_t g = 0;  // next chunk to consume
  issue_chunk(0);
  const int nit1 = SC * (Nc4 / 4);  // items of the first product (SC samples x Nc4 / 4)
  const bool warp_seg = (SC % 32) == 0;
  // tiles of the second product and the lanes that share one (a power of two)
  const int nt2 = kq * (Nc4 / 4);
  int KS2 = 1;
  while (KS2 < 8 && nt2 * KS2 * 2 <= ST && KS2 * 2 <= SC) KS2 *= 2;
  for (int64_t s = 0; s < a.total_steps; ++s) {
    const int par = (int)(s & 1);
    const int64_t pos0 = (s % a.spe) * a.b;
    const int64_t beff = min(a.b, a.n - pos0);
    float g2[4][4];  // this lane's part of a tile of the partial columns
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int u = 0; u < 4; ++u) g2[c][u] = 0.f;
    for (int i = tid; i < Nc4; i += ST) psum[i] = 0.f;
    for (int q = 0; q < nchunk; ++q, ++g) {
      issue_chunk(g + 1);
      if (q == 0 && s > 0) issue_vrest(a.Vg + (size_t)par * kp * ld);
      if (a.vec) {  // chunk g and, at a step's first chunk, the block's rows of V
        mwait((int)(g & 1));
        if (out_g == g) out_g = -1;
        if (q == 0 && s > 0) mwait(2);
      } else if (q == 0 && s > 0) {
        cp_wait_two();   // the block's rows of V and chunk g have landed
      } else {
        cp_wait_one();
      }
      __syncthreads();
      const float* Yb = Ysb + (size_t)(g & 1) * L.nview * SC * ld;
      // first product: A_A, A_B for 4 block components x 1 sample per item
      for (int base = 0; base < nit1; base += ST) {
        const int item = base + tid;
        const bool act = item < nit1;
        const int t = item % SC, i0 = 4 * (act ? item / SC : 0);
        float pr[4] = {0.f, 0.f, 0.f, 0.f};
        if (act) {
          const float* ya = Yb + (size_t)t * ld;
          const float* yb = SYM ? ya : Yb + ((size_t)SC + t) * ld;
          float xa[4] = {0.f, 0.f, 0.f, 0.f}, xb[4] = {0.f, 0.f, 0.f, 0.f};
          const float* vr[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int gi = c0 + i0 + j;
            vr[j] = (i0 + j < Nc && gi < k) ? Vs + (size_t)gi * ld : Vs;
          }
#pragma unroll 4
          for (int r = 0; r < kp; r += 4) {
            const float4 yA = *reinterpret_cast<const float4*>(ya + r);
            const float4 yB = SYM ? yA : *reinterpret_cast<const float4*>(yb + r);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float4 v = *reinterpret_cast<const float4*>(vr[j] + r);
              xa[j] = dot4(v, yA, xa[j]);
              if (!SYM) xb[j] = dot4(v, yB, xb[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            const bool on = i < Nc && c0 + i < k;
            const float xA = on ? xa[j] : 0.f, xB = on ? (SYM ? xa[j] : xb[j]) : 0.f;
            pr[j] = xA * xB;
            Bs[t * Nc4 + i] = a.c1 * pr[j] - a.c2 * (aB[i] * xA + aA[i] * xB);
          }
        }
        // sum of A_A o A_B over the samples: the lanes of a warp hold 32 samples
        // of the same 4 components when SC is a multiple of 32
        if (warp_seg) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float v = pr[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && act) atomicAdd(&psum[i0 + j], v);
          }
        } else if (act) {
#pragma unroll
          for (int j = 0; j < 4; ++j) atomicAdd(&psum[i0 + j], pr[j]);
        }
      }
      __syncthreads();
      // second product: the partial columns sum_t y_C,t B[t, i], 4 coordinates x 4
      // block components per tile, the samples split over KS2 neighbouring lanes
      // (per-lane sums carried over the step's chunks)
      {
        const float* yc = SYM ? Yb : Yb + 2 * (size_t)SC * ld;
        const int tile = tid / KS2, ks = tid % KS2;
        if (tile < nt2) {
          const int r0 = 4 * (tile % kq), i0 = 4 * (tile / kq);
#pragma unroll 4
          for (int t = ks; t < SC; t += KS2) {
            const float4 y4 = *reinterpret_cast<const float4*>(yc + (size_t)t * ld + r0);
            const float4 b4 = *reinterpret_cast<const float4*>(Bs + t * Nc4 + i0);
            const float yv[4] = {y4.x, y4.y, y4.z, y4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int u = 0; u < 4; ++u) g2[c][u] = fmaf(bv[c], yv[u], g2[c][u]);
          }
        }
      }
      __syncthreads();  // the chunk buffer and B are reused by the next chunk
    }
    {  // the step's partial columns: sum the KS2 lanes of each tile, store
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          for (int o = KS2 / 2; o > 0; o >>= 1) g2[c][u] += __shfl_xor_sync(0xffffffffu, g2[c][u], o);
      const int tile = tid / KS2, ks = tid % KS2;
      if (tile < nt2 && ks == 0) {
        const int r0 = 4 * (tile % kq), i0 = 4 * (tile / kq);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          *reinterpret_cast<float4*>(part + (size_t)(i0 + c) * kpp + r0) =
              make_float4(g2[c][0], g2[c][1], g2[c][2], g2[c][3]);
      }
    }
    if (tid < Nc4) part[(size_t)tid * kpp + kp] = psum[tid];
    if (a.vec) {     // all of V has landed (the owners' Gram term reads it)
      if (s > 0) mwait(3);
    } else {
      cp_wait_all();
    }
    cluster.sync();

    // owners: sum the partial columns of each owned component, Gram term, update
    float* Vnext = a.Vg + (size_t)(par ^ 1) * kp * ld;
    float* Mnext = a.Mg + (size_t)(par ^ 1) * 2 * kp;
    const float beta = (float)a.beta0 / sqrtf((float)(s + 1));
    const float inv_b = 1.f / (float)beff;
    for (int lc = sl; lc < Nc && c0 + lc < k; lc += CL) {
      const int own = c0 + lc;
      // the CL partial columns (and sums) through distributed shared memory: all
      // loads issued before the Gram term, which needs only V
      const int r = tid;  // coordinate (r == kp: the sum of A_A o A_B)
      float dsum = 0.f;
      if (r <= kp) {
        float pv[SP_CLMAX];
#pragma unroll
        for (int c = 0; c < SP_CLMAX; ++c)
          if (c < CL) pv[c] = *cluster.map_shared_rank(part + (size_t)lc * kpp + r, c);
#pragma unroll
        for (int c = 0; c < SP_CLMAX; ++c)
          if (c < CL) dsum += pv[c];
      }
      {  // (v_j . v_own)^2: two threads per component j, alternate float4 of coordinates
        const int j = tid >> 1, h = tid & 1;
        float hv = 0.f;
        if (j < k) {
          const float* vi = Vs + (size_t)own * ld;
          const float* vj = Vs + (size_t)j * ld;
#pragma unroll 4
          for (int q = 4 * h; q < kp; q += 8)
            hv = dot4(*reinterpret_cast<const float4*>(vi + q), *reinterpret_cast<const float4*>(vj + q), hv);
        }
        hv += __shfl_xor_sync(0xffffffffu, hv, 1);
        if (h == 0 && j < kp) hs[j] = j < k ? hv * hv : 0.f;
      }
      __syncthreads();
      {  // Gram column: two halves of the components, one coordinate per thread
        const int rr = tid & 127, hh = tid >> 7;
        if (rr < kp) {
          const int kh = (k + 1) / 2, j0 = hh * kh, j1 = min(k, j0 + kh);
          float gg = 0.f;
#pragma unroll 4
          for (int j = j0; j < j1; ++j) gg = fmaf(hs[j], Vs[(size_t)j * ld + rr], gg);
          gpart[hh * kp + rr] = gg;
        }
      }
      if (r == kp) red[2 * (ST / 32)] = dsum;  // s_i
      __syncthreads();
      float x = 0.f, y = 0.f;
      if (r < kp) {
        const float gg = gpart[r] + gpart[kp + r];
        const float ai = aA[lc], bi = aB[lc], si = red[2 * (ST / 32)];
        const float gdata = dsum * inv_b + ybC[r] * (a.c3 * ai * bi - a.c2 * si * inv_b);
        const float v = r < k ? Vs[(size_t)own * ld + r] - beta * (a.kappa * gg - gdata) : 0.f;
        Vnext[(size_t)own * ld + r] = v;
        x = v * ybA[r];
        y = v * ybB[r];
        if (r < k) {
          if (a.snapshot_every > 0 && (s + 1) % a.snapshot_every == 0)
            a.V_snap[((s + 1) / a.snapshot_every - 1) * (int64_t)k * k + (int64_t)own * k + r] = v;
          if (s + 1 == a.total_steps) a.V[(int64_t)own * k + r] = v;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      if (lane == 0) {
        red[warp] = x;
        red[ST / 32 + warp] = y;
      }
      __syncthreads();
      if (tid == 0) {
        float tx = 0.f, ty = 0.f;
#pragma unroll
        for (int w = 0; w < ST / 32; ++w) {
          tx += red[w];
          ty += red[ST / 32 + w];
        }
        Mnext[own] = tx;
        Mnext[kp + own] = ty;
      }
      __syncthreads();  // hs, gpart and red are reused by the next owned component
    }
    __threadfence();
    fence_async_global();  // the new rows are read by bulk copies on other SMs
    if (!cluster_grid_barrier(cluster, a.bar, a.flag, &s_ok)) {
      // the whole cluster leaves here together; its peers read rank 0's flag
      // before the final cluster barrier; no bulk copy is left in flight
      for (int lc = sl; lc < Nc && c0 + lc < k; lc += CL)
        for (int r = tid; r < k; r += ST) a.V[(int64_t)(c0 + lc) * k + r] = __int_as_float(0x7fc00000);
      if (a.vec && out_g >= 0) mwait((int)(out_g & 1));
      cp_wait_all();
      cluster.sync();
      return;
    }
    if (s + 1 < a.total_steps) {
      // the block's rows of the new V (the products need only these; the other
      // rows are copied while the first product runs) and the block's means
      const int r1 = min(c0 + Nc, kp);
      if (a.vec) {
        if (tid == 0) {
          fence_async_global();
          tc::fence_async_smem();
          tc::mbar_expect_tx(&s_mb[2], (uint32_t)((r1 - c0) * ld * 4));
          bulk_g2s(Vs + (size_t)c0 * ld, Vnext + (size_t)c0 * ld, (uint32_t)((r1 - c0) * ld * 4),
                   &s_mb[2]);
        }
      } else {
        for (int idx = c0 * ld / 4 + tid; idx < r1 * ld / 4; idx += ST)
          cp16(Vs + 4 * idx, Vnext + 4 * idx, true);
        cp_commit();
      }
      for (int i = tid; i < Nc4; i += ST) {
        const int gi = c0 + i;
        aA[i] = (i < Nc && gi < k) ? __ldcg(Mnext + gi) : 0.f;
        aB[i] = (i < Nc && gi < k) ? __ldcg(Mnext + kp + gi) : 0.f;
      }
    }
  }
  cp_wait_all();
  if (bad)  // a bounded wait on a bulk copy gave up: the result is not to be used
    for (int lc = sl; lc < Nc && c0 + lc < k; lc += CL)
      for (int r = tid; r < k; r += ST) a.V[(int64_t)(c0 + lc) * k + r] = __int_as_float(0x7fc00000);
  cluster.sync();  // no CTA leaves while a peer may still read its shared memory
}

int split_sms() {
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (sms[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? v : 1;
  }
  return sms[dev];
}

int split_smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (v <= 0) v = 227 * 1024;
  }
  return v;
}

// Launch shape: cluster size CL, C clusters, components per block Nc (at most
// two per CTA), samples per CTA and step Sb, chunk SC.
struct SplitPlan {
  int CL, Nc, C, Sb, SC;
  size_t smem;
};

bool split_plan(int64_t k, int64_t b, bool sym, int CL, int C, SplitPlan* out) {
  if (k < 1 || k > SP_KMAX || b < 1 || C < 1) return false;
  const int Nc = (int)((k + C - 1) / C);
  if (Nc > 2 * CL || C * CL > split_sms()) return false;
  const int kq = (int)((k + 3) & ~3) / 4;
  if (Nc * kq > 2 * ST) return false;  // each thread accumulates at most two float4 outputs
  const int Sb = (int)((b + CL - 1) / CL);
  for (int SC : {64, 32, 16}) {
    // chunks of a multiple of 4 samples (the products' tiles); samples past the
    // slice are zero rows
    const int sc = std::min(SC, (std::max(Sb, 1) + 3) & ~3);
    const SLayout L = s_layout((int)k, sym, Nc, sc);
    const size_t bytes = L.total * sizeof(float);
    if (bytes + 1024 <= (size_t)split_smem_optin()) {
      *out = {CL, Nc, C, Sb, sc, bytes};
      return true;
    }
  }
  return false;
}

template <bool SYM>
cudaLaunchConfig_t split_cfg(const SplitPlan& P, cudaStream_t st, cudaLaunchAttribute* attr,
                             bool cooperative) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P.C * P.CL, 1, 1);
  cfg.blockDim = dim3(ST, 1, 1);
  cfg.dynamicSmemBytes = P.smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P.CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cooperative ? 2 : 1;
  return cfg;
}

// Sets the kernel's launch attributes for plan P (before every launch or
// occupancy query: plans of different shared-memory size share the kernel).
template <bool SYM>
bool split_attrs(const SplitPlan& P) {
  auto kern = sgd_split_kernel<SYM>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (P.CL > 8 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Clusters of plan P that can be resident at once.
template <bool SYM>
int split_resident(const SplitPlan& P) {
  if (!split_attrs<SYM>(P)) return 0;
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = split_cfg<SYM>(P, nullptr, attr, false);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)sgd_split_kernel<SYM>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// The plan for (k, b, views), cached per (device, k, b, sym): for 8- and
// 16-CTA clusters the largest C whose clusters are all resident at once; of
// those, the one with more CTAs (the smaller cluster on a tie).
bool split_choose(int64_t k, int64_t b, bool sym, SplitPlan* out) {
  struct Entry {
    int dev;
    int64_t k, b;
    bool sym, ok;
    SplitPlan P;
  };
  static Entry cache[64];
  static int ncache = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < ncache; ++i)
    if (cache[i].dev == dev && cache[i].k == k && cache[i].b == b && cache[i].sym == sym) {
      *out = cache[i].P;
      return cache[i].ok;
    }
  bool ok = false;
  SplitPlan best{};
  for (int CL : {8, 16}) {
    for (int C = (int)((k + CL - 1) / CL); C >= 1; --C) {
      if ((k + C - 1) / C > 2 * CL) break;  // more than two components per CTA
      SplitPlan Q;
      if (!split_plan(k, b, sym, CL, C, &Q)) continue;
      const int res = sym ? split_resident<true>(Q) : split_resident<false>(Q);
      if (res >= C) {
        if (!ok || C * CL > best.C * best.CL) best = Q;
        ok = true;
        break;
      }
    }
  }
  if (ncache < 64) cache[ncache++] = {dev, k, b, sym, ok, best};
  *out = best;
  return ok;
}

template <bool SYM>
otm_status launch_split(SplitArgs& args, const SplitPlan& P, cudaStream_t st) {
  auto kern = sgd_split_kernel<SYM>;
  if (!split_attrs<SYM>(P))
    return set_error(OTM_ECUDA, "sgd split form: cannot set the kernel's launch attributes");
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = split_cfg<SYM>(P, st, attr, true);
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args);
  if (e != cudaSuccess) {
    // the cooperative attribute is not accepted with clusters here: residency
    // was checked by split_choose, every wait is bounded
    cudaGetLastError();
    cfg = split_cfg<SYM>(P, st, attr, false);
    OTM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, args));
  }
  count_launch();
  return OTM_OK;
}

WorkspaceSize split_ws(int64_t k) {
  const int kp = (int)((k + 3) & ~3);
  const int ld = ((kp / 4) & 1) ? kp : kp + 4;
  WorkspaceSize w;
  w.add<float>(2 * (size_t)kp * ld).add<float>(4 * (size_t)kp).add<unsigned>(1).add<int>(1);
  return w;
}

}  // namespace

bool sgd_split_applicable(int64_t k, int64_t b, bool sym) {
  SplitPlan P;
  return split_choose(k, b, sym, &P);
}

size_t sgd_split_workspace(int64_t k) { return (k >= 1 && k <= SP_KMAX) ? split_ws(k).bytes() : 0; }

otm_status sgd_split_run(float* V, const float* YA, const float* YB, const float* YC, int64_t n,
                         int64_t k, const double* ybar3, const int32_t* perm, int64_t epochs,
                         int64_t b, double beta0, double theta, double alpha0,
                         int64_t snapshot_every, float* V_snap, void* ws_ptr, size_t ws_bytes,
                         cudaStream_t st) {
  const bool sym = (YA == YB) && (YB == YC);
  SplitPlan P;
  if (!split_choose(k, b, sym, &P))
    return set_error(OTM_EINVAL, "sgd split form: k=%lld, b=%lld does not fit", (long long)k,
                     (long long)b);
  if (!ws_ptr || ws_bytes < split_ws(k).bytes())
    return set_error(OTM_EINVAL, "sgd split form: workspace too small (need %zu bytes)",
                     split_ws(k).bytes());
  SplitArgs args;
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
  args.Nc = P.Nc;
  args.Sb = P.Sb;
  args.SC = P.SC;
  args.vec = (k % 4 == 0) && ((reinterpret_cast<uintptr_t>(YA) | reinterpret_cast<uintptr_t>(YB) |
                                reinterpret_cast<uintptr_t>(YC)) & 15) == 0;
  args.beta0 = beta0;
  args.c1 = (float)((alpha0 + 1.0) * (alpha0 + 2.0) / 2.0);
  args.c2 = (float)(alpha0 * (alpha0 + 1.0) / 2.0);
  args.c3 = (float)(alpha0 * alpha0);
  args.kappa = (float)(0.5 * (1.0 + theta));
  const int kp = (int)((k + 3) & ~3);
  const int ld = ((kp / 4) & 1) ? kp : kp + 4;
  Workspace ws(ws_ptr, ws_bytes);
  args.Vg = ws.take<float>(2 * (size_t)kp * ld);
  args.Mg = ws.take<float>(4 * (size_t)kp);
  args.bar = ws.take<unsigned>(1);
  args.flag = ws.take<int>(1);
  OTM_CHECK_CUDA(cudaMemsetAsync(args.bar, 0, sizeof(unsigned), st));
  return sym ? launch_split<true>(args, P, st) : launch_split<false>(args, P, st);
}

}  // namespace otm

using namespace otm;

extern "C" otm_status otm_sgd_split_shape(int64_t k, int64_t b, int sym, int* clusters,
                                          int* cluster_size) {
  clear_error();
  OTM_REQUIRE(clusters && cluster_size, "otm_sgd_split_shape: null pointer");
  SplitPlan P;
  if (!split_choose(k, b, sym != 0, &P)) {
    *clusters = 0;
    *cluster_size = 0;
    return OTM_OK;
  }
  *clusters = P.C;
  *cluster_size = P.CL;
  return OTM_OK;
}
