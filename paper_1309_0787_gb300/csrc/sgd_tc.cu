// Precision form of the fused STGD step (Section 3.2, Lemma 3) on the
// fifth-generation tensor cores.  Per step, for the components i a CTA owns:
//   A = Y_b V_own            (samples x owned components, K = coordinates)
//   B = c1 A_A o A_B - c2 (a_B o A_A + a_A o A_B)      (registers)
//   G_data = Y_C^T B / b + ybar_C (c3 a_A o a_B - c2 s / b)^T
//   H = V^T V_own,  G_gram = V (H o H)                  (Gram term)
//   V_own <- V_own - beta_t (kappa G_gram - G_data)
// Every product runs as tcgen05.mma (BF16: kind::f16; FP8 e4m3: kind::f8f6f4
// for the two data products) with FP32 accumulators in tensor memory; the
// master V and all sums stay FP32.
//
// Organisation (one thread-block cluster per decomposition): CTA q owns N
// consecutive components (N a multiple of 16) and streams every sample tile
// of the minibatch, so no partial product is ever reduced across CTAs.  After
// its update a CTA writes the BF16 image of its new columns into every CTA's
// V image (double-buffered, one cluster barrier per step).  Sample tiles
// arrive by cp.async into a ring of shared-memory stages, up to NS - 1 tiles
// ahead (across step boundaries); with three or more stages the first product
// of tile n + 1 is issued before the epilogue of tile n so that its latency
// is hidden.  One thread issues every MMA; completion is signalled by
// tcgen05.commit to mbarriers whose waits are bounded.
//
// k > 128 (256 padded coordinates, the WIDE instantiation): a CTA keeps only
// its own rows of the BF16 image on chip and publishes them after its update
// to one of two image buffers per cluster in global memory (step s reads
// buffer s & 1 and writes the other); once the step's last tile is consumed
// the whole image is copied into the sample stages for the Gram products, and
// the next step's tiles are issued only after those.  Its FP32 master rows
// live in tensor memory (lane = coordinate within a 128-row block, one column
// per owned component), and a_A, a_B are summed on the CUDA cores.
//
// Scaling: samples are stored quantised with one scale per sample (FP8; BF16
// stores scale 1); the owned rows of V are re-quantised every step with one
// scale per component (FP8); B with one scale per component per 128-sample
// tile (FP8).  Scales are applied to the FP32 accumulators in the epilogues.
// The Gram term always uses the BF16 image of V.
//
// FP8 keeps V as two e4m3 terms with the same per-component scale s_i:
// V_hi = e4m3(V / s_i) and V_lo = e4m3(V / s_i - V_hi), and issues the first
// product once for each into the same accumulator, so that Y (V_hi + V_lo) s_i
// carries about seven significant bits of V instead of four.  V's rounding is
// common to every sample of a minibatch and does not average out over the
// minibatch the way the per-sample rounding of the samples and of B does;
// it was the largest error of the single-term form.
//
// Precision 3 (FP8 with two-term operands) also keeps every sample as two
// e4m3 terms at its one scale (Y_hi, Y_lo: a second plane of the sample image,
// n rows after the first) and B as two terms at its per-tile scales (B_hi,
// B_lo: a second plane of the B image), and issues Y_hi V_hi + Y_hi V_lo +
// Y_lo V_hi for the first product and Y_hi^T B_hi + Y_lo^T B_hi + Y_hi^T B_lo
// for the second.  On long whitened samples the three-bit rounding of the
// samples and of B is what remains above the tolerance of the low-precision
// forms once V has two terms.
//
// Operand layouts in shared memory (no swizzle; 8-row x 16-byte core
// matrices; LBO = stride between cores along K, SBO = along M/N):
//   sample tile: core (tg, rg) = 8 samples x 16 B of coordinates at
//                (tg * CR + rg) * 128, CR = KP * esize / 16; read K-major by
//                the first product and MN-major (M = coordinates) by the second;
//   V image:     core (ng, rg) = 8 components x 16 B of coordinates (BF16,
//                128 rows): K-major for A = Y V_own and H = V^T V_own, MN-major
//                (M = coordinates, K = components) for G_gram = V (H o H);
//   B image:     core (tg, ng) = 8 samples x 16 B of owned components, MN-major;
//   H image:     core (jg, ng) = 8 components j x 16 B of owned components.
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

using namespace tc;

constexpr int TILE = 128;        // samples per tile (M of the first product)
// Coordinates and components are padded to KPc = 128 (k <= 128) or 256 (k <= 256);
// products whose M runs over coordinates or components are issued per 128-row block.
constexpr int TC_THREADS = 256;  // 8 warps: two per 32-lane TMEM quarter
constexpr uint32_t TMEM_COLS = 512;
constexpr int TC_KMAX = 256;
constexpr size_t VIMG_BYTES = (size_t)2 * 256 * 256 * 2;  // k > 128: two BF16 images per cluster
constexpr int NMBAR = 5;         // mbarriers: first product x2, second x2, Gram

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
  int64_t lo_off;     // bytes from a sample's first e4m3 term to its second (0: one term)
  int64_t n, b, spe, total_steps, snapshot_every;
  int k, ldq;
  int nc;             // components: k, or R k for R restarts of one problem stacked
                      // (their V matrices contiguous from V on, the Gram term per restart)
  double beta0;
  float c1, c2, c3, kappa;
};

__host__ __device__ constexpr int round16(int x) { return (x + 15) & ~15; }

// Components per CTA for k and a cluster of cl CTAs.
__host__ __device__ inline int own_cols(int k, int cl) {
  return round16((round16(k) + cl - 1) / cl);
}

struct TcLayout {
  int N, nv, NS, es, KPc, CR, CRb, CBn, CBh;
  bool dbl;
  bool vstr; // (KPc = 256) only the owned rows of the BF16 image of V stay in shared memory;
             // the whole image is streamed from global scratch into the sample stages for
             // the Gram term, and the FP32 master rows live in tensor memory
  size_t y_view, y_stage, off_v[2], off_vq, off_yb, off_b[2], off_h, off_f;
  size_t blo;  // bytes from a B image to its second e4m3 plane (two-term operands; else 0)
  size_t vm, ybA, ybB, ybC, aA, aB, vsc, bsc, amax, spw, red, ssc, nfloat;
  size_t total;
};

__host__ __device__ inline size_t al128(size_t x) { return (x + 127) & ~(size_t)127; }

// KPc: 128 or 256 padded coordinates; the second B image exists only with four
// stages (where the second product is waited for two tiles later)
__host__ __device__ inline TcLayout tc_layout(int N, bool sym, int es, int NS, bool dbl,
                                              int KPc, int planes = 1) {
  TcLayout L;
  const int KP = KPc;
  L.KPc = KPc;
  L.N = N;
  L.nv = sym ? 1 : 3;
  L.NS = NS;
  L.es = es;
  L.dbl = dbl;
  L.vstr = KPc > 128;
  L.CR = KP * es / 16;
  L.CRb = KP * 2 / 16;
  L.CBn = N * es / 16;
  L.CBh = N * 2 / 16;
  L.y_view = (size_t)TILE * KP * es;
  L.y_stage = (size_t)planes * L.nv * L.y_view;  // second terms of the views after the first
  // KPc rows (components) x KPc coordinates, or only the N owned rows when streamed
  const size_t v_bytes = (size_t)(L.vstr ? N : KP) * KP * 2;
  L.off_v[0] = NS * L.y_stage;
  L.off_v[1] = dbl && !L.vstr ? L.off_v[0] + v_bytes : L.off_v[0];
  L.off_vq = L.off_v[1] + v_bytes;
  // FP8: two e4m3 images of the owned rows, V_hi and the residual V_lo (same scales)
  const size_t vq_bytes = es == 1 ? (size_t)2 * N * KP : 0;
  const size_t b_bytes = (size_t)TILE * N * es;
  // the B images, the H image and the ybar image (16 rows: ybar_A, ybar_B, zeros;
  // rebuilt at the start of every step) share one region: they are live at
  // different times of a step.  With a single sample stage nothing is loaded
  // into it between the last tile of a step and the first of the next, which
  // is when the H and ybar images are live, so they use the stage instead.
  const size_t h_bytes = (size_t)KP * N * 2;
  const size_t yb_bytes = (size_t)16 * KP * 2;
  const bool in_stage = NS == 1 && !L.vstr && h_bytes <= L.y_stage && yb_bytes <= L.y_stage;
  L.off_b[0] = al128(L.off_vq + vq_bytes);
  L.off_b[1] = NS >= 4 ? L.off_b[0] + b_bytes : L.off_b[0];
  // two-term operands: the second planes of the B images after both first planes
  L.blo = planes > 1 ? L.off_b[1] + b_bytes - L.off_b[0] : 0;
  L.off_yb = in_stage ? 0 : L.off_b[0];
  L.off_h = in_stage ? 0 : L.off_b[0];  // the H image reuses both B images (free by then)
  size_t end = L.off_b[1] + b_bytes + L.blo;
  if (L.off_h + h_bytes > end) end = L.off_h + h_bytes;
  if (L.off_yb + yb_bytes > end) end = L.off_yb + yb_bytes;
  L.off_f = al128(end);
  size_t f = 0;
  L.vm = f;   f += L.vstr ? 0 : (size_t)N * KP;
  L.ybA = f;  f += KP;
  L.ybB = f;  f += KP;
  L.ybC = f;  f += KP;
  L.aA = f;   f += N;
  L.aB = f;   f += N;
  L.vsc = f;  f += N;
  L.bsc = f;  f += 2 * (size_t)N;
  L.amax = f; f += 2 * (size_t)N;
  L.spw = f;  f += 4 * (size_t)N;
  L.red = f;  f += 4 * (size_t)N;
  L.ssc = f;  f += (size_t)NS * 3 * TILE;
  L.nfloat = f;
  L.total = L.off_f + f * 4 + 64;
  return L;
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st8(uint32_t addr, const float (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}

__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_async_cluster() {
  asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
}

struct TcCtx {
  uint64_t* mbar;  // NMBAR barriers
  int* abort;
  uint32_t tmem;
  uint32_t ph;     // phase bits: 0-1 first product slots, 2-3 second, 4 Gram
};

// Samples of a tile handled by a thread: warp w takes samples 16 w .. 16 w + 15,
// lane l samples 16 w + (l & 7) and 16 w + 8 + (l & 7).
__device__ __forceinline__ int tile_sample(int j) {
  return 16 * (threadIdx.x >> 5) + 8 * j + (threadIdx.x & 7);
}

// Sample tile into ring stage `stage` by cp.async (zero fill outside the
// minibatch), with the samples' scales.  One warp instruction copies four
// consecutive 16-byte groups (64 contiguous bytes) of each of eight samples, so
// that it touches eight rows in global memory and writes four conflict-free
// 128-byte rows of the K-major image.  Only the coordinates the first product
// reads (k rounded up to its K step) are copied: the second product's rows for
// coordinates beyond k feed update rows that are never formed.  raw[j]: the
// permutation entry of sample tile_sample(j) (-1 outside the minibatch), loaded
// one issue earlier so that its latency is hidden.
template <bool FP8, bool SYM>
__device__ __forceinline__ void load_tile(const TcArgs& a, const TcLayout& L, uint8_t* smem,
                                          float* F, const int (&raw)[2], int stage) {
  constexpr int ES = FP8 ? 1 : 2;
  const int lane = threadIdx.x & 31;
  const int s8 = lane & 7, c4 = lane >> 3;
  constexpr int KSTEP = FP8 ? 32 : 16;
  const int kload = (a.k + KSTEP - 1) / KSTEP * KSTEP;  // coordinates read by the first product
  const int nq = L.CR / 4;  // 64-byte quarters of a sample row
  uint8_t* Ys = smem + (size_t)stage * L.y_stage;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int t = tile_sample(j);
    const int64_t row = (raw[j] >= 0 && raw[j] < a.n) ? raw[j] : -1;
    for (int v = 0; v < L.nv; ++v) {
      const uint8_t* Yg = v == 0 ? a.YA : (v == 1 ? a.YB : a.YC);
      uint8_t* dst = Ys + v * L.y_view + ((size_t)(t >> 3) * L.CR << 7) + (s8 << 4);
      for (int m = 0; m < nq; ++m) {
        const int rg = 4 * m + c4;
        const int c0 = rg * (16 / ES);
        if (c0 >= kload) break;
        const bool in = row >= 0 && c0 < a.ldq;
        const uint8_t* src = in ? Yg + ((size_t)row * a.ldq + c0) * ES : Yg;
        cp_async16(dst + ((size_t)rg << 7), src, in ? 16u : 0u);
        if (FP8 && a.lo_off)  // the second terms, into the views after the first
          cp_async16(dst + (size_t)L.nv * L.y_view + ((size_t)rg << 7), in ? src + a.lo_off : Yg,
                     in ? 16u : 0u);
      }
      if (c4 == 0) {
        const float* sv = v == 0 ? a.sA : (v == 1 ? a.sB : a.sC);
        float* sd = F + L.ssc + ((size_t)stage * 3 + v) * TILE + t;
        if (sv)
          cp_async4(sd, row >= 0 ? sv + row : sv, row >= 0 ? 4u : 0u);
        else
          *sd = row >= 0 ? 1.f : 0.f;
      }
    }
  }
  cp_async_commit();
}

// The owned rows own_lo .. own_lo + N - 1 of V (k x k, component-contiguous)
// into tensor memory from column base tcol on: lane = coordinate within a
// 128-row block, column mbk N + i = component own_lo + i (zeros outside k x k).
// Kept out of line: it runs once per chain and inlining it costs the step loop
// registers.
__device__ __noinline__ void tmem_load_rows(const float* __restrict__ V, int k, int own_lo, int N,
                                            uint32_t tcol) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qd = warp & 3, hf = warp >> 2;
  for (int c = 0; c < N / 16; ++c)
    for (int mbk = 0; mbk < 2; ++mbk) {
      const int r = mbk * 128 + 32 * qd + lane, c0 = 16 * c + 8 * hf;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int comp = own_lo + c0 + j;
        v[j] = (comp < k && r < k) ? V[(int64_t)comp * k + r] : 0.f;
      }
      tmem_st8(tcol + (uint32_t)(mbk * N + c0), v);
    }
  tmem_st_wait();
}

// One STGD chain (one decomposition), run by one cluster (WIDE: k > 128, 256
// padded coordinates, the code path of the streamed image); TMEM and the
// mbarriers are set up by the caller.  Ends with a cluster barrier so that the
// caller may reuse shared memory afterwards.
template <bool FP8, bool SYM, bool WIDE>
__device__ void tc_chain(const TcArgs& a, uint8_t* smem, TcCtx& cx, int NS, bool dbl,
                         uint8_t* vimg_cl) {
  constexpr int ES = FP8 ? 1 : 2;
  constexpr int KSTEP = FP8 ? 32 : 16;            // K of one MMA
  constexpr uint32_t FMT = FP8 ? 0u : 1u;         // E4M3 / BF16
  constexpr float QMAX = FP8 ? 448.f : 1.f;
  constexpr int NVD = SYM ? 1 : 2;                // views through the first product
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int qd = warp & 3, hf = warp >> 2;
  const int k = a.k;    // coordinates
  const int nc = a.nc;  // components
  constexpr int KPc = WIDE ? 256 : 128;  // padded coordinates / components
  constexpr int MB = KPc / 128;           // 128-row blocks
  if ((k > 128) != WIDE) {  // launched for the other width: report, leave V as it is
    if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
    return;
  }
  const int N = own_cols(nc, CL);
  const TcLayout L = tc_layout(N, SYM, ES, NS, dbl, KPc, FP8 && a.lo_off ? 2 : 1);
  const bool two_y = FP8 && a.lo_off != 0;
  const int own_lo = q * N;
  const bool active = own_lo < nc;
  const int nch = N / 16;
  float* F = reinterpret_cast<float*>(smem + L.off_f);
  float* Vm = F + L.vm;  // owned rows [N][KPc] (k <= 128)
  float* ybA = F + L.ybA;
  float* ybB = F + L.ybB;
  float* ybC = F + L.ybC;
  float* aA = F + L.aA;
  float* aB = F + L.aB;
  float* vsc = F + L.vsc;
  float* bsc = F + L.bsc;
  unsigned* amax = reinterpret_cast<unsigned*>(F + L.amax);
  float* spw = F + L.spw;
  float* red = F + L.red;
  uint8_t* Vimg0 = smem + L.off_v[0];
  uint8_t* Vimg1 = smem + L.off_v[1];
  // streamed image: Vown = the owned rows (local row index), Vfull = the whole image
  // copied into the sample stages for the Gram term, gimg = the cluster's two global
  // images (step s reads image s & 1 and writes image (s + 1) & 1)
  uint8_t* Vown = Vimg0;
  uint8_t* Vfull = smem;
  const size_t img_bytes = (size_t)KPc * KPc * 2;
  uint8_t* Vq = smem + L.off_vq;
  uint8_t* Bimg0 = smem + L.off_b[0];
  uint8_t* Bimg1 = smem + L.off_b[1];
  uint8_t* Himg = smem + L.off_h;
  uint64_t* mb = cx.mbar;
  int& s_abort = *cx.abort;
  const uint32_t tmem = cx.tmem;
  uint32_t ph = cx.ph;
  const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
  // TMEM columns: first product (2 slots x views), second product per coordinate block
  // (two slots each for FP8), the means (16), G_gram per coordinate block; H per
  // component block reuses the first product's columns
  const uint32_t colD2b = (uint32_t)(2 * NVD * N);
  const uint32_t d2w = (uint32_t)((FP8 ? 2 : 1) * N);
  const uint32_t colY = colD2b + (uint32_t)MB * d2w;
  const uint32_t colGGb = MB == 1 ? (uint32_t)N : colY + (WIDE ? 0u : 16u);
  // k > 128: the FP32 master rows, lane = coordinate within a 128-row block,
  // column colVm + mbk N + i = owned component i
  const uint32_t colVm = colGGb + (uint32_t)(MB * N);
  const int ks1 = (k + KSTEP - 1) / KSTEP;  // coordinate steps of the first product
  const int kg16 = (k + 15) / 16;           // 16-steps over coordinates (H = V^T V_own)
  const int kgc = (nc + 15) / 16;           // 16-steps over components (V (H o H))
  const size_t own_off = ((size_t)(own_lo >> 3) * L.CRb) << 7;

  // ---- initial state: owned FP32 rows, BF16 image of all rows, means ----
  if (WIDE) {
    tmem_load_rows(a.V, k, own_lo, N, tmem + lane_base + colVm);
  } else {
    for (int idx = tid; idx < N * KPc; idx += TC_THREADS) {
      const int i = idx / KPc, r = idx % KPc, c = own_lo + i;
      Vm[idx] = (c < nc && r < k) ? a.V[(int64_t)c * k + r] : 0.f;
    }
  }
  for (int idx = tid; idx < (WIDE ? N : KPc) * L.CRb; idx += TC_THREADS) {
    const int c = idx / L.CRb + (WIDE ? own_lo : 0), rg = idx % L.CRb;
    const int cl = WIDE ? c - own_lo : c;  // row of the shared-memory image
    float v[8];
#pragma unroll
    for (int z = 0; z < 8; ++z) {
      const int r = rg * 8 + z;
      v[z] = (c < nc && r < k) ? a.V[(int64_t)c * k + r] : 0.f;
    }
    uint4 w;
    w.x = pack_bf16(v[0], v[1]);
    w.y = pack_bf16(v[2], v[3]);
    w.z = pack_bf16(v[4], v[5]);
    w.w = pack_bf16(v[6], v[7]);
    const size_t off = (((size_t)(cl >> 3) * L.CRb + rg) << 7) + ((cl & 7) << 4);
    *reinterpret_cast<uint4*>(Vimg0 + off) = w;
    if (dbl) *reinterpret_cast<uint4*>(Vimg1 + off) = w;
  }
  // streamed image: the owned rows into global image dst (contiguous: N rows x KPc
  // coordinates from row own_lo on), visible to the cluster after its next barrier
  auto publish_own = [&](uint8_t* dst) {
    const uint4* src = reinterpret_cast<const uint4*>(Vown);
    uint4* d = reinterpret_cast<uint4*>(dst + (size_t)own_lo * KPc * 2);
    for (int idx = tid; idx < N * KPc / 8; idx += TC_THREADS) d[idx] = src[idx];
    __threadfence();
  };
  if (WIDE && active) {
    __syncthreads();
    publish_own(vimg_cl);
  }
  for (int r = tid; r < KPc; r += TC_THREADS) {
    ybA[r] = r < k ? (float)a.ybar3[r] : 0.f;
    ybB[r] = r < k ? (float)a.ybar3[k + r] : 0.f;
    ybC[r] = r < k ? (float)a.ybar3[2 * k + r] : 0.f;
  }
  for (int i = tid; i < 2 * N; i += TC_THREADS) amax[i] = 0u;
  uint8_t* Ybimg = smem + L.off_yb;
  // ybar image: rows 0, 1 = ybar_A, ybar_B (BF16, K-major like V), rows 2..15 zero
  auto build_ybar_image = [&]() {
    for (int idx = tid; idx < 16 * L.CRb; idx += TC_THREADS) {
      const int c = idx / L.CRb, rg = idx % L.CRb;
      float v[8];
#pragma unroll
      for (int z = 0; z < 8; ++z) {
        const int r = rg * 8 + z;
        v[z] = (r < k && c < 2) ? (c == 0 ? ybA[r] : ybB[r]) : 0.f;
      }
      uint4 w;
      w.x = pack_bf16(v[0], v[1]);
      w.y = pack_bf16(v[2], v[3]);
      w.z = pack_bf16(v[4], v[5]);
      w.w = pack_bf16(v[6], v[7]);
      *reinterpret_cast<uint4*>(Ybimg + (((size_t)(c >> 3) * L.CRb + rg) << 7) + ((c & 7) << 4)) =
          w;
    }
  };
  __syncthreads();
  if (FP8) {
    for (int i = warp; i < N; i += TC_THREADS / 32) {
      float m = 0.f;
      if (WIDE) {
        if (own_lo + i < nc)
          for (int r = lane; r < k; r += 32)
            m = fmaxf(m, fabsf(a.V[(int64_t)(own_lo + i) * k + r]));
      } else {
        for (int r = lane; r < KPc; r += 32) m = fmaxf(m, fabsf(Vm[i * KPc + r]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) vsc[i] = m > 0.f ? m / QMAX : 1.f;
    }
  } else {
    for (int i = tid; i < N; i += TC_THREADS) vsc[i] = 1.f;
  }
  __syncthreads();

  // FP8: owned rows of V quantised with one scale per component (K-major)
  auto build_vq = [&]() {
    if (WIDE) {  // from tensor memory: thread = coordinate r, one byte per component
      for (int c = 0; c < nch; ++c)
        for (int mbk = 0; mbk < MB; ++mbk) {
          const int r = mbk * 128 + 32 * qd + lane, c0 = 16 * c + 8 * hf;
          float x[8];
          tmem_ld8(tmem + lane_base + colVm + (uint32_t)(mbk * N + c0), x);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int i = c0 + j;
            const float z = x[j] * (1.f / vsc[i]);
            const __nv_fp8_e4m3 qh(z);
            const __nv_fp8_e4m3 ql(z - float(qh));
            const size_t off =
                (((size_t)(i >> 3) * L.CR + (r >> 4)) << 7) + ((i & 7) << 4) + (r & 15);
            Vq[off] = *reinterpret_cast<const uint8_t*>(&qh);
            Vq[(size_t)N * KPc + off] = *reinterpret_cast<const uint8_t*>(&ql);
          }
        }
      return;
    }
    for (int idx = tid; idx < N * L.CR; idx += TC_THREADS) {
      const int i = idx / L.CR, rg = idx % L.CR;
      const float inv = 1.f / vsc[i];
      const float* vr = Vm + i * KPc + rg * 16;
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int z = 0; z < 4; ++z)
        split_e4m3(vr[4 * z] * inv, vr[4 * z + 1] * inv, vr[4 * z + 2] * inv,
                   vr[4 * z + 3] * inv, hi[z], lo[z]);
      const size_t off = (((size_t)(i >> 3) * L.CR + rg) << 7) + ((i & 7) << 4);
      *reinterpret_cast<uint4*>(Vq + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(Vq + (size_t)N * KPc + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  };
  if (FP8) build_vq();
  fence_async_smem();
  cluster.sync();

  // the owned FP32 rows into dst (k x k, component-contiguous)
  auto write_rows = [&](float* dst) {
    if (WIDE) {
      for (int c = 0; c < nch; ++c)
        for (int mbk = 0; mbk < MB; ++mbk) {
          const int r = mbk * 128 + 32 * qd + lane, c0 = 16 * c + 8 * hf;
          float x[8];
          tmem_ld8(tmem + lane_base + colVm + (uint32_t)(mbk * N + c0), x);
          if (r < k) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (own_lo + c0 + j < nc) dst[(int64_t)(own_lo + c0 + j) * k + r] = x[j];
          }
        }
      return;
    }
    for (int idx = tid; idx < N * k; idx += TC_THREADS) {
      const int i = idx / k, r = idx % k;
      if (own_lo + i < nc) dst[(int64_t)(own_lo + i) * k + r] = Vm[i * KPc + r];
    }
  };

  // bounded mbarrier wait by every thread (phases tracked identically)
  auto wait_mb = [&](int idx) {
    if (!mbar_wait_or_abort(&mb[idx], (ph >> idx) & 1u, &s_abort) && lane == 0) {
      s_abort = 1;
      atomicExch(a.err, 1);
    }
    ph ^= 1u << idx;
    tc_after();
  };

  // ---- tile loader: the global sequence of (step, tile) ----
  // W = how many tiles back the second product is waited for before its sample
  // stage is refilled (two with four stages, so that wait is never exposed)
  const int W = NS >= 4 ? 2 : 1;
  const bool early = NS - W >= 2;  // the next tile is resident one tile ahead
  int64_t ld_s = 0, ld_e = 0, ld_jb = 0;  // step, epoch, minibatch of the next tile to issue
  int ld_n = 0, ld_nt = 0, ld_stage = 0;
  int64_t issued = 0;
  auto tiles_of = [&](int64_t jb) {
    return (int)((min(a.b, a.n - jb * a.b) + TILE - 1) / TILE);
  };
  auto row_raw = [&](int64_t e, int64_t jb, int n_tile, int t) {
    const int64_t pos0 = jb * a.b;
    const int64_t p = (int64_t)n_tile * TILE + t;
    if (p >= min(a.b, a.n - pos0)) return -1;
    return a.perm ? a.perm[e * a.n + pos0 + p] : (int)(pos0 + p);
  };
  ld_nt = a.total_steps > 0 ? tiles_of(0) : 0;
  int next_raw[2];
#pragma unroll
  for (int j = 0; j < 2; ++j)
    next_raw[j] = a.total_steps > 0 ? row_raw(0, 0, 0, tile_sample(j)) : -1;
  auto issue_one = [&]() {
    if (ld_s >= a.total_steps) return;
    load_tile<FP8, SYM>(a, L, smem, F, next_raw, ld_stage);
    ++issued;
    if (++ld_stage == NS) ld_stage = 0;
    if (++ld_n >= ld_nt) {
      ld_n = 0;
      ++ld_s;
      if (++ld_jb == a.spe) {
        ld_jb = 0;
        ++ld_e;
      }
      ld_nt = tiles_of(ld_jb);
    }
    if (ld_s < a.total_steps) {
#pragma unroll
      for (int j = 0; j < 2; ++j) next_raw[j] = row_raw(ld_e, ld_jb, ld_n, tile_sample(j));
    }
  };
  auto wait_tile = [&](int64_t g) {
    const int64_t pend = issued - 1 - g;
    cp_async_wait(pend < 0 ? 0 : (pend > 3 ? 3 : (int)pend));
    fence_async_smem();
    tc_before();
    __syncthreads();
    tc_after();
  };
  // streamed image: the stages hold the image during the Gram term, so no tile of
  // a later step is issued before that step's Gram products are done
  if (active)
    for (int i = 0; i < NS - W && (!WIDE || ld_s == 0); ++i) issue_one();

  int cur = 0;
  int64_t gbase = 0;
  int gstage = 0;  // ring stage of the step's first tile
  int64_t jb = 0;  // minibatch index within the epoch
  for (int64_t s = 0; s < a.total_steps; ++s) {
    const int64_t pos0 = jb * a.b;
    const int64_t beff = min(a.b, a.n - pos0);
    const int nt = (int)((beff + TILE - 1) / TILE);
    const float beta = (float)a.beta0 / sqrtf((float)(s + 1));
    const float inv_b = 1.f / (float)beff;
    uint8_t* Vc = cur ? Vimg1 : Vimg0;
    uint8_t* Vn = dbl ? (cur ? Vimg0 : Vimg1) : Vc;

    if (active) {
      float spart[8][8];
#pragma unroll
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int j = 0; j < 8; ++j) spart[c][j] = 0.f;
      float gacc[FP8 ? 2 : 1][FP8 ? 4 : 1][8];
#pragma unroll
      for (int u = 0; u < (FP8 ? 2 : 1); ++u)
#pragma unroll
        for (int c = 0; c < (FP8 ? 4 : 1); ++c)
#pragma unroll
          for (int j = 0; j < 8; ++j) gacc[u][c][j] = 0.f;

      // descriptors (the start address is the low 14-bit field, in 16-byte units)
      const uint64_t dV_own = sdesc(WIDE ? Vown : Vc + own_off, 128, (uint32_t)L.CRb * 128);
      const uint64_t dVq = sdesc(Vq, 128, (uint32_t)L.CR * 128);
      const uint64_t dVq_lo = sdesc(Vq + (size_t)N * KPc, 128, (uint32_t)L.CR * 128);
      const uint32_t id1 = make_idesc(FMT, 0, 0, TILE, (uint32_t)N);
      const uint32_t id2 = make_idesc(FMT, 1, 1, 128, (uint32_t)N);

      // first product A = Y V_own of the tile in stage st (thread 0)
      auto gemm1 = [&](int slot, int st) {
        const uint8_t* Ys = smem + (size_t)st * L.y_stage;
        for (int v = 0; v < NVD; ++v) {
          const uint64_t dY = sdesc(Ys + v * L.y_view, 128, (uint32_t)L.CR * 128);
          const uint64_t dB = FP8 ? dVq : dV_own;
          for (int ks = 0; ks < ks1; ++ks) {
            mma<FP8>(tmem + (uint32_t)((slot * NVD + v) * N), dY + (uint64_t)(16 * ks),
                     dB + (uint64_t)(16 * ks), id1, ks > 0 ? 1u : 0u);
            if (FP8)  // the residual term of V into the same accumulator
              mma<FP8>(tmem + (uint32_t)((slot * NVD + v) * N), dY + (uint64_t)(16 * ks),
                       dVq_lo + (uint64_t)(16 * ks), id1, 1u);
            if (two_y)  // the samples' second term times V_hi
              mma<FP8>(tmem + (uint32_t)((slot * NVD + v) * N),
                       sdesc(Ys + (L.nv + v) * L.y_view, 128, (uint32_t)L.CR * 128) +
                           (uint64_t)(16 * ks),
                       dB + (uint64_t)(16 * ks), id1, 1u);
          }
        }
        mma_commit(&mb[slot]);
      };
      // second product G += Y_C^T B of tile n in stage st (thread 0)
      auto gemm2 = [&](int n, int st) {
        const int slot = n & 1;
        const uint8_t* YC = smem + (size_t)st * L.y_stage + (SYM ? 0 : 2 * L.y_view);
        const uint64_t dB = sdesc(slot ? Bimg1 : Bimg0, (uint32_t)L.CBn * 128, 128);
        const uint64_t dBl = sdesc((slot ? Bimg1 : Bimg0) + L.blo, (uint32_t)L.CBn * 128, 128);
        const uint64_t stepA = (uint64_t)((KSTEP / 8) * L.CR * 8);   // (KSTEP/8) core groups
        const uint64_t stepB = (uint64_t)((KSTEP / 8) * L.CBn * 8);  // in 16-byte units
        for (int mbk = 0; mbk < MB; ++mbk) {  // 128 coordinates = 1024 ES bytes along M
          const uint64_t dA = sdesc(YC + (size_t)mbk * 1024 * ES, (uint32_t)L.CR * 128, 128);
          const uint32_t col = colD2b + (uint32_t)mbk * d2w + (FP8 ? (uint32_t)(slot * N) : 0u);
          for (int ks = 0; ks < TILE / KSTEP; ++ks) {
            mma<FP8>(tmem + col, dA + stepA * ks, dB + stepB * ks, id2,
                     (FP8 ? ks > 0 : (n > 0 || ks > 0)) ? 1u : 0u);
            if (two_y) {  // Y_lo^T B_hi and Y_hi^T B_lo into the same accumulator
              mma<FP8>(tmem + col,
                       sdesc(YC + (size_t)L.nv * L.y_view + (size_t)mbk * 1024 * ES,
                             (uint32_t)L.CR * 128, 128) + stepA * ks,
                       dB + stepB * ks, id2, 1u);
              mma<FP8>(tmem + col, dA + stepA * ks, dBl + stepB * ks, id2, 1u);
            }
          }
        }
        mma_commit(&mb[2 + slot]);
      };
      // FP8: per-tile second product, scaled by the tile's B scales
      auto epi2 = [&](int n) {
        const int slot = n & 1;
#pragma unroll
        for (int u = 0; u < (FP8 ? 2 : 1); ++u) {
          if (u < MB) {
#pragma unroll
            for (int c = 0; c < (FP8 ? 4 : 1); ++c) {
              if (c < nch) {
                const int c0 = 16 * c + 8 * hf;
                float x[8];
                tmem_ld8(tmem + lane_base + colD2b + (uint32_t)u * d2w + (uint32_t)(slot * N + c0),
                         x);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                  gacc[u][c][j] = fmaf(x[j], bsc[slot * N + c0 + j], gacc[u][c][j]);
              }
            }
          }
        }
      };

      // a_A = V^T ybar_A, a_B = V^T ybar_B for the 128 components of the block holding
      // the owned ones (one MMA chain, N = 16)
      const int mbo = own_lo >> 7;
      if (!WIDE) {
        build_ybar_image();
        fence_async_smem();
      }
      tc_before();
      __syncthreads();
      tc_after();
      if (!WIDE && tid == 0 && !s_abort) {
        const uint64_t dA = sdesc(Vc + (((size_t)mbo * 16 * L.CRb) << 7), 128, (uint32_t)L.CRb * 128);
        const uint64_t dB = sdesc(Ybimg, 128, (uint32_t)L.CRb * 128);
        const uint32_t id = make_idesc(1, 0, 0, 128, 16);
        for (int ks = 0; ks < kg16; ++ks)
          mma<false>(tmem + colY, dA + (uint64_t)(16 * ks), dB + (uint64_t)(16 * ks), id,
                     ks > 0 ? 1u : 0u);
        mma_commit(&mb[4]);
      }
      int st = gstage;  // stage of tile g
      if (early) {
        wait_tile(gbase);
        if (tid == 0 && !s_abort) gemm1(0, st);
      }
      if (WIDE) {
        // from the owned rows' BF16 image: warp w sums components 8w..8w+7, lanes
        // 8j..8j+7 take coordinate groups j, j + 4, ... (one 128-byte row per group)
        for (int i8 = warp; i8 < N / 8; i8 += TC_THREADS / 32) {
          float sa = 0.f, sb = 0.f;
          for (int rg = lane >> 3; rg < L.CRb; rg += 4) {
            const uint4 w = *reinterpret_cast<const uint4*>(
                Vown + (((size_t)i8 * L.CRb + rg) << 7) + ((lane & 7) << 4));
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
            for (int z = 0; z < 4; ++z) {
              const float2 v = __bfloat1622float2(h[z]);
              const int r = rg * 8 + 2 * z;
              sa = fmaf(v.x, ybA[r], fmaf(v.y, ybA[r + 1], sa));
              if (!SYM) sb = fmaf(v.x, ybB[r], fmaf(v.y, ybB[r + 1], sb));
            }
          }
          sa += __shfl_xor_sync(0xffffffffu, sa, 8);
          sa += __shfl_xor_sync(0xffffffffu, sa, 16);
          sb += __shfl_xor_sync(0xffffffffu, sb, 8);
          sb += __shfl_xor_sync(0xffffffffu, sb, 16);
          if (lane < 8) {
            aA[i8 * 8 + lane] = sa;
            aB[i8 * 8 + lane] = SYM ? sa : sb;
          }
        }
      } else {
        wait_mb(4);
        if (hf == 0) {  // lanes = components: keep the owned ones
          float x[8];
          tmem_ld8(tmem + lane_base + colY, x);
          const int j = mbo * 128 + 32 * qd + lane;
          if (j >= own_lo && j < own_lo + N) {
            aA[j - own_lo] = x[0];
            aB[j - own_lo] = SYM ? x[0] : x[1];
          }
        }
      }
      tc_before();
      __syncthreads();
      tc_after();

      for (int n = 0; n < nt; ++n) {
        const int64_t g = gbase + n;
        const int slot = n & 1;
        const int st_next = st + 1 == NS ? 0 : st + 1;
        if (early && n + 1 < nt) {
          wait_tile(g + 1);
          if (tid == 0 && !s_abort) gemm1((n + 1) & 1, st_next);
        }
        if (n >= W) {
          wait_mb(2 + ((n - W) & 1));
          if (FP8) epi2(n - W);
        }
        while (issued <= g + NS - W && ld_s < a.total_steps && (!WIDE || ld_s == s))
          issue_one();
        if (!early) {
          wait_tile(g);
          if (tid == 0 && !s_abort) gemm1(slot, st);
        }
        wait_mb(slot);

        // -- epilogue 1: B = c1 A_A o A_B - c2 (a_B o A_A + a_A o A_B) --
        {
          const int t = 32 * qd + lane;
          const float* ss = F + L.ssc + (size_t)st * 3 * TILE;
          const float sa = ss[t], sb = SYM ? sa : ss[TILE + t], sc = SYM ? sa : ss[2 * TILE + t];
          uint8_t* Bi = slot ? Bimg1 : Bimg0;
          if (FP8) {
            // pass 1: B column maxima over the tile (and the sums s_i)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              if (c < nch) {
                const int c0 = 16 * c + 8 * hf;
                float xa[8], xb[8];
                tmem_ld8(tmem + lane_base + (uint32_t)(slot * NVD * N + c0), xa);
                if (!SYM) tmem_ld8(tmem + lane_base + (uint32_t)((slot * NVD + 1) * N + c0), xb);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const int i = c0 + j;
                  const float va = xa[j] * sa * vsc[i];
                  const float vb = SYM ? va : xb[j] * sb * vsc[i];
                  const float pr = va * vb;
                  spart[c][j] += pr;
                  float m = fabsf(sc * (a.c1 * pr - a.c2 * (aB[i] * va + aA[i] * vb)));
#pragma unroll
                  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                  if (lane == 0) atomicMax(&amax[slot * N + i], __float_as_uint(m));
                }
              }
            }
            tc_before();
            __syncthreads();
            tc_after();
            if (tid < N) {
              const unsigned m = amax[slot * N + tid];
              bsc[slot * N + tid] = m ? __uint_as_float(m) / QMAX : 1.f;
              amax[slot * N + tid] = 0u;
            }
            __syncthreads();
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (c < nch) {
              const int c0 = 16 * c + 8 * hf;
              float xa[8], xb[8];
              tmem_ld8(tmem + lane_base + (uint32_t)(slot * NVD * N + c0), xa);
              if (!SYM) tmem_ld8(tmem + lane_base + (uint32_t)((slot * NVD + 1) * N + c0), xb);
              float w[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int i = c0 + j;
                const float va = xa[j] * sa * vsc[i];
                const float vb = SYM ? va : xb[j] * sb * vsc[i];
                const float pr = va * vb;
                if (!FP8) spart[c][j] += pr;
                const float b = sc * (a.c1 * pr - a.c2 * (aB[i] * va + aA[i] * vb));
                w[j] = FP8 ? b / bsc[slot * N + i] : b;
              }
              if constexpr (FP8) {
                const size_t off = (((size_t)(t >> 3) * L.CBn + c) << 7) + ((t & 7) << 4) + 8 * hf;
                uint2 u;
                if (two_y) {  // B_hi and the residual B_lo, one scale
                  uint2 ul;
                  split_e4m3(w[0], w[1], w[2], w[3], u.x, ul.x);
                  split_e4m3(w[4], w[5], w[6], w[7], u.y, ul.y);
                  *reinterpret_cast<uint2*>(Bi + L.blo + off) = ul;
                } else {
                  u.x = pack_e4m3(w[0], w[1], w[2], w[3]);
                  u.y = pack_e4m3(w[4], w[5], w[6], w[7]);
                }
                *reinterpret_cast<uint2*>(Bi + off) = u;
              } else {
                uint4 u;
                u.x = pack_bf16(w[0], w[1]);
                u.y = pack_bf16(w[2], w[3]);
                u.z = pack_bf16(w[4], w[5]);
                u.w = pack_bf16(w[6], w[7]);
                *reinterpret_cast<uint4*>(Bi + ((((size_t)(t >> 3) * L.CBn + (c0 >> 3)) << 7) +
                                                ((t & 7) << 4))) = u;
              }
            }
          }
        }
        fence_async_smem();
        tc_before();
        __syncthreads();
        tc_after();
        if (tid == 0 && !s_abort) gemm2(n, st);
        st = st_next;
      }
      for (int n = nt - W < 0 ? 0 : nt - W; n < nt; ++n) {
        wait_mb(2 + (n & 1));
        if (FP8) epi2(n);
      }
      if (WIDE) {
        // the stages are free: copy this step's image (rows >= k read as zeros)
        const uint8_t* src = vimg_cl + (size_t)(s & 1) * img_bytes;
        for (int c16 = tid; c16 < (int)(img_bytes >> 4); c16 += TC_THREADS) {
          const size_t off = (size_t)c16 << 4;
          const int comp = (int)((off >> 7) / L.CRb) * 8 + (int)((off >> 4) & 7);
          const bool in = comp < nc;
          cp_async16(Vfull + off, in ? src + off : src, in ? 16u : 0u);
        }
        cp_async_commit();
      }

      // s_i = sum over the minibatch of A_A o A_B (per owned component)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c < nch) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float v = spart[c][j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) spw[qd * N + 16 * c + 8 * hf + j] = v;
          }
        }
      }
      // -- Gram term: H = V^T V_own, then G_gram = V (H o H) --
      uint8_t* Vg = WIDE ? Vfull : Vc;  // the whole image
      if (WIDE) {
        cp_async_wait(0);
        fence_async_smem();
      }
      tc_before();
      __syncthreads();
      tc_after();
      if (tid == 0 && !s_abort) {
        const uint32_t id = make_idesc(1, 0, 0, 128, (uint32_t)N);
        for (int mbk = 0; mbk < MB; ++mbk) {  // components j in blocks of 128 rows
          const uint64_t dA =
              sdesc(Vg + (((size_t)mbk * 16 * L.CRb) << 7), 128, (uint32_t)L.CRb * 128);
          for (int ks = 0; ks < kg16; ++ks)
            mma<false>(tmem + (uint32_t)(mbk * N), dA + (uint64_t)(16 * ks),
                       dV_own + (uint64_t)(16 * ks), id, ks > 0 ? 1u : 0u);
        }
        mma_commit(&mb[4]);
      }
      wait_mb(4);
      for (int mbk = 0; mbk < MB; ++mbk) {
        const int j = mbk * 128 + 32 * qd + lane;
        const int rj = j / k;  // restart of component j (stacked restarts)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c < nch) {
            const int c0 = 16 * c + 8 * hf;
            float x[8];
            tmem_ld8(tmem + lane_base + (uint32_t)(mbk * N + c0), x);
            if (nc > k) {  // the Gram term couples only components of the same restart
#pragma unroll
              for (int jj = 0; jj < 8; ++jj)
                if ((own_lo + c0 + jj) / k != rj) x[jj] = 0.f;
            }
            uint4 u;
            u.x = pack_bf16(x[0] * x[0], x[1] * x[1]);
            u.y = pack_bf16(x[2] * x[2], x[3] * x[3]);
            u.z = pack_bf16(x[4] * x[4], x[5] * x[5]);
            u.w = pack_bf16(x[6] * x[6], x[7] * x[7]);
            *reinterpret_cast<uint4*>(Himg + ((((size_t)(j >> 3) * L.CBh + (c0 >> 3)) << 7) +
                                              ((j & 7) << 4))) = u;
          }
        }
      }
      fence_async_smem();
      tc_before();
      __syncthreads();
      tc_after();
      if (tid == 0 && !s_abort) {
        const uint64_t dB = sdesc(Himg, (uint32_t)L.CBh * 128, 128);
        const uint32_t id = make_idesc(1, 1, 1, 128, (uint32_t)N);
        for (int mbk = 0; mbk < MB; ++mbk) {  // coordinates in blocks of 128 (2048 bytes)
          const uint64_t dA = sdesc(Vg + (size_t)mbk * 2048, (uint32_t)L.CRb * 128, 128);
          for (int ks = 0; ks < kgc; ++ks)
            mma<false>(tmem + colGGb + (uint32_t)(mbk * N), dA + (uint64_t)(2 * L.CRb * 8 * ks),
                       dB + (uint64_t)(2 * L.CBh * 8 * ks), id, ks > 0 ? 1u : 0u);
        }
        mma_commit(&mb[4]);
      }
      wait_mb(4);
      // streamed image: the stages are free again; the next step's first tiles load
      // during the update
      if (WIDE)
        while (issued < gbase + nt + NS - W && ld_s == s + 1 && ld_s < a.total_steps)
          issue_one();

      // -- update of the owned columns (thread = coordinate r, per 128-row block) --
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c < nch) {
          const int c0 = 16 * c + 8 * hf;
          float mcol[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) mcol[j] = 0.f;
          for (int mbk = 0; mbk < MB; ++mbk) {
            const int r = mbk * 128 + 32 * qd + lane;
            float gg[8], gd[8], vm8[8];
            tmem_ld8(tmem + lane_base + colGGb + (uint32_t)(mbk * N + c0), gg);
            if (WIDE) tmem_ld8(tmem + lane_base + colVm + (uint32_t)(mbk * N + c0), vm8);
            if constexpr (FP8) {
#pragma unroll
              for (int j = 0; j < 8; ++j) gd[j] = gacc[mbk & 1][c < 4 ? c : 0][j];
            } else {
              tmem_ld8(tmem + lane_base + colD2b + (uint32_t)mbk * d2w + (uint32_t)c0, gd);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int i = c0 + j, comp = own_lo + i;
              if (comp < nc) {
                float vnew = 0.f;
                if (r < k) {
                  const float s_i = spw[i] + spw[N + i] + spw[2 * N + i] + spw[3 * N + i];
                  const float gdata =
                      gd[j] * inv_b + ybC[r] * (a.c3 * aA[i] * aB[i] - a.c2 * s_i * inv_b);
                  vnew = (WIDE ? vm8[j] : Vm[i * KPc + r]) - beta * (a.kappa * gg[j] - gdata);
                  if (WIDE)
                    vm8[j] = vnew;
                  else
                    Vm[i * KPc + r] = vnew;
                }
                const int ci = WIDE ? i : comp;  // row of the shared-memory image
                *reinterpret_cast<__nv_bfloat16*>(
                    (WIDE ? Vown : Vn) + ((((size_t)(ci >> 3) * L.CRb + (r >> 3)) << 7) +
                                            ((ci & 7) << 4) + ((r & 7) << 1))) =
                    __float2bfloat16_rn(vnew);
                mcol[j] = fmaxf(mcol[j], fabsf(vnew));
              }
            }
            if (WIDE) tmem_st8(tmem + lane_base + colVm + (uint32_t)(mbk * N + c0), vm8);
          }
          if (FP8) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float m = mcol[j];
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
              if (lane == 0) red[qd * N + c0 + j] = m;
            }
          }
        }
      }
      if (WIDE) tmem_st_wait();
      tc_before();
      __syncthreads();
      tc_after();
      if (FP8 && tid < N) {
        const float m = fmaxf(fmaxf(red[tid], red[N + tid]), fmaxf(red[2 * N + tid], red[3 * N + tid]));
        vsc[tid] = m > 0.f ? m / QMAX : 1.f;
      }
      if (a.snapshot_every > 0 && (s + 1) % a.snapshot_every == 0)
        write_rows(a.V_snap + ((s + 1) / a.snapshot_every - 1) * (int64_t)nc * k);
      __syncthreads();
      if (FP8) build_vq();
      if (WIDE) publish_own(vimg_cl + (size_t)((s + 1) & 1) * img_bytes);
    }

    // -- the new owned rows into every CTA's V image --
    if (CL > 1 && !WIDE) {
      if (!dbl) cluster.sync();  // single image: every CTA has finished reading it
      if (active) {
        const int nrow = min(N, nc - own_lo);
        for (int idx = tid; idx < nrow * L.CRb; idx += TC_THREADS) {
          const int i = idx / L.CRb, rg = idx % L.CRb, comp = own_lo + i;
          const size_t off = (((size_t)(comp >> 3) * L.CRb + rg) << 7) + ((comp & 7) << 4);
          const uint4 w = *reinterpret_cast<const uint4*>(Vn + off);
          for (int c = 0; c < CL; ++c)
            if (c != q) *reinterpret_cast<uint4*>(cluster.map_shared_rank(Vn + off, c)) = w;
        }
      }
      fence_async_cluster();
    }
    fence_async_smem();
    cluster.sync();
    fence_async_smem();
    if (dbl) cur ^= 1;
    gbase += nt;
    gstage = (int)((gstage + nt) % NS);
    if (++jb == a.spe) jb = 0;
  }
  cp_async_wait(0);
  if (active) write_rows(a.V);
  cx.ph = ph;
  cluster.sync();
}

__device__ __forceinline__ void tc_setup(TcCtx& cx, uint64_t* mbar, uint32_t* tmem_base,
                                         int* s_abort) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tmem_alloc(tmem_base, TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < NMBAR; ++i) mbar_init(&mbar[i], 1);
    mbar_fence_init();
    *s_abort = 0;
  }
  tc_before();
  __syncthreads();
  tc_after();
  cx.mbar = mbar;
  cx.abort = s_abort;
  cx.tmem = *tmem_base;
  cx.ph = 0;
}

// Frees TMEM; after a timeout, first waits (bounded) for this CTA's MMAs.
__device__ __forceinline__ void tc_teardown(TcCtx& cx) {
  if (threadIdx.x == 0 && *cx.abort) {
    mma_commit(&cx.mbar[4]);
    mbar_wait(&cx.mbar[4], (cx.ph >> 4) & 1u);
  }
  tc_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(cx.tmem, TMEM_COLS);
}

template <bool FP8, bool SYM, bool WIDE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    sgd_tc_kernel(TcArgs a, int NS, int dbl, uint8_t* vimg) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[NMBAR];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  TcCtx cx;
  tc_setup(cx, mbar, &tmem_base, &s_abort);
  tc_chain<FP8, SYM, WIDE>(a, smem, cx, NS, dbl != 0, vimg);
  tc_teardown(cx);
}

// Persistent batched form: every cluster takes (problem, restart) chains from
// a cost-ordered work list until it is exhausted.  Cluster rank 0 claims the
// next item with one atomic and broadcasts it through distributed shared memory.
template <bool FP8, bool WIDE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    sgd_tc_batched_kernel(const TcArgs* __restrict__ items, int nitems, int* counter, int NS,
                          int dbl, uint8_t* vimg) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[NMBAR];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  __shared__ int s_item;
  cg::cluster_group cluster = cg::this_cluster();
  TcCtx cx;
  tc_setup(cx, mbar, &tmem_base, &s_abort);
  while (true) {
    if (cluster.block_rank() == 0 && threadIdx.x == 0) {
      const int it = atomicAdd(counter, 1);
      for (int c = 0; c < (int)cluster.num_blocks(); ++c) *cluster.map_shared_rank(&s_item, c) = it;
    }
    cluster.sync();
    const int it = s_item;
    if (it >= nitems) break;
    const TcArgs a = items[it];
    tc_chain<FP8, true, WIDE>(a, smem, cx, NS, dbl != 0,
                        vimg ? vimg + (size_t)(blockIdx.x / cluster.num_blocks()) * VIMG_BYTES
                             : nullptr);
  }
  tc_teardown(cx);
}

// quantise rows: FP8 -> per-row scale amax/448; BF16 -> scale 1.  Output row
// stride ldq (zero padded).  two (FP8 only): the rounding residual's e4m3 term
// into a second plane n rows after the first, at the same scale.
template <bool FP8>
__global__ void quantize_rows_kernel(const float* __restrict__ Y, int64_t n, int k, int ldq,
                                     uint8_t* __restrict__ Yq, float* __restrict__ scale,
                                     int two) {
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
      if (two) {
        const __nv_fp8_e4m3 q2(v - (float)q);
        Yq[(n + r) * ldq + c] = *reinterpret_cast<const uint8_t*>(&q2);
      }
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      reinterpret_cast<__nv_bfloat16*>(Yq)[r * ldq + c] = h;
    }
  }
  if (lane == 0 && scale) scale[r] = sc;
}

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

// Launch shape of one chain: cluster size, owned components per CTA, sample
// stages, single or double V image, dynamic shared memory.
struct TcPlan {
  int CL, N, NS;
  bool dbl;
  size_t smem;
  bool wide;  // k > 128: needs VIMG_BYTES of global scratch per cluster (streamed V images)
};

// Whether the schedule (CL CTAs per chain, NS sample stages, single or double V
// image) fits tensor memory, registers and shared memory for k components.
bool tc_plan_fits(int k, bool sym, bool fp8, int CL, bool dbl, int NS, TcPlan* out,
                  int planes = 1) {
  const int N = own_cols(k, CL);
  const int KPc = k <= 128 ? 128 : 256, MB = KPc / 128;
  if (N > 128 || (fp8 && N > 64)) return false;
  if (MB > 1 && 128 % N != 0) return false;  // owned rows inside one 128-row block
  const int nvd = sym ? 1 : 2;
  // tensor memory columns: first product, second product, then either the means (16)
  // or, for k > 128, G_gram and the FP32 master rows per 128-row block
  if (2 * nvd * N + MB * (fp8 ? 2 : 1) * N + (MB > 1 ? 2 * MB * N : 16) > (int)TMEM_COLS)
    return false;
  if (dbl && CL == 1) return false;
  const size_t lim = (size_t)max_smem_optin() - 1024;  // static shared variables
  const TcLayout L = tc_layout(N, sym, fp8 ? 1 : 2, NS, dbl, KPc, planes);
  if (L.vstr && (dbl || (size_t)NS * L.y_stage < (size_t)KPc * KPc * 2)) return false;
  if (L.total > lim) return false;
  *out = {CL, N, NS, dbl, L.total, L.vstr};
  return true;
}

// The schedules tried for a cluster size, deepest pipeline and double-buffered V
// image first.
constexpr int kSchedules[8][2] = {{1, 4}, {1, 3}, {0, 4}, {0, 3}, {1, 2}, {0, 2}, {1, 1}, {0, 1}};

// The first schedule of kSchedules that fits; false if none does.
bool tc_plan(int k, bool sym, bool fp8, int CL, TcPlan* out, int planes = 1) {
  for (const auto& o : kSchedules)
    if (tc_plan_fits(k, sym, fp8, CL, o[0] != 0, o[1], out, planes)) return true;
  return false;
}

// Single chain: the smallest power-of-two cluster giving every CTA at most 16
// components (more CTAs per chain shorten each step), growing if needed.
bool tc_plan_single(int k, bool sym, bool fp8, TcPlan* out, int planes = 1) {
  int CL = 1;
  while (CL < 16 && CL * 16 < round16(k)) CL *= 2;
  for (; CL <= 16; CL *= 2)
    if (tc_plan(k, sym, fp8, CL, out, planes)) return true;
  return false;
}

template <bool FP8, bool SYM>
otm_status launch_tc(const TcArgs& args, const TcPlan& P, cudaStream_t st, uint8_t* vimg) {
  auto kern = P.wide ? sgd_tc_kernel<FP8, SYM, true> : sgd_tc_kernel<FP8, SYM, false>;
  OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem));
  if (P.CL > 8)
    OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P.CL, 1, 1);
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = P.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P.CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  uint8_t* vi = P.wide ? vimg : nullptr;
  OTM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, args, P.NS, (int)P.dbl, vi));
  count_launch();
  return OTM_OK;
}

cudaLaunchConfig_t batched_cfg(const TcPlan& P, int nclusters, cudaStream_t st,
                               cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P.CL * nclusters, 1, 1);
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = P.smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P.CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// configure = set the kernel's shared-memory / cluster attributes (done by the
// prepare call, so that the launch itself issues stream work only)
template <bool FP8>
otm_status launch_batched(const TcPlan& P, const TcArgs* items, int nitems, int* counter,
                          int nclusters, cudaStream_t st, bool configure, uint8_t* vimg) {
  auto kern = P.wide ? sgd_tc_batched_kernel<FP8, true> : sgd_tc_batched_kernel<FP8, false>;
  if (configure) {
    // the device's largest shared-memory size and non-portable clusters: every
    // plan of this kernel launches under the same attributes, so a later prepare
    // (another schedule) never invalidates an earlier plan
    OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        max_smem_optin() - 1024));
    OTM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  }
  if (nitems == 0) return OTM_OK;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batched_cfg(P, nclusters, st, attr);
  uint8_t* vi = P.wide ? vimg : nullptr;
  OTM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, items, nitems, counter, P.NS, (int)P.dbl, vi));
  count_launch();
  return OTM_OK;
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

// Clusters of the batched kernel resident at once (the persistent grid); call
// after the attributes are set.  One CTA per SM if the query fails.
int batched_clusters(bool fp8, const TcPlan& P) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batched_cfg(P, 1, nullptr, attr);
  int n = 0;
  auto kern = fp8 ? (P.wide ? sgd_tc_batched_kernel<true, true> : sgd_tc_batched_kernel<true, false>)
                  : (P.wide ? sgd_tc_batched_kernel<false, true> : sgd_tc_batched_kernel<false, false>);
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
  if (e != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = std::max(1, num_sms_tc() / P.CL);
  }
  return n;
}

// A schedule of a batched group: CTAs per chain, single or double V image, sample stages.
struct Sched {
  int CL;
  bool dbl;
  int NS;
};

// autotuner cache: (group, precision, largest k, chains) -> chosen schedule
std::mutex g_tune_mu;
std::map<long long, Sched> g_tune_cache;

}  // namespace
}  // namespace otm

using namespace otm;

extern "C" {

otm_status otm_quantize_samples(const float* Y, int64_t n, int64_t k, int precision, void* Yq,
                                float* scales, void* stream) {
  clear_error();
  OTM_REQUIRE(Y && Yq && n >= 1 && k >= 1 && k <= TC_KMAX, "otm_quantize_samples: bad arguments");
  OTM_REQUIRE(precision == OTM_PREC_BF16 || precision == OTM_PREC_FP8 ||
                  precision == OTM_PREC_FP8X2,
              "otm_quantize_samples: precision must be OTM_PREC_BF16, OTM_PREC_FP8 or "
              "OTM_PREC_FP8X2");
  OTM_REQUIRE(precision == OTM_PREC_BF16 || scales, "otm_quantize_samples: FP8 needs scales");
  const int ldq = (int)((k + 15) & ~15);
  cudaStream_t st = as_stream(stream);
  const unsigned grid = (unsigned)((n + 7) / 8);
  if (precision != OTM_PREC_BF16)
    quantize_rows_kernel<true><<<grid, 256, 0, st>>>(Y, n, (int)k, ldq, (uint8_t*)Yq, scales,
                                                     precision == OTM_PREC_FP8X2);
  else
    quantize_rows_kernel<false><<<grid, 256, 0, st>>>(Y, n, (int)k, ldq, (uint8_t*)Yq, scales, 0);
  OTM_CHECK_LAUNCH();
  return OTM_OK;
}

// The error flag (256 bytes), then, for k > 128, the cluster's two streamed BF16
// images of V.
size_t otm_sgd_run_lp_workspace(void) { return 256 + VIMG_BYTES; }

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
  OTM_REQUIRE(precision == OTM_PREC_BF16 || precision == OTM_PREC_FP8 ||
                  precision == OTM_PREC_FP8X2,
              "otm_sgd_run_lp: precision must be OTM_PREC_BF16, OTM_PREC_FP8 or OTM_PREC_FP8X2");
  OTM_REQUIRE(snapshot_every >= 0 && (snapshot_every == 0 || V_snap),
              "otm_sgd_run_lp: V_snap required for snapshots");
  OTM_REQUIRE(ws && ws_bytes >= otm_sgd_run_lp_workspace(), "otm_sgd_run_lp: workspace too small");
  if (epochs == 0) return OTM_OK;
  const bool fp8 = precision != OTM_PREC_BF16;
  const bool two_y = precision == OTM_PREC_FP8X2;
  const bool sym = (YA == YB) && (YB == YC);
  TcPlan P;
  OTM_REQUIRE(tc_plan_single((int)k, sym, fp8, &P, two_y ? 2 : 1),
              "otm_sgd_run_lp: k=%lld does not fit on chip with %s views", (long long)k,
              sym ? "one" : "three");
  cudaStream_t st = as_stream(stream);
  int* err = static_cast<int*>(ws);
  OTM_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  TcArgs args{};
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
  args.lo_off = two_y ? n * args.ldq : 0;
  args.nc = (int)k;
  args.beta0 = beta0;
  args.c1 = (float)((alpha0 + 1.0) * (alpha0 + 2.0) / 2.0);
  args.c2 = (float)(alpha0 * (alpha0 + 1.0) / 2.0);
  args.c3 = (float)(alpha0 * alpha0);
  args.kappa = (float)(0.5 * (1.0 + theta));
  otm_status s_;
  uint8_t* vimg = static_cast<uint8_t*>(ws) + 256;
  if (fp8)
    s_ = sym ? launch_tc<true, true>(args, P, st, vimg) : launch_tc<true, false>(args, P, st, vimg);
  else
    s_ = sym ? launch_tc<false, true>(args, P, st, vimg) : launch_tc<false, false>(args, P, st, vimg);
  if (s_ != OTM_OK) return s_;
  int h = 0;
  OTM_CHECK_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h) return set_error(OTM_ETIMEOUT, "otm_sgd_run_lp: a tensor-core wait timed out");
  return OTM_OK;
}

// Batched workspace: header, work list, trial work list, trial V matrices, and
// for the k > 128 group the streamed V images (VIMG_BYTES for each of at most
// WIDE_CLUSTERS clusters of at least 4 CTAs).
constexpr int WIDE_CLUSTERS = 64;

// Clusters of plan P whose images fit the wide scratch.
static int wide_clusters_cap(const TcPlan&) { return WIDE_CLUSTERS; }
struct BatchedWs {
  int* hdr;
  TcArgs* dev_items;
  TcArgs* trial_items;
  float* scratchV;
  uint8_t* vimg_wide;
};

static BatchedWs batched_ws(void* ws, size_t ws_bytes, int64_t nitems) {
  Workspace w(ws, ws_bytes);
  BatchedWs b;
  b.hdr = w.take<int>(64);
  b.dev_items = w.take<TcArgs>(nitems);
  b.trial_items = w.take<TcArgs>(nitems);
  b.scratchV = w.take<float>((size_t)std::min<int64_t>(nitems, 512) * TC_KMAX * TC_KMAX);
  b.vimg_wide = w.take<uint8_t>((size_t)WIDE_CLUSTERS * VIMG_BYTES);
  return b;
}

size_t otm_sgd_batched_workspace(int64_t nitems) {
  WorkspaceSize w;
  w.add<int>(64).add<TcArgs>(nitems).add<TcArgs>(nitems).add<float>(
      (size_t)std::min<int64_t>(nitems, 512) * TC_KMAX * TC_KMAX)
      .add<uint8_t>((size_t)WIDE_CLUSTERS * VIMG_BYTES);
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
    // restarts of a problem with k <= 64 share samples, permutation and schedule: up to
    // floor(128 / k) of them run as one chain of R k components, so that each sample tile
    // is loaded and multiplied once for all of them (the Gram term stays per restart)
    const int64_t rs = P.k <= 64 ? 128 / P.k : 1;
    for (int64_t r = 0; r < P.restarts; r += rs) {
      const int64_t cnt = std::min<int64_t>(rs, P.restarts - r);
      TcArgs a{};
      a.YA = a.YB = a.YC = static_cast<const uint8_t*>(P.Yq);
      a.lo_off = 0;  // one e4m3 term per sample (two-term samples: single chains only)
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
      a.nc = (int)(cnt * P.k);
      a.beta0 = P.beta0;
      a.c1 = (float)((P.alpha0 + 1.0) * (P.alpha0 + 2.0) / 2.0);
      a.c2 = (float)(P.alpha0 * (P.alpha0 + 1.0) / 2.0);
      a.c3 = (float)(P.alpha0 * P.alpha0);
      a.kappa = (float)(0.5 * (1.0 + P.theta));
      items.push_back(a);
      cost.push_back((double)a.total_steps *
                     ((double)P.b * a.nc * P.k + (double)a.nc * a.nc * P.k));
    }
  }
  const int nitems = (int)items.size();
  OTM_REQUIRE(ws_bytes >= otm_sgd_batched_workspace(nitems),
              "otm_sgd_batched_prepare: workspace too small (need %zu bytes)",
              otm_sgd_batched_workspace(nitems));
  // two groups, each its own persistent launch: k <= 128 (autotuned cluster) first,
  // then k > 128 (256 padded coordinates, 4- to 16-CTA clusters); longest chains first
  // within a group, so that the tail of each persistent loop holds short ones
  std::vector<int> order(nitems);
  for (int i = 0; i < nitems; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const bool wx = items[x].k > 128, wy = items[y].k > 128;
    if (wx != wy) return wy;
    return cost[x] > cost[y];
  });
  std::vector<TcArgs> sorted(nitems);
  for (int i = 0; i < nitems; ++i) sorted[i] = items[order[i]];
  int n_wide = 0, max_k_wide = 0;
  max_k = 0;
  for (const TcArgs& a : sorted) {  // plans are sized by components (k <= 128: up to 128)
    if (a.k > 128) {
      ++n_wide;
      max_k_wide = std::max(max_k_wide, a.nc);
    } else {
      max_k = std::max(max_k, a.nc);
    }
  }
  const int n_narrow = nitems - n_wide;
  const BatchedWs bw = batched_ws(ws, ws_bytes, nitems);
  int* hdr = bw.hdr;
  TcArgs* dev_items = bw.dev_items;
  TcArgs* trial_items = bw.trial_items;
  float* scratchV = bw.scratchV;
  cudaStream_t st = as_stream(stream);
  for (int i = 0; i < nitems; ++i) sorted[i].err = hdr + 1;
  OTM_CHECK_CUDA(cudaMemcpyAsync(dev_items, sorted.data(), sizeof(TcArgs) * nitems,
                                 cudaMemcpyHostToDevice, st));
  OTM_CHECK_CUDA(cudaMemsetAsync(hdr, 0, 64 * sizeof(int), st));
  // Schedules of a group: the cluster size (CTAs per chain: the width of a CTA's
  // tile of components), the number of sample stages and a single or double V
  // image.  Cluster sizes that leave a CTA without components of the group's
  // largest chain are used only when no other fits.
  auto schedules = [&](int kmax, bool wide, int only_cl) {
    std::vector<Sched> full, idle;
    const int cls[5] = {1, 2, 4, 8, 16};
    for (int c : cls) {
      if (wide && c < 4) continue;
      if (only_cl && c != only_cl) continue;
      const bool busy = (c - 1) * own_cols(kmax, c) < round16(kmax);
      for (const auto& o : kSchedules) {
        TcPlan Pc;
        if (!tc_plan_fits(kmax, true, fp8, c, o[0] != 0, o[1], &Pc)) continue;
        (busy ? full : idle).push_back({c, o[0] != 0, o[1]});
      }
    }
    return full.empty() ? idle : full;
  };
  // The autotuner: a short trial of the group's chains (at most 512, at most 4
  // steps each, on scratch V) for each schedule, the fastest of two timed
  // repetitions kept; cached per (precision, group, largest k, chains).
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto tune = [&](const std::vector<Sched>& cands, int kmax, int first, int count, bool wide,
                  Sched* best_out) -> otm_status {
    const long long key = ((long long)wide << 62) | ((long long)precision << 40) |
                          ((long long)kmax << 24) | count;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto f = g_tune_cache.find(key);
      if (f != g_tune_cache.end()) {
        *best_out = f->second;
        return OTM_OK;
      }
    }
    Sched best = cands.front();
    if (cands.size() > 1) {
      const int ntrial = std::min(count, 512);
      std::vector<TcArgs> trial(sorted.begin() + first, sorted.begin() + first + ntrial);
      for (int i = 0; i < ntrial; ++i) {
        trial[i].V = scratchV + (size_t)i * TC_KMAX * TC_KMAX;
        trial[i].total_steps = std::min<int64_t>(trial[i].total_steps, 4);
      }
      OTM_CHECK_CUDA(cudaMemsetAsync(scratchV, 0, sizeof(float) * ntrial * TC_KMAX * TC_KMAX, st));
      OTM_CHECK_CUDA(cudaMemcpyAsync(trial_items, trial.data(), sizeof(TcArgs) * ntrial,
                                     cudaMemcpyHostToDevice, st));
      if (!e0) {
        OTM_CHECK_CUDA(cudaEventCreate(&e0));
        OTM_CHECK_CUDA(cudaEventCreate(&e1));
      }
      float best_ms = 3.0e38f;
      for (const Sched& c : cands) {
        TcPlan Pc;
        tc_plan_fits(kmax, true, fp8, c.CL, c.dbl, c.NS, &Pc);
        OTM_TRY(fp8 ? launch_batched<true>(Pc, trial_items, 0, hdr + 8, 1, st, true, nullptr)
                    : launch_batched<false>(Pc, trial_items, 0, hdr + 8, 1, st, true, nullptr));
        int ncl = std::min(batched_clusters(fp8, Pc), ntrial);
        if (wide) ncl = std::min(ncl, wide_clusters_cap(Pc));
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
          OTM_CHECK_CUDA(cudaMemsetAsync(hdr + 8, 0, sizeof(int), st));
          OTM_CHECK_CUDA(cudaEventRecord(e0, st));
          OTM_TRY(fp8 ? launch_batched<true>(Pc, trial_items, ntrial, hdr + 8, ncl, st, false,
                                             wide ? bw.vimg_wide : nullptr)
                      : launch_batched<false>(Pc, trial_items, ntrial, hdr + 8, ncl, st, false,
                                              wide ? bw.vimg_wide : nullptr));
          OTM_CHECK_CUDA(cudaEventRecord(e1, st));
          OTM_CHECK_CUDA(cudaEventSynchronize(e1));
          OTM_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));  // the second: code and caches warm
        }
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    *best_out = best;
    return OTM_OK;
  };
  Sched sn{16, false, 1}, sw{16, false, 1};
  otm_status tuned = OTM_OK;
  if (n_narrow > 0) {
    // a given cluster size keeps its first fitting schedule (the single-chain one)
    const std::vector<Sched> cands = schedules(max_k, false, cluster);
    if (cands.empty()) {
      tuned = set_error(OTM_EINVAL, cluster ? "otm_sgd_batched_prepare: cluster %d does not fit k=%d"
                                            : "otm_sgd_batched_prepare: k=%d does not fit shared memory",
                        cluster ? cluster : max_k, max_k);
    } else if (cluster) {
      sn = cands.front();
    } else {
      tuned = tune(cands, max_k, 0, n_narrow, false, &sn);
    }
  }
  if (tuned == OTM_OK && n_wide > 0) {
    const std::vector<Sched> cands = schedules(max_k_wide, true, 0);
    if (cands.empty())
      tuned = set_error(OTM_EINVAL, "otm_sgd_batched_prepare: k=%d does not fit on chip", max_k_wide);
    else
      tuned = tune(cands, max_k_wide, n_narrow, n_wide, true, &sw);
  }
  if (e0) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (tuned != OTM_OK) return tuned;
  TcPlan Pch{}, Pw{};
  if (n_narrow > 0)
    OTM_REQUIRE(tc_plan_fits(max_k, true, fp8, sn.CL, sn.dbl, sn.NS, &Pch),
                "otm_sgd_batched_prepare: no plan");
  if (n_wide > 0)
    OTM_REQUIRE(tc_plan_fits(max_k_wide, true, fp8, sw.CL, sw.dbl, sw.NS, &Pw),
                "otm_sgd_batched_prepare: no plan");
  // each group's kernel takes the launch attributes
  for (int grp = 0; grp < 2; ++grp) {
    if ((grp == 0 ? n_narrow : n_wide) == 0) continue;
    const TcPlan& Pg = grp == 0 ? Pch : Pw;
    otm_status s3 = fp8 ? launch_batched<true>(Pg, dev_items, 0, hdr, 1, st, true, nullptr)
                        : launch_batched<false>(Pg, dev_items, 0, hdr, 1, st, true, nullptr);
    if (s3 != OTM_OK) return s3;
  }
  OTM_CHECK_CUDA(cudaStreamSynchronize(st));
  plan->nitems = nitems;
  plan->cluster = n_narrow > 0 ? sn.CL : 0;
  plan->precision = precision;
  plan->max_k = max_k;
  plan->smem_bytes = (int64_t)Pch.smem;
  plan->grid_clusters = n_narrow > 0 ? std::min(batched_clusters(fp8, Pch), n_narrow) : 0;
  plan->nitems_wide = n_wide;
  plan->max_k_wide = max_k_wide;
  plan->cluster_wide = n_wide > 0 ? sw.CL : 0;
  plan->grid_clusters_wide =
      n_wide > 0 ? std::min(std::min(batched_clusters(fp8, Pw), wide_clusters_cap(Pw)), n_wide) : 0;
  plan->stages = n_narrow > 0 ? sn.NS : 0;
  plan->vimg2 = n_narrow > 0 ? (int32_t)sn.dbl : 0;
  plan->stages_wide = n_wide > 0 ? sw.NS : 0;
  plan->vimg2_wide = n_wide > 0 ? (int32_t)sw.dbl : 0;
  plan->ws = ws;
  plan->ws_bytes = ws_bytes;
  return OTM_OK;
}

otm_status otm_sgd_batched_launch(const otm_batch_plan* plan, void* stream) {
  clear_error();
  OTM_REQUIRE(plan && plan->ws && plan->nitems >= 1 && plan->nitems_wide >= 0 &&
                  plan->nitems_wide <= plan->nitems,
              "otm_sgd_batched_launch: invalid plan");
  const int n_wide = plan->nitems_wide, n_narrow = plan->nitems - n_wide;
  cudaStream_t st = as_stream(stream);
  const BatchedWs bw = batched_ws(plan->ws, plan->ws_bytes, plan->nitems);
  int* hdr = bw.hdr;
  TcArgs* dev_items = bw.dev_items;
  OTM_CHECK_CUDA(cudaMemsetAsync(hdr, 0, 3 * sizeof(int), st));  // counters and the flag
  const bool fp8 = plan->precision == OTM_PREC_FP8;
  if (n_narrow > 0) {
    TcPlan P;
    OTM_REQUIRE(tc_plan_fits(plan->max_k, true, fp8, plan->cluster, plan->vimg2 != 0,
                             plan->stages, &P) &&
                    (int64_t)P.smem == plan->smem_bytes && plan->grid_clusters >= 1,
                "otm_sgd_batched_launch: plan does not match this library");
    OTM_TRY(fp8 ? launch_batched<true>(P, dev_items, n_narrow, hdr, plan->grid_clusters, st,
                                       false, nullptr)
                : launch_batched<false>(P, dev_items, n_narrow, hdr, plan->grid_clusters, st,
                                        false, nullptr));
  }
  if (n_wide > 0) {
    TcPlan P;
    OTM_REQUIRE(tc_plan_fits(plan->max_k_wide, true, fp8, plan->cluster_wide,
                             plan->vimg2_wide != 0, plan->stages_wide, &P) &&
                    plan->grid_clusters_wide >= 1 &&
                    plan->grid_clusters_wide <= wide_clusters_cap(P),
                "otm_sgd_batched_launch: plan does not match this library");
    OTM_TRY(fp8 ? launch_batched<true>(P, dev_items + n_narrow, n_wide, hdr + 2,
                                       plan->grid_clusters_wide, st, false, bw.vimg_wide)
                : launch_batched<false>(P, dev_items + n_narrow, n_wide, hdr + 2,
                                        plan->grid_clusters_wide, st, false, bw.vimg_wide));
  }
  return OTM_OK;
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
