// Grid-wide barrier for kernels launched cooperatively (every CTA resident).
#pragma once

namespace otm {

// About 2 s at the maximum SM clock: far beyond any legitimate wait.
constexpr long long GRID_WAIT_CYCLES = 4000000000LL;

// One counter, to which CTA 0 adds 2^31 - (gridDim.x - 1) and every other CTA
// 1, so that bit 31 flips once all have arrived; arrival is a release, the
// wait an acquire.  The counter starts at zero and is never reset.  Returns
// false if the wait timed out; *flag is then set to `code`.
__device__ __forceinline__ bool grid_barrier(unsigned* count, int* flag, int code) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    unsigned old, v;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(count), "r"(add) : "memory");
    const long long t0 = clock64();
    do {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (((v ^ old) & 0x80000000u) != 0u) break;
      if (clock64() - t0 > GRID_WAIT_CYCLES) {
        atomicExch(flag, code);
        ok = 0;
        break;
      }
    } while (true);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace otm
