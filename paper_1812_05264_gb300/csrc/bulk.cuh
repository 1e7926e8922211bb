// Shared-memory staging helpers for the TMA-fed kernels: mbarrier operations with bounded
// waits and one-dimensional bulk (cp.async.bulk) global -> shared copies.
#pragma once
#include <stdint.h>

namespace tbk {

// A wait gives up after WAIT_NS of wall time (the GPU's global timer), or after WAIT_SPINS polls
// as a backstop; no wait of a healthy launch comes near either.
constexpr uint32_t WAIT_SPINS = 1u << 22;
constexpr uint64_t WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-blocking test of a phase: a consumer tests the next stage before it works on the current
// one, so the barrier's round trip overlaps that work; true carries the same acquire as a wait.
__device__ __forceinline__ uint32_t mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// The slow path of a wait, kept out of line so that the waiting kernels' register allocation
// does not carry the timer.
static __device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < WAIT_SPINS; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u && global_ns() - t0 > WAIT_NS) return false;
  }
  return false;
}
// Bounded wait; false when the limit expired.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_slow(bar, parity);
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}


// One neighbour tile of the FP32 block product with packed f32x2 FMAs over probe pairs:
//   acc[i][h] += H^[i][l] * (x[l][2h], x[l][2h+1])   for l = 0..8,
// X: 9 x P tile in shared memory, Hs: column-major block (columns padded to 12 floats), pl: the
// thread's first probe (4 probes: h = 0, 1).  Every accumulator sums l = 0..8 in order (same
// rounding as scalar FMAs); the 9 rows need 18 packed FMAs per column, no padding row.
__device__ __forceinline__ void spmm_tile_f2(const float* X, const float* Hs, int P, int pl,
                                             float2 (&acc)[9][2]) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const float4 t = *reinterpret_cast<const float4*>(X + l * P + pl);
    const float2 x01 = make_float2(t.x, t.y), x23 = make_float2(t.z, t.w);
    float hc[12];
#pragma unroll
    for (int j = 0; j < 12; j += 4) {
      const float4 u = *reinterpret_cast<const float4*>(Hs + l * 12 + j);
      hc[j] = u.x; hc[j + 1] = u.y; hc[j + 2] = u.z; hc[j + 3] = u.w;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float2 h2 = make_float2(hc[i], hc[i]);
      acc[i][0] = __ffma2_rn(h2, x01, acc[i][0]);
      acc[i][1] = __ffma2_rn(h2, x23, acc[i][1]);
    }
  }
}

}  // namespace tbk
