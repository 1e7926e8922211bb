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


// One neighbour tile of the FP32 block product with packed f32x2 FMAs:
//   acc(i, v) += H^[i][l] * x[l][v]   for l = 0..8,
// X: 9 x P tile in shared memory, Hs: column-major block (columns padded to 12 floats), pl: the
// thread's first probe (4 probes v = 0..3).  Rows 0..7 are packed in pairs (2j, 2j + 1), whose
// H^ values sit side by side in a column, against one probe: acc[2j + (v >> 1)][v & 1]; row 8 is
// packed over probe pairs: acc[8][h] = probes (2h, 2h + 1).  Per column this takes 18 packed
// FMAs with 4 probe values and one H^ value duplicated into pairs (9 duplications when every row
// is packed over probes).  Every accumulator sums l = 0..8 in order (same rounding as scalar
// FMAs); acc_at() reads the accumulator of (i, v).
__device__ __forceinline__ void spmm_tile_f2(const float* X, const float* Hs, int P, int pl,
                                             float2 (&acc)[9][2]) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const float4 t = *reinterpret_cast<const float4*>(X + l * P + pl);
    const float xv[4] = {t.x, t.y, t.z, t.w};
    const float4 u0 = *reinterpret_cast<const float4*>(Hs + l * 12);
    const float4 u1 = *reinterpret_cast<const float4*>(Hs + l * 12 + 4);
    const float h8 = Hs[l * 12 + 8];
    const float2 hp[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y),
                          make_float2(u1.z, u1.w)};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float2 x2 = make_float2(xv[v], xv[v]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2& a = acc[2 * j + (v >> 1)][v & 1];
        a = __ffma2_rn(hp[j], x2, a);
      }
    }
    const float2 h2 = make_float2(h8, h8);
    acc[8][0] = __ffma2_rn(h2, make_float2(t.x, t.y), acc[8][0]);
    acc[8][1] = __ffma2_rn(h2, make_float2(t.z, t.w), acc[8][1]);
  }
}

// The accumulator of row i, probe v (0..3) in the layout spmm_tile_f2 fills.
__device__ __forceinline__ float acc_at(const float2 (&acc)[9][2], int i, int v) {
  if (i == 8) return (v & 1) ? acc[8][v >> 1].y : acc[8][v >> 1].x;
  const float2 p = acc[2 * (i >> 1) + (v >> 1)][v & 1];
  return (i & 1) ? p.y : p.x;
}

// The same tile product with every row packed over probe pairs: acc[i][h] += H^[i][l] *
// (x[l][2h], x[l][2h + 1]), nine H^ values duplicated into packed operands per column.  The
// single-warp step kernel (128-probe tasks) measured faster with this form (0.317 against
// 0.333 ms per launch on the 64-cluster batch); the per-element sums are the same, so both forms
// give the same bits.  acc_at_pp() reads the accumulator of (i, v).
__device__ __forceinline__ void spmm_tile_f2_pp(const float* X, const float* Hs, int P, int pl,
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

__device__ __forceinline__ float acc_at_pp(const float2 (&acc)[9][2], int i, int v) {
  return (v & 1) ? acc[i][v >> 1].y : acc[i][v >> 1].x;
}

// Compensated FP32 accumulation (Knuth's TwoSum): s + c carries the running sum of the q's with
// each addition's rounding error kept in c, so that (double)s + (double)c matches an FP64 sum of
// the q's to ~n 2^-48 relative.  Used for a task's moment partials, which then take one FP64
// conversion and add per task instead of one per row (FP64 is a 1/64-rate pipe on this part).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float q) {
  const float t = __fadd_rn(s, q);
  const float bb = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(q, bb));
  s = t;
  c = __fadd_rn(c, err);
}

}  // namespace tbk
