// Tensor-core recurrence step (tcgen05, TF32 split three ways for FP32 accuracy).
//
// One task = one block row a and a chunk of 128 probes (one probe per consumer thread).  For
// every neighbour block (a, b) the producer warp streams the 9 x 128 panel tile of y_in rows
// 9b..9b+8 and the mapped block H^_ab into a shared-memory ring (bulk copies on mbarriers, as in
// the TMA-fed SIMT kernel).  Each consumer thread reads the 9 orbital values of its probe, splits
// them into a TF32 head and a remainder, and stores both into TMEM (lane = probe) as the A operand
// (M = 128 probes x K = 9 per tile, tiles stacked along K in groups of GROUP); the block is written
// K-major into shared memory as the B operand (N = 16 output rows, 9 used), head and remainder.
// One thread then issues, per K step of 8, the three MMAs  A_hi B_hi + A_hi B_lo + A_lo B_hi  into
// the accumulator D[128 x 16] in TMEM.  After the task's last group the consumers read D back
// (tcgen05.ld, one probe per lane) and finish the step exactly as the SIMT kernels do:
//   y_out = alpha D + c_r r - y_prev, with the moment partial sums.
// Every wait is bounded; on expiry the CTA raises *err = 2, stops waiting, runs its remaining
// control flow to the end and still frees its TMEM.
#include "bulk.cuh"
#include "cheb.cuh"

namespace tbk {

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // shared-memory matrix descriptor: start >> 4, leading (K) and stride (8-row group) byte
  // offsets >> 4, version 1, no swizzle
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

__device__ __forceinline__ void tm_st1(uint32_t addr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void tm_st8(uint32_t addr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

template <int GROUP, int D>
struct TcCfg {
  static constexpr int P = 128;
  static constexpr int XB = 9 * P * 4;
  static constexpr int HB = Layout<float, 9>::BS * 4;
  static constexpr int SB = ((XB + HB + 127) / 128) * 128;
  static constexpr int KG = 9 * GROUP;
  static constexpr int KP = ((KG + 7) / 8) * 8;
  static constexpr int LBO = 128;                 // next core matrix along K
  static constexpr int SBO = (KP / 4) * 128;      // next group of 8 rows (N)
  static constexpr int BBYTES = 16 * KP * 4;      // one B operand buffer (16 rows)
  static constexpr int NCOL = 16 + 2 * KP;        // TMEM columns used: D | A_hi | A_lo
  static constexpr int TCOLS = NCOL <= 32 ? 32 : (NCOL <= 64 ? 64 : (NCOL <= 128 ? 128 : 256));
  static constexpr int SMEM = D * SB + 2 * BBYTES + 8 * (2 * D + 2) + 16;
  static constexpr int THREADS = 160;
};

template <int GROUP, int D>
__global__ void __launch_bounds__(160)
cheb_step_tc(const int n_atoms, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
             const float* __restrict__ hv, const float* __restrict__ yin, const float* yprev,
             float* yout, const float alpha, const float c_r, const uint64_t seed, const int s,
             const int direct, double* __restrict__ partials, int* __restrict__ err) {
  using C = TcCfg<GROUP, D>;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* Bh = smem + D * C::SB;
  unsigned char* Bl = Bh + C::BBYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bl + C::BBYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * D + 2);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (D + i); };
  const uint32_t mma_bar = bar0 + 8u * (2 * D);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_chunks = s / C::P;
  const int n_tasks = n_atoms * n_chunks;
  const bool has_prev = yprev != nullptr;

  if (tid == 0) {
    for (int i = 0; i < D; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 4);
    }
    mbar_init(mma_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B rows 9..15 (and every pad column) stay zero
  for (int e = tid; e < 2 * C::BBYTES / 16; e += blockDim.x)
    reinterpret_cast<float4*>(Bh)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = *tmem_slot;

  if (warp == 4) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int task = blockIdx.x; task < n_tasks && ok; task += gridDim.x) {
        const int a = task / n_chunks, ch = task - a * n_chunks;
        const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
        const int nt = k1 - k0 + (has_prev ? 1 : 0);
        for (int q = 0; q < nt && ok; ++q) {
          const bool is_prev = q == k1 - k0;
          const int b = is_prev ? a : __ldg(col + k0 + q);
          const int st = it % D;
          ok = mbar_wait(empty(st), ((it / D) & 1) ^ 1);
          if (!ok) break;
          const uint32_t dst = smem_u32(smem + st * C::SB), bar = full(st);
          const float* src = (is_prev ? yprev : yin) + (int64_t)9 * b * s + (int64_t)ch * C::P;
          mbar_expect_tx(bar, C::XB + (is_prev ? 0 : C::HB));
          if (C::P == s) {
            bulk_g2s(dst, src, C::XB, bar);
          } else {
            for (int l = 0; l < 9; ++l) bulk_g2s(dst + l * C::P * 4, src + (int64_t)l * s, C::P * 4, bar);
          }
          if (!is_prev) bulk_g2s(dst + C::XB, hv + (int64_t)(k0 + q) * Layout<float, 9>::BS, C::HB, bar);
          ++it;
        }
      }
      if (!ok) {
        atomicOr(err, 2);
        for (int j = (it > D ? it - D : 0); j < it; ++j) mbar_wait(full(j % D), (j / D) & 1);
      }
    }
  } else {
    // ---------------- consumers: thread tid <-> probe tid of the chunk <-> TMEM lane tid ----------------
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
    double sum0 = 0.0, sum1 = 0.0;
    int it = 0, ncommit = 0;
    bool ok = true;
    // B entry (n = row i, k) of one buffer, bytes
    auto boff = [&](int n, int k) { return (n >> 3) * C::SBO + (k >> 2) * C::LBO + (n & 7) * 16 + (k & 3) * 4; };
    for (int task = blockIdx.x; task < n_tasks; task += gridDim.x) {
      const int a = task / n_chunks, ch = task - a * n_chunks;
      const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
      const int ntile = k1 - k0;
      float yc[9];
#pragma unroll
      for (int l = 0; l < 9; ++l) yc[l] = 0.f;
      bool first_mma = true;
      for (int g0 = 0; g0 < ntile; g0 += GROUP) {
        const int gn = min(GROUP, ntile - g0);
        const int kfill = 9 * gn, ksteps = (kfill + 7) / 8;
        // the previous group's MMAs must be done before A and B are overwritten
        if (ncommit > 0 && ok) ok = mbar_wait(mma_bar, (ncommit - 1) & 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // zero the pad columns of the last K step (A in TMEM, B in shared memory)
        for (int k = kfill; k < 8 * ksteps; ++k) {
          tm_st1(tm + lane_base + 16 + k, 0u);
          tm_st1(tm + lane_base + 16 + C::KP + k, 0u);
        }
        for (int e = tid; e < 9 * (8 * ksteps - kfill); e += 128) {
          const int n = e / (8 * ksteps - kfill), k = kfill + e % (8 * ksteps - kfill);
          *reinterpret_cast<float*>(Bh + boff(n, k)) = 0.f;
          *reinterpret_cast<float*>(Bl + boff(n, k)) = 0.f;
        }
        for (int slot = 0; slot < gn; ++slot) {
          const int q = g0 + slot;
          const int st = it % D;
          if (ok) ok = mbar_wait(full(st), (it / D) & 1);
          const float* X = reinterpret_cast<const float*>(smem + st * C::SB);
          const float* Hs = reinterpret_cast<const float*>(smem + st * C::SB + C::XB);
          uint32_t hi[9], lo[9];
#pragma unroll
          for (int l = 0; l < 9; ++l) {
            const float v = X[l * C::P + tid];
            const float h = tf32_head(v);
            hi[l] = __float_as_uint(h);
            lo[l] = __float_as_uint(v - h);
          }
          if (__ldg(col + k0 + q) == a) {
#pragma unroll
            for (int l = 0; l < 9; ++l) yc[l] = X[l * C::P + tid];
          }
          const uint32_t c0 = 16 + 9 * slot;
          tm_st8(tm + lane_base + c0, hi);
          tm_st1(tm + lane_base + c0 + 8, hi[8]);
          tm_st8(tm + lane_base + C::KP + c0, lo);
          tm_st1(tm + lane_base + C::KP + c0 + 8, lo[8]);
          if (tid < 81) {
            // block entry (i, l) = stored column l, row i; B[n = i][k = 9 slot + l]
            const int i = tid / 9, l = tid - 9 * (tid / 9);
            const float v = Hs[l * 12 + i], h = tf32_head(v);
            *reinterpret_cast<float*>(Bh + boff(i, 9 * slot + l)) = h;
            *reinterpret_cast<float*>(Bl + boff(i, 9 * slot + l)) = v - h;
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(empty(st));
          ++it;
        }
        // hand A (TMEM) and B (shared memory) to the tensor core
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t bh = smem_u32(Bh) + ks * 2 * C::LBO, bl = smem_u32(Bl) + ks * 2 * C::LBO;
            const uint64_t dh = umma_desc(bh, C::LBO, C::SBO), dl = umma_desc(bl, C::LBO, C::SBO);
            const uint32_t ah = tm + 16 + 8 * ks, al = tm + 16 + C::KP + 8 * ks;
            const uint32_t acc0 = first_mma ? 0u : 1u;
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
                         ::"r"(tm), "r"(ah), "l"(dh), "r"(idesc), "r"(acc0));
            asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;"
                         ::"r"(tm), "r"(ah), "l"(dl), "r"(idesc));
            asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;"
                         ::"r"(tm), "r"(al), "l"(dh), "r"(idesc));
            first_mma = false;
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mma_bar)
                       : "memory");
        }
        first_mma = false;
        ++ncommit;
      }
      // the task's last MMAs, then D back to registers (lane = probe, columns = output rows)
      if (ok) ok = mbar_wait(mma_bar, (ncommit - 1) & 1);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t dr[16];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(dr[0]), "=r"(dr[1]), "=r"(dr[2]), "=r"(dr[3]), "=r"(dr[4]), "=r"(dr[5]), "=r"(dr[6]),
                     "=r"(dr[7]), "=r"(dr[8]), "=r"(dr[9]), "=r"(dr[10]), "=r"(dr[11]), "=r"(dr[12]),
                     "=r"(dr[13]), "=r"(dr[14]), "=r"(dr[15])
                   : "r"(tm + lane_base));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float yp[9];
#pragma unroll
      for (int l = 0; l < 9; ++l) yp[l] = 0.f;
      if (has_prev) {
        const int st = it % D;
        if (ok) ok = mbar_wait(full(st), (it / D) & 1);
        const float* X = reinterpret_cast<const float*>(smem + st * C::SB);
#pragma unroll
        for (int l = 0; l < 9; ++l) yp[l] = X[l * C::P + tid];
        __syncwarp();
        if (lane == 0) mbar_arrive(empty(st));
        ++it;
      }
      const int p = ch * C::P + tid;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int64_t row = (int64_t)9 * a + i;
        float yo = alpha * __uint_as_float(dr[i]);
        float r = 0.f;
        if (c_r != 0.f || direct) r = tbk_probe_sign(seed, row, p);
        if (c_r != 0.f) yo = fmaf(c_r, r, yo);
        yo -= yp[i];
        yout[row * s + p] = yo;
        if (partials) {
          sum0 += (double)(yo * (direct ? r : yc[i]));
          sum1 += (double)(yo * yo);
        }
      }
    }
    if (!ok) atomicOr(err, 2);
    // make sure no MMA of this CTA is still running before TMEM is released
    if (tid == 0 && ncommit > 0) mbar_wait(mma_bar, (ncommit - 1) & 1);
    if (partials) {
      __shared__ double red[2][4];
      for (int o = 16; o > 0; o >>= 1) {
        sum0 += __shfl_xor_sync(0xffffffffu, sum0, o);
        sum1 += __shfl_xor_sync(0xffffffffu, sum1, o);
      }
      if (lane == 0) {
        red[0][warp] = sum0;
        red[1][warp] = sum1;
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (tid == 0) {
        partials[2 * blockIdx.x] = red[0][0] + red[0][1] + red[0][2] + red[0][3];
        partials[2 * blockIdx.x + 1] = red[1][0] + red[1][1] + red[1][2] + red[1][3];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (warp == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(C::TCOLS));
    }
  }
}

constexpr int TC_GROUP = 4;
constexpr int TC_D = 4;

static int tc_occupancy() {
  using C = TcCfg<TC_GROUP, TC_D>;
  static int occ[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!occ[dev]) {
    cudaFuncSetAttribute(cheb_step_tc<TC_GROUP, TC_D>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cheb_step_tc<TC_GROUP, TC_D>, C::THREADS, C::SMEM);
    // TMEM: 512 columns per SM shared by the resident CTAs
    n = std::min(n, 512 / C::TCOLS);
    occ[dev] = n > 0 ? n : -1;
  }
  return occ[dev];
}

bool tc_eligible(const HOp& op, int s) {
  return op.prec == TBK_MIXED && op.B == 9 && s % 128 == 0 && tc_occupancy() > 0;
}

int tc_grid(tbk_ctx* ctx) { return std::max(1, tc_occupancy()) * ctx->num_sms; }

void launch_step_tc(tbk_ctx* ctx, const HOp& op, const StepArgs& a, int G) {
  using C = TcCfg<TC_GROUP, TC_D>;
  cheb_step_tc<TC_GROUP, TC_D><<<G, C::THREADS, C::SMEM, ctx->stream>>>(
      op.n_atoms, op.row_ptr, op.col, (const float*)op.hv, (const float*)a.yin, (const float*)a.yprev,
      (float*)a.yout, (float)a.alpha, (float)a.c_r, a.seed, a.s, a.direct, a.partials, a.err);
  post_launch(ctx, "cheb_step_tc");
}

}  // namespace tbk
