// Sampled outer products of the adjoint on the tensor cores (tcgen05, TF32 split three ways).
//
// For one backward index j of the adjoint of the doubled moments (Sec. II.D, Eq.
// polynomial_response in the doubled-moment form) and every stored block (a, b) of the pattern:
//   Gacc_ab[i][l] += w sum_p y[9a + i][p] x[9b + l][p],      y = y_j, x = ybar_{j+1} (FP32 panels).
// One CTA task is one block row a.  The contraction over the probes runs on the tensor cores as
//   D[m][n] = sum_p A[m][p] B[n][p]   (M = 128, N = 16, K = the probes, 32 per chunk),
// with B = the 16 panel rows of y from row 9a (the 9 of atom a used; a TMA box of 32 x 16 in the
// 128-byte swizzle, read by the MMA from shared memory) and A, held in TMEM (lane = row, one
// 32-bit column per probe), one of:
//   group g (g < NG): rows 0..7 of the neighbour tiles x_b of blocks 16g .. 16g + 15 of the row
//     (A row 8 q' + l = row l of tile 16 g + q'; a swizzled TMA box of 32 x 8 per tile and chunk);
//   the row-8 group: row 8 (the ninth orbital) of every tile of the row (A row q = tile q; a
//     32 x 1 box per tile and chunk).
// With N = 16 an operand read from shared memory would cost 4 KB per 16K multiply-adds, so the
// MMAs would wait on shared-memory bandwidth; from TMEM they read only B.
//
// FP32 accuracy from TF32 tensor cores: each operand word w is split as head(w) (what the tensor
// core reads: w with its 13 low mantissa bits cleared) + rest(w) = w - head(w), exact in FP32, and
// D accumulates head(A) head(B) + head(A) rest(B) + rest(A) head(B) in FP32 (the product of the
// two rests, below 2^-20 of the product, is dropped).  B's rest is the elementwise image of its
// swizzled head in shared memory; A's head and rest go to TMEM side by side.
//
// Warps: 0 producer (its lanes issue the TMA boxes of a chunk, one tile each, into a ring of NS
// stages), 1 MMA issuer (one thread; it also allocates TMEM), 2-5 converters (A rows from shared
// memory to TMEM, head and rest; B's rest; double-buffered A), 6-9 epilogue (D from TMEM, added to the FP64 accumulator: one CTA owns each block row, so every
// entry has one writer and the sum does not depend on timing).  D is double-buffered in TMEM
// across tasks, so a task's epilogue overlaps the next task's MMAs.  Every wait is bounded; on
// expiry the CTA raises *err = 2, stops issuing, lets its copies and MMAs land, and frees its TMEM.
#include "cheb.cuh"
#include "umma.cuh"

namespace tbk {

template <int NG>
struct TcSdCfg {
  static constexpr int NS = 4;                      // ring stages (one 32-probe chunk each)
  static constexpr int TILES = 16 * NG;             // stored blocks per row at most
  // stage layout (1024-aligned): B head (16 rows) | B rest | rows 0..7 of every tile (swizzled
  // TMA boxes) | row 8 of every tile (unswizzled boxes)
  static constexpr int O_BH = 0, O_BL = 2048, O_A = 4096, O_R8 = O_A + TILES * 1024,
                       STAGE = ((O_R8 + TILES * 128 + 1023) / 1024) * 1024;
  static constexpr int NBAR = 3 * NS + 6;           // full, lo_ready, empty per stage; a_free[2], d_full[2], d_free[2]
  static constexpr int SMEM = NS * STAGE + 8 * NBAR + 16 + 1024;  // + alignment slack
  static constexpr int THREADS = 320;
  // TMEM columns: D buffers (NG groups + the row-8 group, 16 columns each) at 0 and DCOLS; A
  // buffers (per group: 32 head columns, 32 rest columns) at A0 and A0 + ACOLS
  static constexpr int DCOLS = 16 * (NG + 1);
  static constexpr int ACOLS = 64 * (NG + 1);
  static constexpr int A0 = 128;
  static constexpr int TCOLS = 512;
  static_assert(2 * DCOLS <= A0 && A0 + 2 * ACOLS <= TCOLS, "TMEM layout");
};

template <int NG>
__global__ void __launch_bounds__(320, 1)
sddmm_tc(const int n_atoms, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
         const __grid_constant__ CUtensorMap mX8, const __grid_constant__ CUtensorMap mX1,
         const __grid_constant__ CUtensorMap mY16, const int s, const double w, double* __restrict__ Gacc,
         int* __restrict__ err) {
  using C = TcSdCfg<NG>;
  extern __shared__ unsigned char raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::NS * C::STAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + C::NBAR);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto lo_ready = [&](int i) { return bar0 + 8u * (C::NS + i); };
  auto empty = [&](int i) { return bar0 + 8u * (2 * C::NS + i); };
  auto a_free = [&](int i) { return bar0 + 8u * (3 * C::NS + i); };
  auto d_full = [&](int i) { return bar0 + 8u * (3 * C::NS + 2 + i); };
  auto d_free = [&](int i) { return bar0 + 8u * (3 * C::NS + 4 + i); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = s >> 5;

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NS; ++i) {
      mbar_init(full(i), 1);
      mbar_init(lo_ready(i), 128);
      mbar_init(empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(a_free(i), 1);
      mbar_init(d_full(i), 1);
      mbar_init(d_free(i), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tslot), C::TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = *tslot;
  bool ok = true;

  if (warp == 0) {
    // ---------------- producer: the warp's lanes issue one tile each ----------------
    int it = 0;
    for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x) {
      const int k0 = __ldg(row_ptr + a), nb = __ldg(row_ptr + a + 1) - k0;
      int bq = lane < nb ? __ldg(col + k0 + lane) : 0;
      for (int c = 0; c < nchunk; ++c, ++it) {
        const int st = it % C::NS;
        if (lane == 0) ok = mbar_wait(empty(st), ((it / C::NS) & 1) ^ 1);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        unsigned char* stg = smem + st * C::STAGE;
        const uint32_t bar = full(st);
        if (lane == 0) {
          // the stage's previous contents were read by the generic proxy
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(bar, (uint32_t)(nb * (1024 + 128) + 2048));
          tma_load_2d(smem_u32(stg + C::O_BH), &mY16, 32 * c, 9 * a, bar);
        }
        __syncwarp();
        if (lane < nb) {
          tma_load_2d(smem_u32(stg + C::O_A + lane * 1024), &mX8, 32 * c, 9 * bq, bar);
          tma_load_2d(smem_u32(stg + C::O_R8 + lane * 128), &mX1, 32 * c, 9 * bq + 8, bar);
        }
      }
    }
    if (!ok && lane == 0) {
      atomicOr(err, 2);
      // let the copies in flight land before the CTA exits
      for (int j = (it > C::NS ? it - C::NS : 0); j < it; ++j) mbar_wait(full(j % C::NS), (j / C::NS) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(128, 16);
      int it = 0, task = 0;
      for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x, ++task) {
        const int nb = __ldg(row_ptr + a + 1) - __ldg(row_ptr + a);
        const int ng = (nb + 15) >> 4;
        const int db = task & 1;
        // the epilogue of task - 2 has read this D buffer
        ok = mbar_wait(d_free(db), ((task >> 1) & 1) ^ 1);
        if (!ok) break;
        tc_fence_after();
        const uint32_t d0 = tm + db * C::DCOLS;
        for (int c = 0; c < nchunk; ++c, ++it) {
          const int st = it % C::NS;
          ok = mbar_wait(lo_ready(st), (it / C::NS) & 1);
          if (!ok) break;
          tc_fence_after();
          const uint32_t stg = smem_u32(smem + st * C::STAGE);
          const uint32_t ab = tm + C::A0 + (it & 1) * C::ACOLS;
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
            const uint64_t bh = sw128_desc(stg + C::O_BH + 32 * ks, 1024);
            const uint64_t bl = sw128_desc(stg + C::O_BL + 32 * ks, 1024);
            for (int g = 0; g <= ng; ++g) {
              // groups 0 .. ng-1: rows 0..7 of the tiles; the last: the row-8 group
              const int gi = g == ng ? NG : g;
              const uint32_t ah = ab + 64 * gi + 8 * ks, al = ah + 32;
              const uint32_t d = d0 + 16 * gi;
              umma_tf32_ta(d, ah, bh, idesc, acc);
              umma_tf32_ta(d, ah, bl, idesc, 1u);
              umma_tf32_ta(d, al, bh, idesc, 1u);
            }
          }
          umma_commit(empty(st));        // the stage may be refilled
          umma_commit(a_free(it & 1));   // the TMEM A buffer may be rewritten
        }
        if (!ok) break;
        umma_commit(d_full(db));
      }
      if (!ok) {
        atomicOr(err, 2);
        // no MMA of this CTA may run once TMEM is released: wait for the last commits' phases
        for (int j = (it > C::NS ? it - C::NS : 0); j < it; ++j) mbar_wait(empty(j % C::NS), (j / C::NS) & 1);
      }
    }
  } else if (warp < 6) {
    // ---------------- converters: 128 threads, one TMEM lane (A row) each ----------------
    const int quad = warp & 3, m = 32 * quad + lane;
    int it = 0;
    for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x) {
      const int nb = __ldg(row_ptr + a + 1) - __ldg(row_ptr + a);
      const int ng = (nb + 15) >> 4;
      for (int c = 0; c < nchunk; ++c, ++it) {
        const int st = it % C::NS;
        ok = mbar_wait(full(st), (it / C::NS) & 1);
        // the MMAs of chunk it - 2 have read this TMEM A buffer
        if (ok) ok = mbar_wait(a_free(it & 1), ((it >> 1) & 1) ^ 1);
        if (!ok) break;
        tc_fence_after();
        const unsigned char* stg = smem + st * C::STAGE;
        // B rest: 16 rows x 32 words, elementwise on the swizzled words
        {
          const float4 v = reinterpret_cast<const float4*>(stg + C::O_BH)[m];
          reinterpret_cast<float4*>(const_cast<unsigned char*>(stg) + C::O_BL)[m] =
              make_float4(tf32_rest(v.x), tf32_rest(v.y), tf32_rest(v.z), tf32_rest(v.w));
        }
        const uint32_t ab = tm + C::A0 + (it & 1) * C::ACOLS + ((uint32_t)(32 * quad) << 16);
        // A rows: group g row m = tile 16 g + m / 8, its row m % 8; the row-8 group row m = tile m
        for (int g = 0; g <= ng; ++g) {
          const bool r8 = g == ng;
          const int gi = r8 ? NG : g;
          const int q = r8 ? m : 16 * g + (m >> 3);
          // tiles of this warp's 32 lanes: skip the stores when none of them is stored
          const int q_lo = r8 ? 32 * quad : 16 * g + 4 * quad;
          if (q_lo >= nb) continue;
          float h[32], r[32];
          if (q < nb) {
            if (r8) {
              const float4* src = reinterpret_cast<const float4*>(stg + C::O_R8 + q * 128);
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 v = src[j];
                h[4 * j] = v.x; h[4 * j + 1] = v.y; h[4 * j + 2] = v.z; h[4 * j + 3] = v.w;
              }
            } else {
              const int l = m & 7;
              const unsigned char* row = stg + C::O_A + q * 1024 + l * 128;
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 v = *reinterpret_cast<const float4*>(row + ((j ^ l) << 4));
                h[4 * j] = v.x; h[4 * j + 1] = v.y; h[4 * j + 2] = v.z; h[4 * j + 3] = v.w;
              }
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) h[j] = 0.f;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = tf32_rest(h[j]);
          tmem_st32(ab + 64 * gi, h);
          tmem_st32(ab + 64 * gi + 32, r);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        mbar_arrive(lo_ready(st));
      }
    }
    if (!ok) atomicOr(err, 2);
  } else {
    // ---------------- epilogue: 128 threads, one D row per thread ----------------
    const int quad = warp & 3;           // the TMEM lane quarter this warp may read
    const int m = 32 * quad + lane;
    int task = 0;
    for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x, ++task) {
      const int k0 = __ldg(row_ptr + a), nb = __ldg(row_ptr + a + 1) - k0;
      const int ng = (nb + 15) >> 4;
      const int db = task & 1;
      ok = mbar_wait(d_full(db), (task >> 1) & 1);
      if (!ok) break;
      tc_fence_after();
      const uint32_t d0 = tm + db * C::DCOLS + ((uint32_t)(32 * quad) << 16);
      for (int g = 0; g < ng; ++g) {
        float v[16];
        tmem_ld16(d0 + 16 * g, v);
        const int q = 16 * g + (m >> 3), l = m & 7;
        if (q < nb) {
          double* G = Gacc + (int64_t)(k0 + q) * 81 + l;
#pragma unroll
          for (int i = 0; i < 9; ++i) G[9 * i] += w * (double)v[i];
        }
      }
      if (quad * 32 < nb) {
        float v[16];
        tmem_ld16(d0 + 16 * NG, v);
        if (m < nb) {
          double* G = Gacc + (int64_t)(k0 + m) * 81 + 8;
#pragma unroll
          for (int i = 0; i < 9; ++i) G[9 * i] += w * (double)v[i];
        }
      }
      tc_fence_before();
      mbar_arrive(d_free(db));
    }
    if (!ok) atomicOr(err, 2);
  }
  // release TMEM once every warp is done with it
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tm, C::TCOLS);
  }
}

// Longest block row of the pattern (device reduction into *out).
__global__ void max_row_blocks(int n_atoms, const int32_t* __restrict__ row_ptr, int* __restrict__ out) {
  int m = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_atoms; a += gridDim.x * blockDim.x)
    m = max(m, row_ptr[a + 1] - row_ptr[a]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

static int tc_sddmm_occ(int dev) {
  static int occ[64] = {};
  int& o = occ[dev & 63];
  if (!o) {
    using C = TcSdCfg<2>;
    TBK_CUDA(cudaFuncSetAttribute(sddmm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int n = 0;
    TBK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sddmm_tc<2>, C::THREADS, C::SMEM));
    o = n > 0 ? n : -1;
  }
  return o;
}

int tc_sddmm_max_row(tbk_ctx* ctx, const HOp& op) {
  int* d = (int*)scratch(ctx, WS_FLAGS, 64) + 8;
  TBK_CUDA(cudaMemsetAsync(d, 0, sizeof(int), ctx->stream));
  max_row_blocks<<<std::max(1, std::min(ceil_div(op.n_atoms, 256), 1024)), 256, 0, ctx->stream>>>(op.n_atoms, op.row_ptr, d);
  post_launch(ctx, "max_row_blocks");
  int h = 0;
  TBK_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  return h;
}

bool tc_sddmm_eligible(tbk_ctx* ctx, const HOp& op, int s, int max_row) {
  return op.prec == TBK_MIXED && op.B == 9 && s % 32 == 0 && s >= 32 && max_row <= TcSdCfg<2>::TILES &&
         tc_sddmm_occ(ctx->device) > 0;
}

// Gacc += w sum_probes y[a rows] x[b rows]^T on every stored block (y, x: FP32 panels n_rows x s).
void launch_tc_sddmm(tbk_ctx* ctx, const HOp& op, const void* y, const void* x, int s, double w, double* Gacc,
                     int* err) {
  KernelTimerScope timer(ctx, TBK_KERNEL_WINDOW);
  using C = TcSdCfg<2>;
  CUtensorMap mX8, mX1, mY16;
  make_tmap_2d(&mX8, (const float*)x, op.n_rows, s, s, 8, 32, true);
  make_tmap_2d(&mX1, (const float*)x, op.n_rows, s, s, 1, 32, false);
  make_tmap_2d(&mY16, (const float*)y, op.n_rows, s, s, 16, 32, true);
  const int G = std::max(1, std::min(op.n_atoms, tc_sddmm_occ(ctx->device) * ctx->num_sms));
  sddmm_tc<2><<<G, C::THREADS, C::SMEM, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, mX8, mX1, mY16, s, w,
                                                        Gacc, err);
  post_launch(ctx, "sddmm_tc");
}

}  // namespace tbk
