// a5-a7: the fused block-SpMM Chebyshev recurrence with in-kernel probe generation and moment
// partial sums (Sec. II.B.1 Eq. poly_PQ with S = I; Sec. II.C.2 random approximation).
#include <algorithm>
#include <cmath>

#include "bulk.cuh"
#include "cheb.cuh"

namespace tbk {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ void ld16(const T* p, T* x) {
  if constexpr (sizeof(T) == 4) {
    float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else {
    double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x; x[1] = v.y;
  }
}
template <typename T>
__device__ __forceinline__ void ldg16(const T* p, T* x) {
  if constexpr (sizeof(T) == 4) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    x[0] = v.x; x[1] = v.y;
  }
}
template <typename T>
__device__ __forceinline__ void st16(T* p, const T* x) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  }
}

// ---- H^ in the padded kernel layout --------------------------------------------------------

template <typename T, int B>
__global__ void map_h_kernel(int n_atoms, const int32_t* __restrict__ row_ptr,
                             const int32_t* __restrict__ col, const double* __restrict__ H,
                             double shift, double inv_half_w, T* __restrict__ out, int* __restrict__ err) {
  constexpr int RS = Layout<T, B>::RS, BS = Layout<T, B>::BS;
  // blockDim (8, 16): the 8 lanes of a row are 8 consecutive lanes of one warp
  const int a = blockIdx.x * blockDim.y + threadIdx.y;
  if (a >= n_atoms) return;
  bool has_diag = false;
  for (int k = row_ptr[a] + threadIdx.x; k < row_ptr[a + 1]; k += blockDim.x) {
    const bool diag = col[k] == a;
    has_diag |= diag;
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < RS; ++j) {
        // stored element (major index i, minor index j): H^[i][j] row-major, H^[j][i] column-major
        const int r = Layout<T, B>::COLMAJOR ? j : i, c = Layout<T, B>::COLMAJOR ? i : j;
        double v = 0.0;
        if (j < B) {
          v = H[(int64_t)k * B * B + r * B + c];
          if (diag && r == c) v -= shift;
          v *= inv_half_w;
        }
        out[(int64_t)k * BS + i * RS + j] = (T)v;
      }
  }
  if (!__any_sync(0xFFu << (8 * (threadIdx.y & 3)), has_diag) && threadIdx.x == 0) atomicOr(err, ERR_NO_DIAGONAL);
}

HOp prepare_hop(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, int prec, Slot slot, int* err) {
  TBK_CHECK_ARG(H != nullptr, "H is NULL");
  TBK_CHECK_ARG(H->n_orb == 1 || H->n_orb == 9, "n_orb must be 1 or 9");
  TBK_CHECK_ARG(H->n_atoms >= 1 && H->nnzb >= H->n_atoms, "empty or inconsistent matrix");
  TBK_CHECK_ARG(H->row_ptr && H->col && H->val, "NULL matrix array");
  TBK_CHECK_ARG(H->nnzb < INT32_MAX, "nnzb must be below 2^31");
  TBK_CHECK_ARG(std::isfinite(emin) && std::isfinite(emax) && emax > emin, "need emax > emin");
  TBK_CHECK_ARG(prec == TBK_MIXED || prec == TBK_FP64, "unknown precision");
  HOp op;
  op.n_atoms = H->n_atoms;
  op.B = H->n_orb;
  op.prec = prec;
  op.nnzb = H->nnzb;
  op.n_rows = (int64_t)H->n_atoms * H->n_orb;
  op.row_ptr = H->row_ptr;
  op.col = H->col;
  const double shift = 0.5 * (emax + emin), inv = 2.0 / (emax - emin);
  dim3 blk(8, 16);
  const int grid = ceil_div(op.n_atoms, 16);
#define TBK_MAP(TT, BB)                                                                        \
  {                                                                                            \
    TT* out = (TT*)scratch(ctx, slot, sizeof(TT) * (size_t)op.nnzb * Layout<TT, BB>::BS);      \
    map_h_kernel<TT, BB><<<grid, blk, 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, H->val, \
                                                        shift, inv, out, err);                 \
    post_launch(ctx, "map_h_kernel");                                                          \
    op.hv = out;                                                                               \
  }
  if (prec == TBK_MIXED) {
    if (op.B == 9) TBK_MAP(float, 9) else TBK_MAP(float, 1)
  } else {
    if (op.B == 9) TBK_MAP(double, 9) else TBK_MAP(double, 1)
  }
#undef TBK_MAP
  return op;
}

// ---- the fused step --------------------------------------------------------------------------

constexpr int STEP_THREADS = 128;

template <typename T, int B, bool PROBE_IN>
__global__ void __launch_bounds__(STEP_THREADS)
cheb_step_kernel(const int n_atoms, const int32_t* __restrict__ row_ptr,
                 const int32_t* __restrict__ col, const T* __restrict__ hv,
                 const T* __restrict__ yin, const T* yprev, T* yout, const T alpha,
                 const T c_r, const uint64_t seed, const int s, const int direct,
                 double* __restrict__ partials) {
  constexpr int VEC = Vec16<T>::N;
  constexpr int RS = Layout<T, B>::RS, BS = Layout<T, B>::BS;
  // tasks: (row group, probe chunk) with chunk fastest; CTAs stride over tasks
  const int chunk_w = blockDim.x * VEC;
  const int n_chunks = (s + chunk_w - 1) / chunk_w;
  const int n_groups = (n_atoms + blockDim.y - 1) / blockDim.y;
  double sum0 = 0.0, sum1 = 0.0;
  for (int task = blockIdx.x; task < n_groups * n_chunks; task += gridDim.x) {
    const int grp = task / n_chunks, chunk = task - grp * n_chunks;
    const int p0 = chunk * chunk_w + threadIdx.x * VEC;
    const int a = grp * blockDim.y + threadIdx.y;
    if (p0 < s && a < n_atoms) {
      T acc[B][VEC];
#pragma unroll
      for (int i = 0; i < B; ++i)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[i][v] = T(0);
      const int k1 = __ldg(row_ptr + a + 1);
      for (int k = __ldg(row_ptr + a); k < k1; ++k) {
        const int b = __ldg(col + k);
        T x[B][VEC];
#pragma unroll
        for (int l = 0; l < B; ++l) {
          const int64_t row = (int64_t)b * B + l;
          if constexpr (PROBE_IN) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) x[l][v] = (T)tbk_probe_sign(seed, row, p0 + v);
          } else {
            ldg16(yin + row * s + p0, x[l]);
          }
        }
        const T* h = hv + (int64_t)k * BS;
        if constexpr (Layout<T, B>::COLMAJOR) {
          // column l of the block against row l of the tile; each acc[i] still sums l = 0..8
#pragma unroll
          for (int l = 0; l < B; ++l) {
            T hc[RS];
#pragma unroll
            for (int j = 0; j < RS; j += VEC) ldg16(h + l * RS + j, hc + j);
#pragma unroll
            for (int i = 0; i < B; ++i)
#pragma unroll
              for (int v = 0; v < VEC; ++v) acc[i][v] = fma(hc[i], x[l][v], acc[i][v]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < B; ++i) {
            T hr[RS];
            if constexpr (B == 1) {
              hr[0] = __ldg(h);
            } else {
#pragma unroll
              for (int j = 0; j < RS; j += VEC) ldg16(h + i * RS + j, hr + j);
            }
#pragma unroll
            for (int l = 0; l < B; ++l)
#pragma unroll
              for (int v = 0; v < VEC; ++v) acc[i][v] = fma(hr[l], x[l][v], acc[i][v]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < B; ++i) {
        const int64_t row = (int64_t)a * B + i;
        const int64_t off = row * s + p0;
        T yo[VEC], r[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) yo[v] = alpha * acc[i][v];
        if (c_r != T(0) || direct || PROBE_IN) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) r[v] = (T)tbk_probe_sign(seed, row, p0 + v);
        }
        if (c_r != T(0)) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) yo[v] = fma(c_r, r[v], yo[v]);
        }
        if (yprev) {
          T t[VEC];
          ld16(yprev + off, t);
#pragma unroll
          for (int v = 0; v < VEC; ++v) yo[v] -= t[v];
        }
        st16(yout + off, yo);
        if (partials) {
          T xin[VEC];
          if (direct || PROBE_IN) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) xin[v] = r[v];
          } else {
            ldg16(yin + off, xin);
          }
          T q0 = T(0), q1 = T(0);
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            q0 = fma(yo[v], xin[v], q0);
            q1 = fma(yo[v], yo[v], q1);
          }
          sum0 += (double)q0;
          sum1 += (double)q1;
        }
      }
    }
  }
  if (partials) {
    __shared__ double red[2][STEP_THREADS / 32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) {
      sum0 += __shfl_xor_sync(0xffffffffu, sum0, o);
      sum1 += __shfl_xor_sync(0xffffffffu, sum1, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = sum0;
      red[1][tid >> 5] = sum1;
    }
    __syncthreads();
    if (tid == 0) {
      double a0 = 0.0, a1 = 0.0;
      for (int w = 0; w < (nthreads + 31) / 32; ++w) {
        a0 += red[0][w];
        a1 += red[1][w];
      }
      partials[2 * blockIdx.x] = a0;
      partials[2 * blockIdx.x + 1] = a1;
    }
  }
}

// ---- TMA-fed step (FP32, 9x9 blocks, panel input) -------------------------------------------
//
// CTA = CW consumer warps + 1 producer warp.  A task is one block row a and a chunk of
// P = 128 CW probes (each consumer thread owns 4 consecutive probes).  The producer streams, for
// every neighbour block k = (a, b) of the task, the 9 x P tile of y_in rows 9b..9b+8 and the
// block H^_ab through a (D + 1)-stage shared-memory ring with cp.async.bulk copies completing on
// mbarriers, in stored order, then the row's own y_in tile a second time (when the moment sums
// need it) and the y_prev tile.  The consumers keep those last two stages until the epilogue
// has read them, so the epilogue reads nothing from global memory but the probe signs it
// regenerates (the second copy of the own tile is normally an L2 hit; holding the first one
// instead would stall the ring in the middle of the row).  Every wait is bounded: on expiry the
// CTA raises *err = 2 and leaves the loop, and the producer waits (bounded) for the copies it
// issued before returning.

template <int CW, int D>
struct BulkCfg {
  static constexpr int P = 128 * CW;                       // probes per task
  static constexpr int XB = 9 * P * 4;                      // tile bytes
  static constexpr int HB = Layout<float, 9>::BS * 4;       // 432 bytes
  static constexpr int SB = ((XB + HB + 127) / 128) * 128;  // stage bytes
  static constexpr int SMEM = (D + 1) * SB + 8 * (2 * D + 4);
  static constexpr int THREADS = 32 * (CW + 1);
};

template <int CW, int D>
__global__ void __launch_bounds__(32 * (CW + 1), 4)
cheb_step_bulk(const int n_atoms, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const float* __restrict__ hv, const float* __restrict__ yin, const float* yprev,
               float* yout, const float alpha, const float c_r, const uint64_t seed, const int s,
               const int direct, double* __restrict__ partials, int* __restrict__ err,
               const BatchRows batch, const int per_task, const int stall) {
  using C = BulkCfg<CW, D>;
  // every tile, the diagonal one included, streams through a ring of R = D + 1 stages (R >= 2:
  // the epilogue holds two)
  constexpr int R = D + 1;
  static_assert(R >= 2, "the epilogue holds two stages");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + R * C::SB);
  // bars: full[0..R), empty[R..2R)
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (R + i); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_chunks = s / C::P;
  const int n_tasks = n_atoms * n_chunks;
  const bool has_prev = yprev != nullptr;
  const bool own = partials != nullptr && !direct;  // the moment sums read the row's own y_in
  if (threadIdx.x == 0) {
    for (int i = 0; i < R; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), CW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == CW) {
    // ---------------- producer ----------------
    // (stall: a test of the bounded waits; nothing is copied, the consumers give up and report)
    if (lane == 0 && !stall) {
      int it = 0;
      bool ok = true;
      for (int task = blockIdx.x; task < n_tasks && ok; task += gridDim.x) {
        const int a = task / n_chunks, ch = task - a * n_chunks;
        const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
        const int nb = k1 - k0;
        const int nt = nb + (own ? 1 : 0) + (has_prev ? 1 : 0);
        for (int q = 0; q < nt && ok; ++q) {
          // tiles: the nb neighbour tiles with their blocks, then the row's own y_in tile again
          // (own: for the moment sums), then y_prev
          const bool is_nb = q < nb, is_prev = q == nt - 1 && has_prev;
          const int k = k0 + q;
          const int b = is_nb ? __ldg(col + k) : a;
          const int st = it % R;
          ok = mbar_wait(empty(st), ((it / R) & 1) ^ 1);
          if (!ok) break;
          const uint32_t dst = smem_u32(smem + st * C::SB), bar = full(st);
          ++it;
          const float* src = (is_prev ? yprev : yin) + (int64_t)9 * b * s + (int64_t)ch * C::P;
          mbar_expect_tx(bar, C::XB + (is_nb ? C::HB : 0));
          if (C::P == s) {
            bulk_g2s(dst, src, C::XB, bar);
          } else {
            for (int l = 0; l < 9; ++l) bulk_g2s(dst + l * C::P * 4, src + (int64_t)l * s, C::P * 4, bar);
          }
          if (is_nb) bulk_g2s(dst + C::XB, hv + (int64_t)k * Layout<float, 9>::BS, C::HB, bar);
        }
      }
      if (!ok) {
        atomicOr(err, 2);
        // wait (bounded) for copies still in flight into the ring before leaving
        for (int j = (it > R ? it - R : 0); j < it; ++j) mbar_wait(full(j % R), (j / R) & 1);
      }
    }
    return;
  }

  // ---------------- consumers ----------------
  // After the neighbour tiles come the row's own y_k tile (own) and the y_prev tile: both stay in
  // the ring (their stages are released after the epilogue, in order) and the epilogue reads them
  // from shared memory.
  double sum0 = 0.0, sum1 = 0.0;
  int it = 0;
  bool ok = true;
  uint32_t rdy = 0;  // stage it % R was found ready by the early test
  for (int task = blockIdx.x; task < n_tasks && ok; task += gridDim.x) {
    const int a = task / n_chunks, ch = task - a * n_chunks;
    const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
    const int nb = k1 - k0;
    const int pl = 4 * threadIdx.x;  // probe offset inside the chunk
    float2 acc[9][2];  // row i, probe v: acc_at(acc, i, v)
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
    int held = 0;  // stages held for the epilogue, starting at it - held
    for (int q = 0; q < nb; ++q) {
      const int st = it % R;
      if (!rdy) ok = mbar_wait(full(st), (it / R) & 1);
      ok = __all_sync(0xffffffffu, ok);  // one decision per warp: the warps meet at a barrier below
      if (!ok) break;
      rdy = mbar_test(full((it + 1) % R), ((it + 1) / R) & 1);
      const unsigned char* base = smem + st * C::SB;
      const float* X = reinterpret_cast<const float*>(base);
      const float* Hs = reinterpret_cast<const float*>(base + C::XB);
      spmm_tile_f2(X, Hs, C::P, pl, acc);
      __syncwarp();
      if (lane == 0) mbar_arrive(empty(st));
      ++it;
    }
    if (!ok) break;
    const float* Xown = nullptr;
    const float* Xprev = nullptr;
    if (own) {
      const int st = it % R;
      if (!rdy) ok = mbar_wait(full(st), (it / R) & 1);
      ok = __all_sync(0xffffffffu, ok);  // one decision per warp: the warps meet at a barrier below
      if (!ok) break;
      rdy = mbar_test(full((it + 1) % R), ((it + 1) / R) & 1);
      Xown = reinterpret_cast<const float*>(smem + st * C::SB);
      ++held;
      ++it;
    }
    if (has_prev) {
      const int st = it % R;
      if (!rdy) ok = mbar_wait(full(st), (it / R) & 1);
      ok = __all_sync(0xffffffffu, ok);  // one decision per warp: the warps meet at a barrier below
      if (!ok) break;
      rdy = mbar_test(full((it + 1) % R), ((it + 1) / R) & 1);
      Xprev = reinterpret_cast<const float*>(smem + st * C::SB);
      ++held;
      ++it;
    }
    // epilogue: y_out = alpha acc + c_r r - y_prev, moment partial sums
    const int p0 = ch * C::P + pl;
    uint64_t sd = seed;          // probe stream and row index within the cluster
    int64_t rloc = (int64_t)9 * a;
    if (batch.atom_cl) {
      const int cl = __ldg(batch.atom_cl + a);
      sd = __ldg(batch.seed + cl);
      rloc = (int64_t)9 * (a - __ldg(batch.atom0 + cl));
    }
    float cs0 = 0.f, cc0 = 0.f, cs1 = 0.f, cc1 = 0.f;  // the task's compensated partial sums
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int64_t row = (int64_t)9 * a + i;
      float yo[4], r[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) yo[v] = alpha * acc_at(acc, i, v);
      if (c_r != 0.f || direct) {
#pragma unroll
        for (int v = 0; v < 4; ++v) r[v] = tbk_probe_sign(sd, rloc + i, p0 + v);
      }
      if (c_r != 0.f) {
#pragma unroll
        for (int v = 0; v < 4; ++v) yo[v] = fmaf(c_r, r[v], yo[v]);
      }
      if (Xprev) {
        const float4 t = *reinterpret_cast<const float4*>(Xprev + i * C::P + pl);
        yo[0] -= t.x; yo[1] -= t.y; yo[2] -= t.z; yo[3] -= t.w;
      }
      *reinterpret_cast<float4*>(yout + row * s + p0) = make_float4(yo[0], yo[1], yo[2], yo[3]);
      if (partials) {
        float xin[4];
        if (direct) {
#pragma unroll
          for (int v = 0; v < 4; ++v) xin[v] = r[v];
        } else {
          // the row's own y_k from its held tile (Xown is set whenever these sums run: the global
          // read is never taken, but with it the kernel compiles to 96 registers without spills)
          const float4 t = Xown ? *reinterpret_cast<const float4*>(Xown + i * C::P + pl)
                                : __ldg(reinterpret_cast<const float4*>(yin + row * s + p0));
          xin[0] = t.x; xin[1] = t.y; xin[2] = t.z; xin[3] = t.w;
        }
        float q0 = 0.f, q1 = 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          q0 = fmaf(yo[v], xin[v], q0);
          q1 = fmaf(yo[v], yo[v], q1);
        }
        two_sum_acc(cs0, cc0, q0);
        two_sum_acc(cs1, cc1, q1);
      }
    }
    if (partials) {
      sum0 += (double)cs0 + (double)cc0;
      sum1 += (double)cs1 + (double)cc1;
    }
    // release the held stages in ring order
    __syncwarp();
    if (lane == 0)
      for (int h = held; h > 0; --h) mbar_arrive(empty((it - h) % R));
    if (per_task && partials) {
      // per (atom, warp) partial sums: no barrier between warps is needed
      for (int o = 16; o > 0; o >>= 1) {
        sum0 += __shfl_xor_sync(0xffffffffu, sum0, o);
        sum1 += __shfl_xor_sync(0xffffffffu, sum1, o);
      }
      if (lane == 0) {
        partials[2 * ((int64_t)a * CW + warp)] = sum0;
        partials[2 * ((int64_t)a * CW + warp) + 1] = sum1;
      }
      sum0 = sum1 = 0.0;
    }
  }
  if (!ok) atomicOr(err, 2);
  if (partials && !per_task) {
    __shared__ double red[2][8];
    for (int o = 16; o > 0; o >>= 1) {
      sum0 += __shfl_xor_sync(0xffffffffu, sum0, o);
      sum1 += __shfl_xor_sync(0xffffffffu, sum1, o);
    }
    if (lane == 0) {
      red[0][warp] = sum0;
      red[1][warp] = sum1;
    }
    // named barrier over the consumer warps only (the producer warp has returned)
    asm volatile("bar.sync 1, %0;" ::"r"(32 * CW) : "memory");
    if (threadIdx.x == 0) {
      double a0 = 0.0, a1 = 0.0;
      for (int w = 0; w < CW; ++w) {
        a0 += red[0][w];
        a1 += red[1][w];
      }
      partials[2 * blockIdx.x] = a0;
      partials[2 * blockIdx.x + 1] = a1;
    }
  }
}

// ---- self-fed step for 128-probe tasks ---------------------------------------------------------
//
// The same step as cheb_step_bulk<1, D> with one warp per CTA and no producer warp: lane 0 keeps
// R tiles in flight and, as soon as the warp has finished with a stage, refills it with the tile
// R positions ahead in the CTA's tile sequence (its tasks' neighbour tiles, then the y_prev tile
// of each task).  With 128 probes a task is quickly done, so a CTA that spends half its warps
// and registers on a producer limits how many consumers an SM holds.
template <int R>
struct SelfCfg {
  static constexpr int P = 128;
  static constexpr int XB = 9 * P * 4;
  static constexpr int HB = Layout<float, 9>::BS * 4;
  static constexpr int SB = ((XB + HB + 127) / 128) * 128;
  static constexpr int SMEM = R * SB + 8 * R;
};

template <int R>
__global__ void __launch_bounds__(32)
cheb_step_self(const int n_atoms, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const float* __restrict__ hv, const float* __restrict__ yin, const float* yprev,
               float* yout, const float alpha, const float c_r, const uint64_t seed, const int s,
               const int direct, double* __restrict__ partials, int* __restrict__ err,
               const BatchRows batch, const int per_task, const int stall) {
  using C = SelfCfg<R>;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t bar0 = smem_u32(smem + R * C::SB);
  auto full = [&](int i) { return bar0 + 8u * i; };
  const int lane = threadIdx.x;
  const int n_chunks = s / C::P;
  const int n_tasks = n_atoms * n_chunks;
  const bool has_prev = yprev != nullptr;
  if (lane == 0) {
    for (int i = 0; i < R; ++i) mbar_init(full(i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // producer cursor (lane 0): the next tile to issue, as (task, tile index within the task)
  int p_task = blockIdx.x, p_q = 0, p_nt = 0, p_k0 = 0, issued = 0;
  auto load_task = [&]() {  // tasks with no tile (an empty row, no y_{k-1}) are skipped
    for (; p_task < n_tasks; p_task += gridDim.x) {
      const int a = p_task / n_chunks;
      p_k0 = __ldg(row_ptr + a);
      p_nt = __ldg(row_ptr + a + 1) - p_k0 + (has_prev ? 1 : 0);
      if (p_nt > 0) break;
    }
  };
  auto issue_next = [&]() {
    if (stall || p_task >= n_tasks) return;
    const int a = p_task / n_chunks, ch = p_task - a * n_chunks;
    const bool is_prev = p_q == p_nt - (has_prev ? 1 : 0) && has_prev;
    const int b = is_prev ? a : __ldg(col + p_k0 + p_q);
    const int st = issued % R;
    const uint32_t dst = smem_u32(smem + st * C::SB), bar = full(st);
    const float* src = (is_prev ? yprev : yin) + (int64_t)9 * b * s + (int64_t)ch * C::P;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, C::XB + (is_prev ? 0 : C::HB));
    if (s == C::P) {
      bulk_g2s(dst, src, C::XB, bar);  // the 9 rows are contiguous
    } else {
      for (int l = 0; l < 9; ++l) bulk_g2s(dst + l * C::P * 4, src + (int64_t)l * s, C::P * 4, bar);
    }
    if (!is_prev) bulk_g2s(dst + C::XB, hv + (int64_t)(p_k0 + p_q) * Layout<float, 9>::BS, C::HB, bar);
    ++issued;
    if (++p_q == p_nt) {
      p_task += gridDim.x;
      p_q = 0;
      load_task();
    }
  };
  if (lane == 0) {
    load_task();
    for (int j = 0; j < R; ++j) issue_next();
  }
  __syncwarp();

  double sum0 = 0.0, sum1 = 0.0;
  int it = 0;
  bool ok = true;
  uint32_t rdy = 0;  // stage it % R was found ready by the early test
  const int pl = 4 * lane;
  auto consumed = [&]() {
    // the warp is done with stage it % R: refill it with the tile R positions ahead
    __syncwarp();
    if (lane == 0) issue_next();
    ++it;
  };
  for (int task = blockIdx.x; task < n_tasks && ok; task += gridDim.x) {
    const int a = task / n_chunks, ch = task - a * n_chunks;
    const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
    float2 acc[9][2];  // row i, probe v: acc_at_pp(acc, i, v)
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
    for (int q = 0; q < k1 - k0; ++q) {
      const int st = it % R;
      if (!rdy) {
        ok = mbar_wait(full(st), (it / R) & 1);
        if (!ok) break;
      }
      rdy = mbar_test(full((it + 1) % R), ((it + 1) / R) & 1);
      const unsigned char* base = smem + st * C::SB;
      spmm_tile_f2_pp(reinterpret_cast<const float*>(base), reinterpret_cast<const float*>(base + C::XB), C::P,
                      pl, acc);
      consumed();
    }
    if (!ok) break;
    float yp[9][4];
    if (has_prev) {
      const int st = it % R;
      if (!rdy) {
        ok = mbar_wait(full(st), (it / R) & 1);
        if (!ok) break;
      }
      rdy = mbar_test(full((it + 1) % R), ((it + 1) / R) & 1);
      const float* X = reinterpret_cast<const float*>(smem + st * C::SB);
#pragma unroll
      for (int l = 0; l < 9; ++l) {
        const float4 t = *reinterpret_cast<const float4*>(X + l * C::P + pl);
        yp[l][0] = t.x; yp[l][1] = t.y; yp[l][2] = t.z; yp[l][3] = t.w;
      }
      consumed();
    }
    const int p0 = ch * C::P + pl;
    uint64_t sd = seed;
    int64_t rloc = (int64_t)9 * a;
    if (batch.atom_cl) {
      const int cl = __ldg(batch.atom_cl + a);
      sd = __ldg(batch.seed + cl);
      rloc = (int64_t)9 * (a - __ldg(batch.atom0 + cl));
    }
    float cs0 = 0.f, cc0 = 0.f, cs1 = 0.f, cc1 = 0.f;  // the task's compensated partial sums
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int64_t row = (int64_t)9 * a + i;
      float yo[4], r[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) yo[v] = alpha * acc_at_pp(acc, i, v);
      if (c_r != 0.f || direct) {
#pragma unroll
        for (int v = 0; v < 4; ++v) r[v] = tbk_probe_sign(sd, rloc + i, p0 + v);
      }
      if (c_r != 0.f) {
#pragma unroll
        for (int v = 0; v < 4; ++v) yo[v] = fmaf(c_r, r[v], yo[v]);
      }
      if (has_prev) {
#pragma unroll
        for (int v = 0; v < 4; ++v) yo[v] -= yp[i][v];
      }
      *reinterpret_cast<float4*>(yout + row * s + p0) = make_float4(yo[0], yo[1], yo[2], yo[3]);
      if (partials) {
        float xin[4];
        if (direct) {
#pragma unroll
          for (int v = 0; v < 4; ++v) xin[v] = r[v];
        } else {
          const float4 t = __ldg(reinterpret_cast<const float4*>(yin + row * s + p0));
          xin[0] = t.x; xin[1] = t.y; xin[2] = t.z; xin[3] = t.w;
        }
        float q0 = 0.f, q1 = 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          q0 = fmaf(yo[v], xin[v], q0);
          q1 = fmaf(yo[v], yo[v], q1);
        }
        two_sum_acc(cs0, cc0, q0);
        two_sum_acc(cs1, cc1, q1);
      }
    }
    if (partials) {
      sum0 += (double)cs0 + (double)cc0;
      sum1 += (double)cs1 + (double)cc1;
    }
    if (per_task && partials) {
      for (int o = 16; o > 0; o >>= 1) {
        sum0 += __shfl_xor_sync(0xffffffffu, sum0, o);
        sum1 += __shfl_xor_sync(0xffffffffu, sum1, o);
      }
      if (lane == 0) {
        partials[2 * (int64_t)a] = sum0;
        partials[2 * (int64_t)a + 1] = sum1;
      }
      sum0 = sum1 = 0.0;
    }
  }
  if (!ok) {
    // let the copies in flight land before the CTA exits
    if (lane == 0) {
      atomicOr(err, 2);
      for (int j = it; j < issued; ++j) mbar_wait(full(j % R), (j / R) & 1);
    }
    return;
  }
  if (partials && !per_task) {
    for (int o = 16; o > 0; o >>= 1) {
      sum0 += __shfl_xor_sync(0xffffffffu, sum0, o);
      sum1 += __shfl_xor_sync(0xffffffffu, sum1, o);
    }
    if (lane == 0) {
      partials[2 * blockIdx.x] = sum0;
      partials[2 * blockIdx.x + 1] = sum1;
    }
  }
}

// ---- launch geometry ---------------------------------------------------------------------------

template <typename T, int B, bool P>
static int occupancy_simple() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cheb_step_kernel<T, B, P>, STEP_THREADS, 0);
  return n > 0 ? n : 1;
}

// two stages: 10 KB of ring per warp, so that the register limit (16 warps per SM), not shared
// memory (14 warps with three stages), sets the occupancy; measured 11 % faster on the batch
constexpr int SELF_R = 2;

static int occupancy_self() {
  using C = SelfCfg<SELF_R>;
  cudaFuncSetAttribute(cheb_step_self<SELF_R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cheb_step_self<SELF_R>, 32, C::SMEM);
  return n;
}

template <int CW, int D>
static int occupancy_bulk() {
  using C = BulkCfg<CW, D>;
  cudaFuncSetAttribute(cheb_step_bulk<CW, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cheb_step_bulk<CW, D>, C::THREADS, C::SMEM);
  return n;
}

// three ring stages and at most 102 registers: four CTAs of the 512-probe kernel per SM (16
// consumer warps), 2.8 % faster per step than three CTAs with four stages at 128 registers
constexpr int BULK_D = 2;

int bulk_consumer_warps(const HOp& op, int s);
// Consumer warps of the TMA-fed kernel for this operator and probe count (0 = not eligible).
static int bulk_warps(const HOp& op, int s) {
  if (op.prec != TBK_MIXED || op.B != 9 || s % 128 != 0) return 0;
  if (s % 512 == 0) return 4;
  if (s % 256 == 0) return 2;
  return 1;
}

int bulk_consumer_warps(const HOp& op, int s) { return bulk_warps(op, s); }

// Consumer warps (probe chunk 128 cw per task) of the TMA-fed step for this operator: the tuned
// choice when tbk_autotune measured this shape, else the widest chunk.  Per-task partial sums
// (batches) keep the default layout.
static int chosen_cw(const tbk_ctx* ctx, const HOp& op, int s, int per_task) {
  const int cw = bulk_warps(op, s);
  if (!cw || per_task) return cw;
  const tbk_ctx::Tuned* t = find_tuned(ctx, op.n_rows, op.nnzb, s);
  return t && t->cw >= 1 && t->cw <= cw && s % (128 * t->cw) == 0 ? t->cw : cw;
}

struct Occ {
  int simple = 0, bulk[5] = {0, 0, 0, 0, 0};
};

static Occ& occ_cache(int dev) {
  static Occ o[64];
  return o[dev < 0 || dev >= 64 ? 0 : dev];
}

template <typename T, int B>
static dim3 simple_block(int s) {
  constexpr int VEC = Vec16<T>::N;
  const int lanes_needed = (s + VEC - 1) / VEC;
  int lanes = 1;  // a power of two, so that every warp of the CTA is complete
  while (lanes < lanes_needed && lanes < STEP_THREADS) lanes <<= 1;
  return dim3(lanes, STEP_THREADS / lanes);
}

bool tc_eligible(const HOp& op, int s);
int tc_grid(tbk_ctx* ctx);
void launch_step_tc(tbk_ctx* ctx, const HOp& op, const StepArgs& a, int G);

int step_grid_ctas(tbk_ctx* ctx, const HOp& op, int s) {
  Occ& o = occ_cache(ctx->device);
  if (!o.simple) {
    int m = 1 << 30;
    m = std::min(m, std::min(occupancy_simple<float, 9, false>(), occupancy_simple<float, 9, true>()));
    m = std::min(m, std::min(occupancy_simple<float, 1, false>(), occupancy_simple<float, 1, true>()));
    m = std::min(m, std::min(occupancy_simple<double, 9, false>(), occupancy_simple<double, 9, true>()));
    m = std::min(m, std::min(occupancy_simple<double, 1, false>(), occupancy_simple<double, 1, true>()));
    o.simple = std::max(1, m);
    o.bulk[1] = occupancy_self();  // 128-probe tasks run on the self-fed kernel
    o.bulk[2] = occupancy_bulk<2, BULK_D>();
    o.bulk[4] = occupancy_bulk<4, BULK_D>();
  }
  // the TMA-fed kernel's occupancy sets the grid where it runs (the first step's plain kernel
  // then just takes more than one wave: every kernel loops over its tasks, none waits on another
  // CTA); the tensor-core step, when selected, runs on this same grid so that the per-CTA partial
  // sums line up
  const int cw = chosen_cw(ctx, op, s, 0);
  const int per_sm = cw && o.bulk[cw] > 0 ? o.bulk[cw] : o.simple;
  return std::max(1, per_sm * ctx->num_sms);
}

template <typename T, int B>
static void launch_simple(tbk_ctx* ctx, const HOp& op, const StepArgs& a, int G) {
  const dim3 blk = simple_block<T, B>(a.s);
  const T* hv = (const T*)op.hv;
  if (a.cur_is_probe)
    cheb_step_kernel<T, B, true><<<G, blk, 0, ctx->stream>>>(
        op.n_atoms, op.row_ptr, op.col, hv, (const T*)a.yin, (const T*)a.yprev, (T*)a.yout, (T)a.alpha,
        (T)a.c_r, a.seed, a.s, a.direct, a.partials);
  else
    cheb_step_kernel<T, B, false><<<G, blk, 0, ctx->stream>>>(
        op.n_atoms, op.row_ptr, op.col, hv, (const T*)a.yin, (const T*)a.yprev, (T*)a.yout, (T)a.alpha,
        (T)a.c_r, a.seed, a.s, a.direct, a.partials);
  post_launch(ctx, "cheb_step_kernel");
}

template <int CW>
static void launch_bulk(tbk_ctx* ctx, const HOp& op, const StepArgs& a, int G) {
  using C = BulkCfg<CW, BULK_D>;
  cheb_step_bulk<CW, BULK_D><<<G, C::THREADS, C::SMEM, ctx->stream>>>(
      op.n_atoms, op.row_ptr, op.col, (const float*)op.hv, (const float*)a.yin, (const float*)a.yprev,
      (float*)a.yout, (float)a.alpha, (float)a.c_r, a.seed, a.s, a.direct, a.partials, a.err,
      a.batch, a.per_task, ctx->stall_next_step);
  ctx->stall_next_step = 0;
  post_launch(ctx, "cheb_step_bulk");
}

static void launch_self(tbk_ctx* ctx, const HOp& op, const StepArgs& a, int G) {
  using C = SelfCfg<SELF_R>;
  cheb_step_self<SELF_R><<<G, 32, C::SMEM, ctx->stream>>>(
      op.n_atoms, op.row_ptr, op.col, (const float*)op.hv, (const float*)a.yin, (const float*)a.yprev,
      (float*)a.yout, (float)a.alpha, (float)a.c_r, a.seed, a.s, a.direct, a.partials, a.err,
      a.batch, a.per_task, ctx->stall_next_step);
  ctx->stall_next_step = 0;
  post_launch(ctx, "cheb_step_self");
}

void launch_step(tbk_ctx* ctx, const HOp& op, const StepArgs& a) {
  KernelTimerScope timer(ctx, TBK_KERNEL_STEP);
  const int G = step_grid_ctas(ctx, op, a.s);
  if (a.use_tc && !a.cur_is_probe && a.err && !a.force_simple && !a.batch.atom_cl && !a.per_task &&
      tc_eligible(op, a.s)) {
    launch_step_tc(ctx, op, a, G);
    return;
  }
  const int cw = chosen_cw(ctx, op, a.s, a.per_task);
  if (cw && !a.cur_is_probe && a.err && !a.force_simple && occ_cache(ctx->device).bulk[cw] > 0) {
    if (cw == 4) launch_bulk<4>(ctx, op, a, G);
    else if (cw == 2) launch_bulk<2>(ctx, op, a, G);
    else launch_self(ctx, op, a, G);
    return;
  }
  if (op.prec == TBK_MIXED) {
    if (op.B == 9) launch_simple<float, 9>(ctx, op, a, G); else launch_simple<float, 1>(ctx, op, a, G);
  } else {
    if (op.B == 9) launch_simple<double, 9>(ctx, op, a, G); else launch_simple<double, 1>(ctx, op, a, G);
  }
}

template <typename T>
__global__ void scaled_probe_kernel(int64_t n_rows, int s, double c, uint64_t seed, T* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows * s) return;
  const int64_t row = i / s;
  const int p = (int)(i - row * s);
  out[i] = (T)(c * (double)tbk_probe_sign(seed, row, p));
}

void launch_scaled_probe(tbk_ctx* ctx, const HOp& op, void* panel, double c, uint64_t seed, int s) {
  const int64_t n = op.n_rows * s;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (op.prec == TBK_MIXED)
    scaled_probe_kernel<float><<<grid, 256, 0, ctx->stream>>>(op.n_rows, s, c, seed, (float*)panel);
  else
    scaled_probe_kernel<double><<<grid, 256, 0, ctx->stream>>>(op.n_rows, s, c, seed, (double*)panel);
  post_launch(ctx, "scaled_probe_kernel");
}

// ---- moment reduction ------------------------------------------------------------------------

// sums[2 j + c] = sum over CTAs of partials[(j * nctas + cta) * 2 + c], Kahan-compensated per
// thread over a fixed strided set, then a fixed-order tree.
__global__ void reduce_partials(const double* __restrict__ partials, int nctas, double* __restrict__ sums) {
  const int j = blockIdx.x;
  __shared__ double sh[2][256];
  double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
  for (int t = threadIdx.x; t < nctas; t += blockDim.x) {
    const double* p = partials + ((int64_t)j * nctas + t) * 2;
    double y = p[0] - c0, u = s0 + y;
    c0 = (u - s0) - y;
    s0 = u;
    y = p[1] - c1;
    u = s1 + y;
    c1 = (u - s1) - y;
    s1 = u;
  }
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[2 * j] = sh[0][0];
    sums[2 * j + 1] = sh[1][0];
  }
}

// Moments from the per-step sums (step j = 1..K stored at index j - 1):
//   direct:   mu_j = S0_j / s
//   doubling: mu_1 = S0_1 / s, mu_2j = 2 S1_j / s - mu_0, mu_2j-1 = 2 S0_j / s - mu_1 (j >= 2)
// (C_m C_n = (C_{m+n} + C_{|m-n|})/2).  mu_0 = n_rows exactly for +-1 probes.  flag = 1 when a
// panel norm exceeds ||r|| (a spectrum outside [-1, 1]) or a sum is not finite.
__global__ void finish_moments(const double* __restrict__ sums, int K, int order, int s,
                               int64_t n_rows, int direct, double* __restrict__ mom,
                               int* __restrict__ flag) {
  const double mu0 = (double)n_rows;
  const double inv_s = 1.0 / s;
  const double mu1 = K >= 1 ? sums[0] * inv_s : 0.0;
  for (int k = threadIdx.x; k < order; k += blockDim.x) {
    double v;
    if (k == 0) v = mu0;
    else if (direct) v = sums[2 * (k - 1)] * inv_s;
    else if (k == 1) v = mu1;
    else if ((k & 1) == 0) v = 2.0 * sums[2 * (k / 2 - 1) + 1] * inv_s - mu0;
    else v = 2.0 * sums[2 * ((k + 1) / 2 - 1)] * inv_s - mu1;
    mom[k] = v;
  }
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    const double e = sums[2 * j + 1] * inv_s, o = sums[2 * j];
    if (!(e <= mu0 * (1.0 + 1e-3)) || !isfinite(o)) atomicOr(flag, 1);
  }
}

// ---- per-probe moments -------------------------------------------------------------------------
//
// After step j, PD_BLOCKS row blocks each sum, for every probe i, the products of the new panel
// y_j with itself and with y_{j-1} (the probe block r for j = 1) over their rows:
//   part[(rb s + i) 2 + 0] = sum_rows y_j y_j   (direct: sum_rows r y_j),
//   part[(rb s + i) 2 + 1] = sum_rows y_j y_{j-1}.
// FP32 panels: products are summed in FP32 over runs of 32 rows, then in FP64.  A second kernel
// adds the row blocks in a fixed order, so the result does not depend on timing.
constexpr int PD_BLOCKS = 304;

template <typename T>
__global__ void __launch_bounds__(256)
probe_dots(int64_t n_rows, int s, int64_t rows_per_block, const T* __restrict__ y,
           const T* __restrict__ x, uint64_t seed, int direct, double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n_rows ? r0 + rows_per_block : n_rows;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double d0 = 0.0, d1 = 0.0;
    for (int64_t b = r0; b < r1; b += 32) {
      const int64_t e = b + 32 < r1 ? b + 32 : r1;
      T t0 = T(0), t1 = T(0);
      for (int64_t row = b; row < e; ++row) {
        const T v = y[row * s + i];
        if (direct) {
          t0 += v * (T)tbk_probe_sign(seed, row, i);
        } else {
          const T u = x ? x[row * s + i] : (T)tbk_probe_sign(seed, row, i);
          t0 += v * v;
          t1 += v * u;
        }
      }
      d0 += (double)t0;
      d1 += (double)t1;
    }
    part[((int64_t)blockIdx.x * s + i) * 2] = d0;
    part[((int64_t)blockIdx.x * s + i) * 2 + 1] = d1;
  }
}

// dots[i 2 + c] = sum over the row blocks, in order, of part[(rb s + i) 2 + c]
__global__ void probe_dots_reduce(int nrb, int s, const double* __restrict__ part, double* __restrict__ dots) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s) return;
  double a = 0.0, b = 0.0;
  for (int rb = 0; rb < nrb; ++rb) {
    a += part[((int64_t)rb * s + i) * 2];
    b += part[((int64_t)rb * s + i) * 2 + 1];
  }
  dots[2 * i] = a;
  dots[2 * i + 1] = b;
}

// per_probe[k s + i] = r_i^T C_k(H^) r_i from the dots of steps j = 1 .. K (dots[((j-1) s + i) 2
// + c]): mu_0 = n_rows; direct: mu_k = (r . y_k); doubling: mu_1 = y_1 . r, mu_2k = 2 y_k . y_k -
// mu_0, mu_2k-1 = 2 y_k . y_{k-1} - mu_1 (the identities the summed moments use).
__global__ void probe_moments_finish(const double* __restrict__ dots, int K, int order, int s,
                                     int64_t n_rows, int direct, double* __restrict__ per_probe) {
  const int64_t n = (int64_t)order * s;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / s), i = (int)(t - (int64_t)k * s);
    auto d = [&](int j, int c) { return dots[((int64_t)(j - 1) * s + i) * 2 + c]; };
    const double mu0 = (double)n_rows;
    double v;
    if (k == 0) v = mu0;
    else if (direct) v = d(k, 0);
    else if (k == 1) v = d(1, 1);
    else if ((k & 1) == 0) v = 2.0 * d(k / 2, 0) - mu0;
    else v = 2.0 * d((k + 1) / 2, 1) - d(1, 1);
    per_probe[t] = v;
  }
}

// ---- building blocks that allocate nothing (for the static-scratch entry point) --------------

size_t mapped_h_bytes(const tbk_bsr* H, int prec) {
  const int bs = H->n_orb == 9 ? (prec == TBK_MIXED ? Layout<float, 9>::BS : Layout<double, 9>::BS) : 1;
  return (size_t)H->nnzb * bs * (prec == TBK_MIXED ? 4 : 8);
}

HOp prepare_hop_into(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, int prec, void* dst, int* err) {
  TBK_CHECK_ARG(H != nullptr, "H is NULL");
  TBK_CHECK_ARG(H->n_orb == 1 || H->n_orb == 9, "n_orb must be 1 or 9");
  TBK_CHECK_ARG(H->n_atoms >= 1 && H->nnzb >= H->n_atoms, "empty or inconsistent matrix");
  TBK_CHECK_ARG(H->row_ptr && H->col && H->val, "NULL matrix array");
  TBK_CHECK_ARG(H->nnzb < INT32_MAX, "nnzb must be below 2^31");
  TBK_CHECK_ARG(std::isfinite(emin) && std::isfinite(emax) && emax > emin, "need emax > emin");
  TBK_CHECK_ARG(prec == TBK_MIXED || prec == TBK_FP64, "unknown precision");
  HOp op;
  op.n_atoms = H->n_atoms;
  op.B = H->n_orb;
  op.prec = prec;
  op.nnzb = H->nnzb;
  op.n_rows = (int64_t)H->n_atoms * H->n_orb;
  op.row_ptr = H->row_ptr;
  op.col = H->col;
  op.hv = dst;
  const double shift = 0.5 * (emax + emin), inv = 2.0 / (emax - emin);
  const dim3 blk(8, 16);
  const int grid = ceil_div(op.n_atoms, 16);
  if (prec == TBK_MIXED) {
    if (op.B == 9)
      map_h_kernel<float, 9><<<grid, blk, 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, H->val, shift, inv, (float*)dst, err);
    else
      map_h_kernel<float, 1><<<grid, blk, 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, H->val, shift, inv, (float*)dst, err);
  } else {
    if (op.B == 9)
      map_h_kernel<double, 9><<<grid, blk, 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, H->val, shift, inv, (double*)dst, err);
    else
      map_h_kernel<double, 1><<<grid, blk, 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, H->val, shift, inv, (double*)dst, err);
  }
  post_launch(ctx, "map_h_kernel");
  return op;
}

void launch_moment_reduction(tbk_ctx* ctx, const double* partials, int nctas, int K, int order, int s,
                             int64_t n_rows, int direct, double* sums, double* moments, int* flag) {
  if (K >= 1) {
    reduce_partials<<<K, 256, 0, ctx->stream>>>(partials, nctas, sums);
    post_launch(ctx, "reduce_partials");
  }
  finish_moments<<<1, 256, 0, ctx->stream>>>(sums, K, order, s, n_rows, direct, moments, flag);
  post_launch(ctx, "finish_moments");
}

}  // namespace tbk

using namespace tbk;

namespace tbk {
// The moments sweep of tbk_chebyshev_moments; with per_probe, every step is followed by the
// per-probe dot products of its panels.  With probe_panel the probe block y_0 is that panel (the
// first step reads it as its source, the second as its y_{j-1}) and the moments divide by s_norm.
void moments_sweep(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, uint64_t probe_seed,
                   int32_t n_probes, int32_t order, int32_t flags, double* moments, double* per_probe,
                   const void* probe_panel, int s_norm) {
  TBK_CHECK_ARG(order >= 1, "order must be >= 1");
  TBK_CHECK_ARG(n_probes >= 4 && n_probes % 4 == 0, "n_probes must be a positive multiple of 4");
  TBK_CHECK_ARG((flags & ~(TBK_FP64 | TBK_MOMENTS_DIRECT | TBK_PLAIN_KERNEL | TBK_TENSOR_CORES)) == 0,
                "unknown flag");
  const int prec = (flags & TBK_FP64) ? TBK_FP64 : TBK_MIXED;
  const int direct = (flags & TBK_MOMENTS_DIRECT) ? 1 : 0;
  TBK_CHECK_ARG(!probe_panel || (!direct && !per_probe), "a stored probe block takes doubled moments only");
  const int nrm = probe_panel && s_norm > 0 ? s_norm : n_probes;
  int* flag = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  HOp op = prepare_hop(ctx, H, emin, emax, prec, WS_HHAT, flag);
  const int s = n_probes;
  const size_t esz = prec == TBK_MIXED ? 4 : 8;
  const size_t panel = (size_t)op.n_rows * s * esz;
  const int K = direct ? order - 1 : order / 2;   // steps: largest moment index 2K >= order - 1
  const int nctas = step_grid_ctas(ctx, op, s);
  double* partials = (double*)scratch(ctx, WS_PARTIALS, sizeof(double) * 2 * (size_t)std::max(1, K) * nctas);
  double* sums = (double*)scratch(ctx, WS_MISC, sizeof(double) * 2 * (size_t)std::max(1, K) + 64);
  void* A = K >= 1 ? scratch(ctx, WS_PANEL0, panel) : nullptr;
  void* Bp = K >= 2 ? scratch(ctx, WS_PANEL1, panel) : nullptr;
  // per-probe dots: row-block partials of one step, then K x s x 2 reduced dots
  const int64_t rpb = (op.n_rows + PD_BLOCKS - 1) / PD_BLOCKS;
  const int nrb = (int)((op.n_rows + rpb - 1) / rpb);
  double* pd_part = per_probe ? (double*)scratch(ctx, WS_PANEL2, sizeof(double) * 2 * (size_t)nrb * s) : nullptr;
  double* pd_dots = per_probe ? (double*)scratch(ctx, WS_SEGMENT, sizeof(double) * 2 * (size_t)std::max(1, K) * s)
                              : nullptr;
  void *cur = nullptr, *prev = nullptr;
  for (int j = 1; j <= K; ++j) {
    StepArgs a;
    a.seed = probe_seed;
    a.s = s;
    a.direct = direct;
    a.partials = partials + (size_t)(j - 1) * nctas * 2;
    a.err = flag;
    a.force_simple = (flags & TBK_PLAIN_KERNEL) ? 1 : 0;
    a.use_tc = (flags & TBK_TENSOR_CORES) ? 1 : 0;
    if (j == 1) {
      a.cur_is_probe = probe_panel ? 0 : 1;
      a.yin = probe_panel;
      a.alpha = 1.0;
      a.yout = A;
      cur = A;
    } else if (j == 2) {
      a.yin = A;
      a.alpha = 2.0;
      if (probe_panel) a.yprev = const_cast<void*>(probe_panel); else a.c_r = -1.0;
      a.yout = Bp;
      prev = A;
      cur = Bp;
    } else {
      a.yin = cur;
      a.yprev = prev;
      a.yout = prev;
      a.alpha = 2.0;
      std::swap(cur, prev);  // y_{j} now lives where y_{j-2} was
    }
    launch_step(ctx, op, a);
    if (per_probe) {
      // y_j at a.yout; y_{j-1} at a.yin (the probe block for j = 1)
      if (prec == TBK_MIXED)
        probe_dots<float><<<nrb, 256, 0, ctx->stream>>>(op.n_rows, s, rpb, (const float*)a.yout,
                                                        (const float*)a.yin, probe_seed, direct, pd_part);
      else
        probe_dots<double><<<nrb, 256, 0, ctx->stream>>>(op.n_rows, s, rpb, (const double*)a.yout,
                                                         (const double*)a.yin, probe_seed, direct, pd_part);
      post_launch(ctx, "probe_dots");
      probe_dots_reduce<<<ceil_div(s, 256), 256, 0, ctx->stream>>>(nrb, s, pd_part,
                                                                    pd_dots + (size_t)(j - 1) * 2 * s);
      post_launch(ctx, "probe_dots_reduce");
    }
  }
  if (K >= 1) {
    reduce_partials<<<K, 256, 0, ctx->stream>>>(partials, nctas, sums);
    post_launch(ctx, "reduce_partials");
  }
  finish_moments<<<1, 256, 0, ctx->stream>>>(sums, K, order, nrm, op.n_rows, direct, moments, flag);
  post_launch(ctx, "finish_moments");
  if (per_probe) {
    const int64_t n = (int64_t)order * s;
    probe_moments_finish<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, ctx->stream>>>(
        pd_dots, K, order, s, op.n_rows, direct, per_probe);
    post_launch(ctx, "probe_moments_finish");
  }
  int hflag = 0;
  TBK_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(hflag);
  if (hflag & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in the recurrence kernel expired");
  if (hflag)
    throw Error(TBK_ERR_SPECTRUM, "a Chebyshev panel grew beyond ||r||: the spectrum of H is not "
                                  "inside [emin, emax]");
}
}  // namespace tbk

extern "C" int tbk_chebyshev_moments(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax,
                                     uint64_t probe_seed, int32_t n_probes, int32_t order,
                                     int32_t flags, double* moments) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG(moments != nullptr, "moments is NULL");
  DeviceGuard dg(ctx);
  moments_sweep(ctx, H, emin, emax, probe_seed, n_probes, order, flags, moments, nullptr);
  TBK_API_END
}

extern "C" int tbk_chebyshev_probe_moments(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax,
                                           uint64_t probe_seed, int32_t n_probes, int32_t order,
                                           int32_t flags, double* moments, double* per_probe) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG(per_probe != nullptr, "per_probe is NULL");
  DeviceGuard dg(ctx);
  double* mom = moments;
  if (!mom) mom = (double*)scratch(ctx, WS_COEF, sizeof(double) * (size_t)std::max(1, order));
  moments_sweep(ctx, H, emin, emax, probe_seed, n_probes, order, flags, mom, per_probe);
  TBK_API_END
}
