// a9-a10: analytic derivative of the polynomial free-energy estimate (Sec. II.D, Eq.
// polynomial_response with S = I) and Hellmann-Feynman forces (Sec. II.A, Eq. observable).
//
// Omega^ = (1/s) sum_i r_i^T q(H^) r_i with q = sum_k c_k C_k, c_k = d_k beta_k[g].  Its gradient
// with respect to H, the bounds held fixed, is
//   G = (2/W)(1/s) sum_i sum_{j=0}^{p-2} y_ij x_ij^T,
//   y_j = C_j(H^) r,   x_j = (2 - delta_j0) b_{j+1},   b_m = sum_{k>=m} c_k U_{k-m}(H^) r,
// and b obeys the backward (Clenshaw) recurrence b_m = c_m r + 2 H^ b_{m+1} - b_{m+2}.  The
// backward sweep runs j = p-2 .. 0, adding y_j b_{j+1}^T on the block pattern and advancing b.
// The y_j are replayed from checkpoints kept every `seg` steps of a forward sweep; each segment
// is recomputed into a panel buffer just before its backward steps.
#include <algorithm>
#include <cmath>
#include <functional>
#include <type_traits>
#include <vector>

#include "bulk.cuh"
#include "cheb.cuh"
#include "model.cuh"
#include "sk.cuh"

namespace tbk {

void coefficients(tbk_ctx* ctx, int fn, int p, double emin, double emax, double mu, double kT,
                  int damping, double* out);

// Gacc[k] += w * sum_probes y[a rows] (x) b[b rows], one warp per stored block k = (a, b).
template <typename T, int B>
__global__ void __launch_bounds__(256)
sddmm_kernel(int n_atoms, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
             const T* __restrict__ y, uint64_t seed, int y_is_probe, const T* __restrict__ bp,
             int s, double w, double* __restrict__ Gacc, int64_t nnzb) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nnzb) return;
  const int k = (int)warp;
  // row of block k: binary search in row_ptr
  int lo = 0, hi = n_atoms;  // row_ptr[lo] <= k < row_ptr[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(row_ptr + mid) <= k) lo = mid; else hi = mid;
  }
  const int a = lo, b = __ldg(col + k);
  T acc[B * B];
#pragma unroll
  for (int e = 0; e < B * B; ++e) acc[e] = T(0);
  for (int p = lane; p < s; p += 32) {
    T yv[B], bv[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int64_t ra = (int64_t)a * B + i, rb = (int64_t)b * B + i;
      yv[i] = y_is_probe ? (T)tbk_probe_sign(seed, ra, p) : y[ra * s + p];
      bv[i] = bp[rb * s + p];
    }
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
      for (int l = 0; l < B; ++l) acc[i * B + l] = fma(yv[i], bv[l], acc[i * B + l]);
  }
#pragma unroll
  for (int e = 0; e < B * B; ++e) {
    double v = (double)acc[e];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == (e & 31)) Gacc[(int64_t)k * B * B + e] += w * v;
  }
}

// ---- fused Clenshaw step + sampled outer product (TMA-fed, FP32, 9x9 blocks, P = s) ------------
//
// For one backward index j and every block row a (one CTA task covers all s probes):
//   b_j[a]   = 2 sum_b H^_ab b_{j+1}[b] + c_j r[a] - b_{j+2}[a]          (skipped when bout = 0)
//   Gacc_ab += w sum_probes y_j[a] b_{j+1}[b]^T   for every neighbour block (a, b)
// The neighbour tiles b_{j+1}[b] and blocks H^_ab stream through a D-stage ring as in the
// forward step; the own-row tile y_j[a] (or the probe block when j = 0) is staged once per task.
// The 9x9 outer product of each tile is split into three groups of 3 rows, each taken by one
// consumer warp (in turn, so the load stays even): its 32 lanes cover interleaved 4-probe
// groups, and a butterfly reduce-scatter over the lanes leaves one entry per lane, added to the
// FP64 accumulator (one CTA owns each block, so each entry has one writer per launch).

template <int CW, bool SD = true>
struct SdCfg {
  static constexpr int D = SD ? 2 : 3;  // SD: 2 stages keep three CTAs within shared memory
  static constexpr int P = 128 * CW;
  static constexpr int XB = 9 * P * 4;
  static constexpr int HB = Layout<float, 9>::BS * 4;
  static constexpr int SB = ((XB + HB + 127) / 128) * 128;
  static constexpr int YB = SD ? ((XB + 127) / 128) * 128 : 0;
  static constexpr int SMEM = (D + 1) * SB + YB + 8 * (2 * D + 6);
  static constexpr int THREADS = 32 * (CW + 1);
};

// 32 lane partials per entry -> lane e holds the lane-sum of entry e.
__device__ __forceinline__ void butterfly32(float (&v)[32], int lane) {
#pragma unroll
  for (int off = 16, n = 32; off >= 1; off >>= 1, n >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < n / 2; ++k) {
      const float send = up ? v[k] : v[k + n / 2];
      const float keep = up ? v[k + n / 2] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
}

// Rows 3g .. 3g+2 of the 9x9 outer product sum_p Y[i][p] X[l][p] over all P probes (lanes cover
// interleaved 4-probe groups): 27 entries, reduced over the lanes by one butterfly and added to
// the FP64 accumulator (one lane per entry).
template <int P>
__device__ __forceinline__ void sddmm_rows3(int g, const float* Y, const float* X, bool y_probe,
                                            uint64_t seed, int64_t rloc, int lane, int64_t k,
                                            double w, double* __restrict__ Gacc) {
  // partial sums of entry (i - 3g) * 9 + l over this lane's probes; scalar accumulators keep the
  // kernel at 128 registers, so that three CTAs fit per SM
  float v1[27];
#pragma unroll
  for (int e = 0; e < 27; ++e) v1[e] = 0.f;
#pragma unroll 1
  for (int m = 0; m < P / 128; ++m) {
    const int pb = 4 * (lane + 32 * m);
    float yv[3][4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (y_probe) {
#pragma unroll
        for (int t = 0; t < 4; ++t) yv[i][t] = tbk_probe_sign(seed, rloc + 3 * g + i, pb + t);
      } else {
        const float4 u = *reinterpret_cast<const float4*>(Y + (3 * g + i) * P + pb);
        yv[i][0] = u.x; yv[i][1] = u.y; yv[i][2] = u.z; yv[i][3] = u.w;
      }
    }
#pragma unroll
    for (int l = 0; l < 9; ++l) {
      const float4 u = *reinterpret_cast<const float4*>(X + l * P + pb);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float t = v1[i * 9 + l];
        t = fmaf(yv[i][0], u.x, t); t = fmaf(yv[i][1], u.y, t);
        t = fmaf(yv[i][2], u.z, t); t = fmaf(yv[i][3], u.w, t);
        v1[i * 9 + l] = t;
      }
    }
  }
  float v[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) v[e] = e < 27 ? v1[e] : 0.f;
  butterfly32(v, lane);
  if (lane < 27)
    // fire-and-forget reduction: one writer per entry and launch, so the sum stays deterministic
    atomicAdd(Gacc + k * 81 + 27 * g + lane, w * (double)v[0]);
}

// SD = false: the Clenshaw step alone (the outer products are left to sddmm_window_g); the own-row
// tile y_j then streams through the ring like the other source terms.  SD = true: three CTAs of
// four consumer warps per SM, whose interleaving hides the latency of the outer product's
// reductions.
template <int CW, bool SD>
__global__ void __launch_bounds__(32 * (CW + 1), SD || CW == 4 ? 3 : 1)
clenshaw_sddmm_bulk(const int n_atoms, const int32_t* __restrict__ row_ptr,
                    const int32_t* __restrict__ col, const float* __restrict__ hv,
                    const float* __restrict__ bin, const float* bprev, float* bout,
                    const float* __restrict__ ypan, const float4 cf, const uint64_t seed,
                    const int s, const double w, double* __restrict__ Gacc, int* __restrict__ err,
                    const BatchRows batch, const float4* __restrict__ cf_cl,
                    const float* __restrict__ ym1, const float* __restrict__ yp1, const int stall) {
  using C = SdCfg<CW, SD>;
  // every tile, the diagonal one included, streams through a ring of R = D + 1 stages
  constexpr int R = C::D + 1;
  extern __shared__ __align__(128) unsigned char smem[];
  float* Ys = reinterpret_cast<float*>(smem + R * C::SB);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + R * C::SB + C::YB);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (R + i); };
  const uint32_t y_full = bar0 + 8u * (2 * R), y_empty = bar0 + 8u * (2 * R + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool has_prev = bprev != nullptr, has_out = bout != nullptr;
  // y_tile: the own-row tile y_j is staged once per task for the outer products
  const bool y_probe = ypan == nullptr, y_tile = SD && !y_probe;
  if (threadIdx.x == 0) {
    for (int i = 0; i < R; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), CW);
    }
    mbar_init(y_full, 1);
    mbar_init(y_empty, CW);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // own-row tiles streamed after the neighbour tiles, with the component of the (per-cluster)
  // coefficient vector that scales them: b_prev (-1), y_k (.y, when it is not staged), y_{k-1}
  // (.z), y_{k+1} (.w).  With per-cluster coefficients a tile is streamed whenever it is given.
  enum { X_PREV = 0, X_Y = 1, X_YM1 = 2, X_YP1 = 3 };
  const float* extra_src[4];
  int extra_kind[4];
  int n_extra = 0;
  if (has_out) {
    const bool any = cf_cl != nullptr;
    if (has_prev) { extra_src[n_extra] = bprev; extra_kind[n_extra++] = X_PREV; }
    if (!SD && ypan && (any || cf.y != 0.f)) { extra_src[n_extra] = ypan; extra_kind[n_extra++] = X_Y; }
    if (ym1 && (any || cf.z != 0.f)) { extra_src[n_extra] = ym1; extra_kind[n_extra++] = X_YM1; }
    if (yp1 && (any || cf.w != 0.f)) { extra_src[n_extra] = yp1; extra_kind[n_extra++] = X_YP1; }
  }
  if (warp == CW) {
    // (stall: a test of the bounded waits; nothing is copied, the consumers give up and report)
    if (lane == 0 && !stall) {
      int it = 0, y_it = 0;
      bool ok = true;
      for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x) {
        const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
        if (y_tile) {
          ok = mbar_wait(y_empty, (y_it & 1) ^ 1);
          if (!ok) break;
          mbar_expect_tx(y_full, C::XB);
          bulk_g2s(smem_u32(Ys), ypan + (int64_t)9 * a * s, C::XB, y_full);
          ++y_it;
        }
        // after the neighbour tiles: the own-row tiles of b_prev, y_{k-1} and y_{k+1} (when used)
        const int nb = k1 - k0;
        const int nt = nb + n_extra;
        for (int q = 0; q < nt && ok; ++q) {
          const bool is_prev = q >= nb;
          const float* extra = is_prev ? extra_src[q - nb] : nullptr;
          const int b = is_prev ? a : __ldg(col + k0 + q);
          const int st = it % R;
          ok = mbar_wait(empty(st), ((it / R) & 1) ^ 1);
          if (!ok) break;
          const uint32_t dst = smem_u32(smem + st * C::SB), bar = full(st);
          ++it;
          const float* src = (is_prev ? extra : bin) + (int64_t)9 * b * s;
          mbar_expect_tx(bar, C::XB + (is_prev ? 0 : C::HB));
          bulk_g2s(dst, src, C::XB, bar);
          if (!is_prev) bulk_g2s(dst + C::XB, hv + (int64_t)(k0 + q) * Layout<float, 9>::BS, C::HB, bar);
        }
      }
      if (!ok) {
        // let the copies in flight land before the CTA exits
        atomicOr(err, 2);
        for (int j = (it > R ? it - R : 0); j < it; ++j) mbar_wait(full(j % R), (j / R) & 1);
        if (y_tile && y_it > 0) mbar_wait(y_full, (y_it - 1) & 1);
      }
    }
    return;
  }

  int it = 0, y_it = 0;
  bool ok = true;
  uint32_t rdy = 0;  // stage it % R was found ready by the early test
  const int pl = 4 * threadIdx.x;
  for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x) {
    const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
    // probe stream and cluster-local row of this atom; per-cluster coefficient in batches
    uint64_t sd = seed;
    int64_t rloc = (int64_t)9 * a;
    float4 cfa = cf;  // (probe, own y, y_{k-1}, y_{k+1}) coefficients of the source term
    if (batch.atom_cl) {
      const int cl = __ldg(batch.atom_cl + a);
      sd = __ldg(batch.seed + cl);
      rloc = (int64_t)9 * (a - __ldg(batch.atom0 + cl));
      if (cf_cl) cfa = cf_cl[cl];
    }
    if (y_tile) {
      ok = mbar_wait(y_full, y_it & 1);
      if (!ok) break;
    }
    float2 acc[9][2];  // row i, probe v: acc_at(acc, i, v)
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
      const float* X = reinterpret_cast<const float*>(base);
      if (has_out) spmm_tile_f2(X, reinterpret_cast<const float*>(base + C::XB), C::P, pl, acc);
      if constexpr (SD) {
        // row group g of this tile goes to warp (q + g + 1) mod CW: with 4 warps one warp rests
        // per tile, in turn
        for (int g = 0; g < 3; ++g)
          if ((q + g + 1) % CW == warp)
            sddmm_rows3<C::P>(g, Ys, X, y_probe, sd, rloc, lane, (int64_t)(k0 + q), w, Gacc);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty(st));
      ++it;
    }
    if (!ok) break;
    if (!has_out) {
      if (y_tile) {
        __syncwarp();
        if (lane == 0) mbar_arrive(y_empty);
        ++y_it;
      }
      continue;
    }
    // y_out = 2 H^ b_in + cf.x r + cf.y y_own + (own-row tiles: -b_prev + cf.z y_{k-1} + cf.w y_{k+1})
    float yo[9][4];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
      for (int v = 0; v < 4; ++v) yo[i][v] = 2.f * acc_at(acc, i, v);
    if (cfa.x != 0.f) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int v = 0; v < 4; ++v) yo[i][v] = fmaf(cfa.x, tbk_probe_sign(sd, rloc + i, pl + v), yo[i][v]);
    }
    if (y_tile && cfa.y != 0.f) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float4 t = *reinterpret_cast<const float4*>(Ys + i * C::P + pl);
        yo[i][0] = fmaf(cfa.y, t.x, yo[i][0]); yo[i][1] = fmaf(cfa.y, t.y, yo[i][1]);
        yo[i][2] = fmaf(cfa.y, t.z, yo[i][2]); yo[i][3] = fmaf(cfa.y, t.w, yo[i][3]);
      }
    }
    for (int e = 0; e < n_extra; ++e) {
      const int st = it % R;
      if (!rdy) {
        ok = mbar_wait(full(st), (it / R) & 1);
        if (!ok) break;
      }
      rdy = mbar_test(full((it + 1) % R), ((it + 1) / R) & 1);
      const float* X = reinterpret_cast<const float*>(smem + st * C::SB);
      const int kd = extra_kind[e];
      const float ce = kd == X_PREV ? -1.f : (kd == X_Y ? cfa.y : (kd == X_YM1 ? cfa.z : cfa.w));
      if (ce != 0.f) {  // a zero coefficient skips the tile (its rows may never have been formed)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const float4 t = *reinterpret_cast<const float4*>(X + i * C::P + pl);
          yo[i][0] = fmaf(ce, t.x, yo[i][0]); yo[i][1] = fmaf(ce, t.y, yo[i][1]);
          yo[i][2] = fmaf(ce, t.z, yo[i][2]); yo[i][3] = fmaf(ce, t.w, yo[i][3]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty(st));
      ++it;
    }
    if (!ok) break;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int64_t row = (int64_t)9 * a + i;
      *reinterpret_cast<float4*>(bout + row * s + pl) = make_float4(yo[i][0], yo[i][1], yo[i][2], yo[i][3]);
    }
    if (y_tile) {
      __syncwarp();
      if (lane == 0) mbar_arrive(y_empty);
      ++y_it;
    }
  }
  if (!ok) atomicOr(err, 2);
}

// ---- outer products of a window of backward steps (TMA-fed, FP32, 9x9 blocks) ------------------
//
// Gacc_ab += w sum_{t < nw} sum_probes y_{k_t}[a] ybar_{k_t + 1}[b]^T for every stored block (a, b).
// Summing nw steps before the cross-lane reduction spreads its cost over nw block products.

constexpr int SDW = 4;  // steps per window

struct WindowPanels {
  const float* y[SDW];  // y_{k_t} panels (n_rows x s); y[0] = NULL: the probe block
  const float* x[SDW];  // ybar_{k_t + 1} panels
};

// One CTA task is one block row a.  Consumer warp (g, c) takes rows 3g .. 3g+2 of the block (27
// entries, one scalar sum each per lane) over probe chunk c (128 probes, 4 per lane), for g < 3
// and c < NC = P / 128.  The producer warp stages the window's own-row tiles y_{k_t}[a] once per
// block row (or writes the probe block when y[0] is NULL, nw = 1) and streams the neighbour tiles
// ybar_{k_t+1}[b] of every block through a D-stage ring read by all 3 NC warps.  Per block, each
// warp reduces its 27 sums over the lanes (one butterfly for all the window's steps) and warp
// (g, 0) adds the NC chunk partials in a fixed order and writes the 27 totals to the FP64
// accumulator: one writer per entry, so the result does not depend on timing.  (One warp holding
// all 81 entries, the earlier form, kept 6 consumer warps per SM at 128 probes: 2.80 ms per window
// on the 64-cluster batch against 2.02 ms.)
template <int NC>
struct WinGCfg {
  static constexpr int P = 128 * NC;
  static constexpr int NWARP = 3 * NC;  // consumer warps
  static constexpr int THREADS = 32 * (NWARP + 1);
  static constexpr int XB = 9 * P * 4;
  static constexpr int D = NC == 4 ? 6 : (NC == 1 ? 4 : 8);
  static constexpr int RED = 2 * 3 * NC * 32 * 4;  // [2 buffers][3 groups][NC chunks][32 lanes]
  static constexpr int NBAR = 2 * D + 2 + 12;
  static constexpr int SMEM = (SDW + D) * XB + RED + 8 * NBAR;
};

template <int NC>
__global__ void __launch_bounds__(32 * (3 * NC + 1), NC == 1 ? 5 : 1)
sddmm_window_g(const int n_atoms, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const WindowPanels wp, const int nw, const uint64_t seed, const int s, const double w,
               double* __restrict__ Gacc, int* __restrict__ err, const BatchRows batch,
               const int32_t* __restrict__ kcl, const int k_lo) {
  using C = WinGCfg<NC>;
  constexpr int D = C::D, P = C::P, NWARP = C::NWARP;
  extern __shared__ __align__(128) unsigned char smem[];
  float* Yw = reinterpret_cast<float*>(smem);                       // SDW own-row tiles
  unsigned char* ring = smem + SDW * C::XB;                          // D neighbour tiles
  float* red = reinterpret_cast<float*>(smem + (SDW + D) * C::XB);   // [2][3][NC][32]
  const uint32_t bar0 = smem_u32(smem + (SDW + D) * C::XB + C::RED);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (D + i); };
  const uint32_t y_full = bar0 + 8u * (2 * D), y_empty = bar0 + 8u * (2 * D + 1);
  auto red_full = [&](int b, int g) { return bar0 + 8u * (2 * D + 2 + 3 * b + g); };
  auto red_empty = [&](int b, int g) { return bar0 + 8u * (2 * D + 8 + 3 * b + g); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool probe = wp.y[0] == nullptr;
  if (threadIdx.x == 0) {
    for (int i = 0; i < D; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), NWARP);
    }
    mbar_init(y_full, 1);
    mbar_init(y_empty, NWARP);
    for (int b = 0; b < 2; ++b)
      for (int g = 0; g < 3; ++g) {
        mbar_init(red_full(b, g), NC);
        mbar_init(red_empty(b, g), 1);
      }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto atom_window = [&](int a, int& nwa, uint64_t& sd, int64_t& rloc) {
    nwa = nw;
    sd = seed;
    rloc = (int64_t)9 * a;
    if (batch.atom_cl) {
      const int cl = __ldg(batch.atom_cl + a);
      sd = __ldg(batch.seed + cl);
      rloc = (int64_t)9 * (a - __ldg(batch.atom0 + cl));
      if (kcl) nwa = min(nw, max(0, __ldg(kcl + cl) - k_lo));
    }
  };

  if (warp == NWARP) {
    // producer warp: lane 0 issues the copies; in the probe case all lanes write the probe block
    int it = 0, y_it = 0;
    bool ok = true;
    for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x) {
      int nwa;
      uint64_t sd;
      int64_t rloc;
      atom_window(a, nwa, sd, rloc);
      if (nwa == 0) continue;
      if (lane == 0) ok = mbar_wait(y_empty, (y_it & 1) ^ 1);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      if (probe) {
        for (int e = lane; e < 9 * P; e += 32) {
          const int i = e / P, pr = e - i * P;
          Yw[e] = tbk_probe_sign(sd, rloc + i, pr);
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) mbar_arrive(y_full);
      } else if (lane == 0) {
        mbar_expect_tx(y_full, nwa * C::XB);
        for (int t = 0; t < nwa; ++t)
          bulk_g2s(smem_u32(Yw + t * 9 * P), wp.y[t] + (int64_t)9 * a * s, C::XB, y_full);
      }
      ++y_it;
      if (lane == 0) {
        const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
        for (int q = k0; q < k1 && ok; ++q) {
          const int b = __ldg(col + q);
          for (int t = 0; t < nwa && ok; ++t) {
            const int st = it % D;
            ok = mbar_wait(empty(st), ((it / D) & 1) ^ 1);
            if (!ok) break;
            mbar_expect_tx(full(st), C::XB);
            bulk_g2s(smem_u32(ring + st * C::XB), wp.x[t] + (int64_t)9 * b * s, C::XB, full(st));
            ++it;
          }
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
    }
    if (!ok && lane == 0) {
      atomicOr(err, 2);
      for (int j = (it > D ? it - D : 0); j < it; ++j) mbar_wait(full(j % D), (j / D) & 1);
      if (y_it > 0 && !probe) mbar_wait(y_full, (y_it - 1) & 1);
    }
    return;
  }

  const int g = warp / NC, c = warp - g * NC;
  const int pl = 128 * c + 4 * lane;  // this lane's 4 probes
  int it = 0, y_it = 0, r_it = 0;
  bool ok = true;
  for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x) {
    int nwa;
    uint64_t sd;
    int64_t rloc;
    atom_window(a, nwa, sd, rloc);
    if (nwa == 0) continue;
    const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
    ok = mbar_wait(y_full, y_it & 1);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) break;
    for (int q = k0; q < k1; ++q) {
      float acc[27];
      // step t of the window for this block (first: the sums start here); false: a wait expired
      auto tile = [&](int t, auto first) {
        const int st = it % D;
        ok = mbar_wait(full(st), (it / D) & 1);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) return false;
        const float* X = reinterpret_cast<const float*>(ring + st * C::XB);
        const float* Y = Yw + t * 9 * P + 3 * g * P;
        float4 yv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) yv[i] = *reinterpret_cast<const float4*>(Y + i * P + pl);
#pragma unroll
        for (int l = 0; l < 9; ++l) {
          const float4 xv = *reinterpret_cast<const float4*>(X + l * P + pl);
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            float u = decltype(first)::value ? yv[i].x * xv.x : fmaf(yv[i].x, xv.x, acc[i * 9 + l]);
            u = fmaf(yv[i].y, xv.y, u);
            u = fmaf(yv[i].z, xv.z, u); u = fmaf(yv[i].w, xv.w, u);
            acc[i * 9 + l] = u;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty(st));
        ++it;
        return true;
      };
      if (nwa == SDW) {  // a full window: the step loop unrolled
        if (tile(0, std::true_type())) {
#pragma unroll
          for (int t = 1; t < SDW; ++t)
            if (!tile(t, std::false_type())) break;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 27; ++e) acc[e] = 0.f;
        for (int t = 0; t < nwa; ++t)
          if (!tile(t, std::false_type())) break;
      }
      if (!ok) break;
      // lanes -> lane e holds this chunk's sum of entry 27 g + e
      float v[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) v[e] = e < 27 ? acc[e] : 0.f;
      butterfly32(v, lane);
      if constexpr (NC == 1) {
        // one chunk: this warp alone holds the totals of its 27 entries (one writer per entry)
        if (lane < 27) atomicAdd(Gacc + (int64_t)q * 81 + 27 * g + lane, w * (double)v[0]);
        continue;
      }
      const int rb = r_it & 1, use = r_it >> 1;
      if (use > 0) {
        ok = mbar_wait(red_empty(rb, g), (use - 1) & 1);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
      }
      float* R = red + (rb * 3 + g) * NC * 32;
      R[c * 32 + lane] = v[0];
      __syncwarp();
      if (lane == 0) mbar_arrive(red_full(rb, g));
      if (c == 0) {
        // fixed-order sum over the chunks, one writer per entry
        ok = mbar_wait(red_full(rb, g), use & 1);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        if (lane < 27) {
          float tsum = R[lane];
#pragma unroll
          for (int cc = 1; cc < NC; ++cc) tsum += R[cc * 32 + lane];
          atomicAdd(Gacc + (int64_t)q * 81 + 27 * g + lane, w * (double)tsum);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(red_empty(rb, g));
      }
      ++r_it;
    }
    if (!ok) break;
    __syncwarp();
    if (lane == 0) mbar_arrive(y_empty);
    ++y_it;
  }
  if (!ok) atomicOr(err, 2);
}

// ---- self-fed adjoint step for 128 probes (windowed schedule) ---------------------------------
//
// clenshaw_sddmm_bulk<1, false> with one warp per CTA and no producer warp: lane 0 keeps R tiles
// in flight (each row's neighbour tiles with their blocks, then its own-row source tiles) and
// refills a stage as soon as the warp is done with it, so more consumer warps fit per SM.
template <int R>
struct ClenSelfCfg {
  static constexpr int P = 128;
  static constexpr int XB = 9 * P * 4;
  static constexpr int HB = Layout<float, 9>::BS * 4;
  static constexpr int SB = ((XB + HB + 127) / 128) * 128;
  static constexpr int SMEM = R * SB + 8 * R;
};

template <int R>
__global__ void __launch_bounds__(32)
clenshaw_self(const int n_atoms, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
              const float* __restrict__ hv, const float* __restrict__ bin, const float* bprev, float* bout,
              const float* __restrict__ ypan, const float4 cf, const uint64_t seed, const int s,
              int* __restrict__ err, const BatchRows batch, const float4* __restrict__ cf_cl,
              const float* __restrict__ ym1, const float* __restrict__ yp1) {
  using C = ClenSelfCfg<R>;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t bar0 = smem_u32(smem + R * C::SB);
  auto full = [&](int i) { return bar0 + 8u * i; };
  const int lane = threadIdx.x;
  enum { X_PREV = 0, X_Y = 1, X_YM1 = 2, X_YP1 = 3 };
  const float* extra_src[4];
  int extra_kind[4];
  int n_extra = 0;
  {
    const bool any = cf_cl != nullptr;
    if (bprev) { extra_src[n_extra] = bprev; extra_kind[n_extra++] = X_PREV; }
    if (ypan && (any || cf.y != 0.f)) { extra_src[n_extra] = ypan; extra_kind[n_extra++] = X_Y; }
    if (ym1 && (any || cf.z != 0.f)) { extra_src[n_extra] = ym1; extra_kind[n_extra++] = X_YM1; }
    if (yp1 && (any || cf.w != 0.f)) { extra_src[n_extra] = yp1; extra_kind[n_extra++] = X_YP1; }
  }
  if (lane == 0) {
    for (int i = 0; i < R; ++i) mbar_init(full(i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  int p_a = blockIdx.x, p_q = 0, p_k0 = 0, p_nb = 0, issued = 0;
  auto load_row = [&]() {  // rows with no tile (no stored block, no source term) are skipped
    for (; p_a < n_atoms; p_a += gridDim.x) {
      p_k0 = __ldg(row_ptr + p_a);
      p_nb = __ldg(row_ptr + p_a + 1) - p_k0;
      if (p_nb + n_extra > 0) break;
    }
  };
  auto issue_next = [&]() {
    if (p_a >= n_atoms) return;
    const bool own = p_q >= p_nb;
    const int b = own ? p_a : __ldg(col + p_k0 + p_q);
    const float* src = (own ? extra_src[p_q - p_nb] : bin) + (int64_t)9 * b * s;
    const int st = issued % R;
    const uint32_t dst = smem_u32(smem + st * C::SB), bar = full(st);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, C::XB + (own ? 0 : C::HB));
    bulk_g2s(dst, src, C::XB, bar);
    if (!own) bulk_g2s(dst + C::XB, hv + (int64_t)(p_k0 + p_q) * Layout<float, 9>::BS, C::HB, bar);
    ++issued;
    if (++p_q == p_nb + n_extra) {
      p_a += gridDim.x;
      p_q = 0;
      load_row();
    }
  };
  if (lane == 0) {
    load_row();
    for (int j = 0; j < R; ++j) issue_next();
  }
  __syncwarp();
  int it = 0;
  bool ok = true;
  uint32_t rdy = 0;  // stage it % R was found ready by the early test
  const int pl = 4 * lane;
  auto consumed = [&]() {
    __syncwarp();
    if (lane == 0) issue_next();
    ++it;
  };
  for (int a = blockIdx.x; a < n_atoms && ok; a += gridDim.x) {
    const int k0 = __ldg(row_ptr + a), k1 = __ldg(row_ptr + a + 1);
    uint64_t sd = seed;
    int64_t rloc = (int64_t)9 * a;
    float4 cfa = cf;
    if (batch.atom_cl) {
      const int cl = __ldg(batch.atom_cl + a);
      sd = __ldg(batch.seed + cl);
      rloc = (int64_t)9 * (a - __ldg(batch.atom0 + cl));
      if (cf_cl) cfa = cf_cl[cl];
    }
    float2 acc[9][2];
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
      spmm_tile_f2(reinterpret_cast<const float*>(base), reinterpret_cast<const float*>(base + C::XB), C::P,
                   pl, acc);
      consumed();
    }
    if (!ok) break;
    float yo[9][4];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
      for (int v = 0; v < 4; ++v) yo[i][v] = 2.f * acc_at(acc, i, v);
    if (cfa.x != 0.f) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int v = 0; v < 4; ++v) yo[i][v] = fmaf(cfa.x, tbk_probe_sign(sd, rloc + i, pl + v), yo[i][v]);
    }
    for (int e = 0; e < n_extra; ++e) {
      const int st = it % R;
      if (!rdy) {
        ok = mbar_wait(full(st), (it / R) & 1);
        if (!ok) break;
      }
      rdy = mbar_test(full((it + 1) % R), ((it + 1) / R) & 1);
      const float* X = reinterpret_cast<const float*>(smem + st * C::SB);
      const int kd = extra_kind[e];
      const float ce = kd == X_PREV ? -1.f : (kd == X_Y ? cfa.y : (kd == X_YM1 ? cfa.z : cfa.w));
      if (ce != 0.f) {  // a zero coefficient skips the tile (its rows may never have been formed)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const float4 t = *reinterpret_cast<const float4*>(X + i * C::P + pl);
          yo[i][0] = fmaf(ce, t.x, yo[i][0]); yo[i][1] = fmaf(ce, t.y, yo[i][1]);
          yo[i][2] = fmaf(ce, t.z, yo[i][2]); yo[i][3] = fmaf(ce, t.w, yo[i][3]);
        }
      }
      consumed();
    }
    if (!ok) break;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int64_t row = (int64_t)9 * a + i;
      *reinterpret_cast<float4*>(bout + row * s + pl) = make_float4(yo[i][0], yo[i][1], yo[i][2], yo[i][3]);
    }
  }
  if (!ok && lane == 0) {
    // let the copies in flight land before the CTA exits
    atomicOr(err, 2);
    for (int j = it; j < issued; ++j) mbar_wait(full(j % R), (j / R) & 1);
  }
}

// two stages: ~21 warps per SM instead of 14 (shared memory sets the limit); measured 11 % faster
// on the batch than three stages
constexpr int CLEN_SELF_R = 2;

// tr[k] = index of block (b, a) for block k = (a, b) (the pattern is symmetric).
__global__ void transpose_map(int n_atoms, const int32_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ col, int32_t* __restrict__ tr, int* err) {
  const int a = blockIdx.x * blockDim.y + threadIdx.y;
  if (a >= n_atoms) return;
  for (int k = row_ptr[a] + threadIdx.x; k < row_ptr[a + 1]; k += blockDim.x) {
    const int b = col[k];
    int lo = row_ptr[b], hi = row_ptr[b + 1] - 1, hit = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = col[mid];
      if (c == a) { hit = mid; break; }
      if (c < a) lo = mid + 1; else hi = mid - 1;
    }
    tr[k] = hit;
    if (hit < 0) atomicOr(err, 1);
  }
}

// G[k] = scale * (Gacc[k] + Gacc[tr[k]]^T) / 2
template <int B>
__global__ void symmetrize(int64_t nnzb, const int32_t* __restrict__ tr, const double* __restrict__ Gacc,
                           double scale, double* __restrict__ G) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzb * B * B) return;
  const int64_t k = t / (B * B);
  const int e = (int)(t - k * B * B), i = e / B, l = e - i * B;
  const int64_t kt = tr[k];
  G[t] = kt < 0 ? 0.0 : 0.5 * scale * (Gacc[t] + Gacc[kt * B * B + l * B + i]);
}

__device__ __forceinline__ double mi(double d, double L) { return L > 0.0 ? d - L * rint(d / L) : d; }

// tq[k] = <G_ab, dH_ab/dd> for every off-diagonal block k = (a, b), d = R_b - R_a (SK model).
__global__ void bond_terms(DevModel M, const double* __restrict__ pos, int n_atoms,
                           const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ G, double* __restrict__ tq) {
  const int a = blockIdx.x * blockDim.y + threadIdx.y;
  if (a >= n_atoms) return;
  for (int k = row_ptr[a] + threadIdx.x; k < row_ptr[a + 1]; k += blockDim.x) {
    const int b = col[k];
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    if (b != a) {
      Dual3 d[3];
      for (int c = 0; c < 3; ++c) {
        d[c] = Dual3(mi(pos[3 * b + c] - pos[3 * a + c], M.box[c]));
        d[c].g[c] = 1.0;
      }
      Dual3 E[81];
      sk_block<Dual3>(d, M.V, M.r0, M.decay, E);
      const double* g = G + (int64_t)k * 81;
      for (int e = 0; e < 81; ++e) {
        t0 += g[e] * E[e].g[0];
        t1 += g[e] * E[e].g[1];
        t2 += g[e] * E[e].g[2];
      }
    }
    tq[3 * k] = t0;
    tq[3 * k + 1] = t1;
    tq[3 * k + 2] = t2;
  }
}

// F_c = -dOmega/dR_c = sum_{b != c} (tq[(c, b)] - tq[(b, c)]), fixed order per atom.
__global__ void gather_forces(int n_atoms, const int32_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ col, const int32_t* __restrict__ tr,
                              const double* __restrict__ tq, double* __restrict__ F) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_atoms) return;
  double f0 = 0.0, f1 = 0.0, f2 = 0.0;
  for (int k = row_ptr[c]; k < row_ptr[c + 1]; ++k) {
    if (col[k] == c) continue;
    const int kt = tr[k];
    if (kt < 0) continue;
    f0 += tq[3 * k] - tq[3 * kt];
    f1 += tq[3 * k + 1] - tq[3 * kt + 1];
    f2 += tq[3 * k + 2] - tq[3 * kt + 2];
  }
  F[3 * c] = f0;
  F[3 * c + 1] = f1;
  F[3 * c + 2] = f2;
}

bool fused_eligible(const HOp& op, int s, int plain) {
  return !plain && op.prec == TBK_MIXED && op.B == 9 && (s == 128 || s == 256 || s == 512);
}

template <int CW, bool SD>
static void launch_fused_cw(tbk_ctx* ctx, const HOp& op, const void* bin, const void* bprev, void* bout,
                            const void* ypan, float4 cf, uint64_t seed, int s, double w, double* Gacc,
                            int* err, const BatchRows& batch, const float4* cf_cl, const void* ym1,
                            const void* yp1) {
  using C = SdCfg<CW, SD>;
  TBK_CUDA(cudaFuncSetAttribute(clenshaw_sddmm_bulk<CW, SD>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  int occ = 0;
  TBK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, clenshaw_sddmm_bulk<CW, SD>, C::THREADS, C::SMEM));
  TBK_CHECK_ARG(occ > 0, "fused adjoint kernel does not fit on this device");
  const int G = std::max(1, std::min(op.n_atoms, occ * ctx->num_sms));
  clenshaw_sddmm_bulk<CW, SD><<<G, C::THREADS, C::SMEM, ctx->stream>>>(
      op.n_atoms, op.row_ptr, op.col, (const float*)op.hv, (const float*)bin, (const float*)bprev,
      (float*)bout, (const float*)ypan, cf, seed, s, w, Gacc, err, batch, cf_cl, (const float*)ym1,
      (const float*)yp1, ctx->stall_next_adjoint);
  ctx->stall_next_adjoint = 0;
  post_launch(ctx, "clenshaw_sddmm_bulk");
}

void launch_fused(tbk_ctx* ctx, const HOp& op, const void* bin, const void* bprev, void* bout,
                  const void* ypan, float4 cf, uint64_t seed, int s, double w, double* Gacc,
                  int* err, const BatchRows& batch, const float4* cf_cl, const void* ym1,
                  const void* yp1) {
  KernelTimerScope timer(ctx, TBK_KERNEL_BACKWARD);
  // Gacc == nullptr: the Clenshaw step alone
  auto go = [&](auto cw, auto sd) {
    launch_fused_cw<decltype(cw)::value, decltype(sd)::value>(ctx, op, bin, bprev, bout, ypan, cf, seed, s, w,
                                                              Gacc, err, batch, cf_cl, ym1, yp1);
  };
  using T = std::true_type;
  using F = std::false_type;
  if (s == 512) Gacc ? go(std::integral_constant<int, 4>(), T()) : go(std::integral_constant<int, 4>(), F());
  else if (s == 256) Gacc ? go(std::integral_constant<int, 2>(), T()) : go(std::integral_constant<int, 2>(), F());
  else if (Gacc) go(std::integral_constant<int, 1>(), T());
  else {
    // the adjoint step alone at 128 probes: the self-fed single-warp kernel
    using C = ClenSelfCfg<CLEN_SELF_R>;
    static int occ_dev[64] = {0};
    int& occ = occ_dev[ctx->device & 63];
    if (!occ) {
      TBK_CUDA(cudaFuncSetAttribute(clenshaw_self<CLEN_SELF_R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
      TBK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, clenshaw_self<CLEN_SELF_R>, 32, C::SMEM));
      TBK_CHECK_ARG(occ > 0, "self-fed adjoint kernel does not fit on this device");
    }
    const int G = std::max(1, std::min(op.n_atoms, occ * ctx->num_sms));
    clenshaw_self<CLEN_SELF_R><<<G, 32, C::SMEM, ctx->stream>>>(
        op.n_atoms, op.row_ptr, op.col, (const float*)op.hv, (const float*)bin, (const float*)bprev,
        (float*)bout, (const float*)ypan, cf, seed, s, err, batch, cf_cl, (const float*)ym1, (const float*)yp1);
    post_launch(ctx, "clenshaw_self");
  }
}

void launch_sddmm(tbk_ctx* ctx, const HOp& op, const void* y, int y_is_probe, uint64_t seed,
                  const void* b, int s, double w, double* Gacc) {
  const int64_t threads = op.nnzb * 32;
  const unsigned grid = (unsigned)((threads + 255) / 256);
#define TBK_SD(TT, BB)                                                                          \
  sddmm_kernel<TT, BB><<<grid, 256, 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col,           \
                                                      (const TT*)y, seed, y_is_probe,           \
                                                      (const TT*)b, s, w, Gacc, op.nnzb)
  if (op.prec == TBK_MIXED) {
    if (op.B == 9) TBK_SD(float, 9); else TBK_SD(float, 1);
  } else {
    if (op.B == 9) TBK_SD(double, 9); else TBK_SD(double, 1);
  }
#undef TBK_SD
  post_launch(ctx, "sddmm_kernel");
}

// ---- pieces shared with the batched driver -------------------------------------------------

void launch_symmetrize(tbk_ctx* ctx, int64_t nnzb, int B, const int32_t* tr, const double* Gacc, double scale,
                       double* G) {
  const int64_t tot = nnzb * B * B;
  if (B == 9)
    symmetrize<9><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(nnzb, tr, Gacc, scale, G);
  else
    symmetrize<1><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(nnzb, tr, Gacc, scale, G);
  post_launch(ctx, "symmetrize");
}

void launch_transpose_map(tbk_ctx* ctx, int n_atoms, const int32_t* row_ptr, const int32_t* col,
                          int32_t* tr, int* err) {
  transpose_map<<<ceil_div(n_atoms, 16), dim3(8, 16), 0, ctx->stream>>>(n_atoms, row_ptr, col, tr, err);
  post_launch(ctx, "transpose_map");
}

// G[k] = scale(cluster of row a) (Gacc[k] + Gacc[tr[k]]^T) / 2 for a merged batch.
__global__ void symmetrize_batched(int n_atoms, const int32_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ tr, const int32_t* __restrict__ atom_cl,
                                   const double* __restrict__ scale_cl, const double* __restrict__ Gacc,
                                   double* __restrict__ G) {
  const int a = blockIdx.x * blockDim.y + threadIdx.y;
  if (a >= n_atoms) return;
  const double sc = scale_cl[atom_cl[a]];
  for (int k = row_ptr[a]; k < row_ptr[a + 1]; ++k)
    for (int e = threadIdx.x; e < 81; e += blockDim.x) {
      const int i = e / 9, l = e - 9 * i;
      const int64_t kt = tr[k];
      G[(int64_t)k * 81 + e] = kt < 0 ? 0.0 : 0.5 * sc * (Gacc[(int64_t)k * 81 + e] + Gacc[kt * 81 + l * 9 + i]);
    }
}

void launch_symmetrize_batched(tbk_ctx* ctx, int n_atoms, const int32_t* row_ptr, const int32_t* tr,
                               const int32_t* atom_cl, const double* scale_cl, const double* Gacc,
                               double* G) {
  symmetrize_batched<<<ceil_div(n_atoms, 8), dim3(32, 8), 0, ctx->stream>>>(n_atoms, row_ptr, tr, atom_cl,
                                                                             scale_cl, Gacc, G);
  post_launch(ctx, "symmetrize_batched");
}

void launch_forces(tbk_ctx* ctx, const DevModel& M, const double* pos, int n_atoms, const int32_t* row_ptr,
                   const int32_t* col, const int32_t* tr, const double* G, double* tq, double* F) {
  bond_terms<<<ceil_div(n_atoms, 8), dim3(4, 8), 0, ctx->stream>>>(M, pos, n_atoms, row_ptr, col, G, tq);
  post_launch(ctx, "bond_terms");
  gather_forces<<<ceil_div(n_atoms, 128), 128, 0, ctx->stream>>>(n_atoms, row_ptr, col, tr, tq, F);
  post_launch(ctx, "gather_forces");
}

template <int NC>
static void launch_window_g(tbk_ctx* ctx, const HOp& op, const WindowPanels& wp, int nw, uint64_t seed,
                            int s, double w, double* Gacc, int* err, const BatchRows& batch,
                            const int32_t* kcl, int k_lo) {
  using C = WinGCfg<NC>;
  TBK_CUDA(cudaFuncSetAttribute(sddmm_window_g<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  int occ = 0;
  TBK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sddmm_window_g<NC>, C::THREADS, C::SMEM));
  TBK_CHECK_ARG(occ > 0, "windowed outer-product kernel does not fit on this device");
  const int G = std::max(1, std::min(op.n_atoms, occ * ctx->num_sms));
  sddmm_window_g<NC><<<G, C::THREADS, C::SMEM, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, wp, nw, seed,
                                                               s, w, Gacc, err, batch, kcl, k_lo);
  post_launch(ctx, "sddmm_window_g");
}

void launch_window(tbk_ctx* ctx, const HOp& op, const WindowPanels& wp, int nw, uint64_t seed, int s,
                   double w, double* Gacc, int* err, const BatchRows& batch, const int32_t* kcl, int k_lo) {
  KernelTimerScope timer(ctx, TBK_KERNEL_WINDOW);
  TBK_CHECK_ARG(nw >= 1 && nw <= SDW && (wp.y[0] != nullptr || nw == 1), "bad outer-product window");
  if (s == 512) launch_window_g<4>(ctx, op, wp, nw, seed, s, w, Gacc, err, batch, kcl, k_lo);
  else if (s == 256) launch_window_g<2>(ctx, op, wp, nw, seed, s, w, Gacc, err, batch, kcl, k_lo);
  else launch_window_g<1>(ctx, op, wp, nw, seed, s, w, Gacc, err, batch, kcl, k_lo);
}

// ---- adjoint of the doubled moments (TMA-fed fused path) ------------------------------------
//
// The moments come from the doubling identities (C_m C_n = (C_{m+n} + C_{|m-n|})/2):
//   mu_2k = 2 e_k - mu_0,  mu_2k-1 = 2 o_k - mu_1,  e_k = <y_k, y_k>/s,  o_k = <y_k, y_{k-1}>/s,
// so Omega^ = sum_m c_m mu_m = const + sum_{k=1..K} (w_k e_k + v_k o_k),  K = floor(p/2), with
//   w_k = 2 c_2k (2k < p),  v_1 = c_1 - sum_{k>=2} c_{2k-1},  v_k = 2 c_{2k-1} (k >= 2, 2k-1 < p).
// Reverse-mode differentiation through y_{k+1} = 2 H^ y_k - y_{k-1} (y_1 = H^ y_0, y_0 = r):
//   ybar_K = g_K,  ybar_k = g_k + 2 H^ ybar_{k+1} - ybar_{k+2},
//   g_k = (2 w_k y_k + v_k y_{k-1} + v_{k+1} y_{k+1}) / s,
//   dOmega^/dH^ = sum_{k=1}^{K-1} 2 ybar_{k+1} y_k^T + ybar_1 y_0^T.
// This needs the y_k only up to K = p/2: half the forward, replay and backward work of the
// Clenshaw form of Eq. polynomial_response, for the same estimator and the same gradient.

__global__ void ybar_init(int64_t n, int s, float ca, const float* __restrict__ yk, float cb,
                          const float* __restrict__ ykm1, uint64_t seed, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * s) return;
  const int64_t row = i / s;
  const int p = (int)(i - row * s);
  const float prev = ykm1 ? ykm1[i] : tbk_probe_sign(seed, row, p);
  out[i] = fmaf(ca, yk[i], cb * prev);
}

// get_coefs() is called once every y_1 .. y_K has been formed for the first time (with
// `partials` != NULL those steps also wrote their moment partial sums at partials + 2 nctas (t-1),
// so the caller can finish the moments, solve for mu and return the coefficients c_0 .. c_{p-1}).
void adjoint_doubling(tbk_ctx* ctx, const HOp& op, uint64_t probe_seed, int s, int p,
                      const std::function<std::vector<double>()>& get_coefs, double* partials, int nctas,
                      int64_t max_panel_bytes, double* Gacc, int* err, int sched, const AdjBatch* bt,
                      const void* probe_panel, int s_norm) {
  TBK_CHECK_ARG(!(bt && probe_panel), "a batch regenerates its probes");
  const bool windowed = sched == 1;
  // outer products on the tensor cores after each backward step, where that kernel applies
  const bool tensor = sched == 2 && !bt && tc_sddmm_eligible(ctx, op, s, tc_sddmm_max_row(ctx, op));
  // a stored probe block y_0 (single system): read wherever the probe enters
  const bool r_panel = probe_panel != nullptr;
  const double nrm = r_panel && s_norm > 0 ? s_norm : s;
  const int K = bt ? (bt->K.empty() ? 0 : bt->K[0]) : p / 2;
  if (K < 1) {
    if (get_coefs) get_coefs();
    return;  // p = 1: the estimate does not depend on H
  }
  // atoms of the (order-sorted) clusters that take part in step t: a prefix of the merged rows
  auto active = [&](int t) {
    if (!bt) return op.n_atoms;
    int64_t r = 0;
    for (size_t ci = 0; ci < bt->K.size() && bt->K[ci] >= t; ++ci) r += bt->n_at[ci];
    return (int)r;
  };
  std::vector<double> w(K + 2, 0.0), v(K + 2, 0.0);
  // a batch brings its per-cluster coefficient table (filled by get_coefs() when given)
  bool have_coefs = bt != nullptr && !get_coefs;
  auto load_coefs = [&]() {
    const std::vector<double> c = get_coefs();
    have_coefs = true;
    if (bt) return;
    for (int k = 1; k <= K; ++k) {
      if (2 * k < p) w[k] = 2.0 * c[2 * k];
      if (k >= 2 && 2 * k - 1 < p) v[k] = 2.0 * c[2 * k - 1];
    }
    v[1] = p > 1 ? c[1] : 0.0;
    for (int k = 2; 2 * k - 1 < p; ++k) v[1] -= c[2 * k - 1];
  };
  auto ca = [&](int k) { return (float)(2.0 * w[k] / nrm); };
  auto cb = [&](int k) { return (float)(v[k] / nrm); };
  auto cc = [&](int k) { return (float)(v[k + 1] / nrm); };

  const size_t panel = (size_t)op.n_rows * s * 4;
  size_t budget = max_panel_bytes > 0 ? (size_t)max_panel_bytes : panel_budget(ctx, WS_CHECKPOINTS);
  const int npan = K;  // y_1 .. y_K
  // ybar_j lives in ring slot j mod NB: the two of the recurrence, plus the window's SDW panels
  // when the outer products are summed over windows of steps; a batch also keeps the probe panel
  const int NB = windowed ? SDW + 2 : 2;
  const int NX = NB + (bt ? 1 : 0);
  int seg = std::max(1, npan);
  auto seg_plan = [&]() {
    // segments of a multiple of SDW steps, so that windows never straddle a segment
    const int r = std::max(2, (int)std::ceil(std::sqrt(2.0 * npan)));
    return ((r + SDW - 1) / SDW) * SDW;
  };
  // A batch's step t runs on the clusters with K_c >= t, a prefix of the merged rows, so its
  // all-stored plan can keep every y_j compactly: panel j holds the rows of the clusters still
  // running at step j - 1 (backward step j - 1 reads y_j on those rows, with a zero coefficient
  // for the clusters that stop there).  poff: byte offsets of P(0 .. npan) and E = y_{npan+1}.
  bool prefix = false;
  std::vector<size_t> poff;
  size_t prefix_tail = 0;
  if (bt) {
    const size_t row_bytes = (size_t)op.B * s * 4;
    poff.resize((size_t)npan + 2);
    size_t o = 0;
    for (int i = 0; i <= npan + 1; ++i) {
      poff[i] = o;
      o += (size_t)active(std::max(i - 1, 0)) * row_bytes;
      o = (o + 255) & ~(size_t)255;
    }
    prefix_tail = o;
    prefix = o + (size_t)NX * panel <= budget;
  }
  if (!prefix && (size_t)(npan + 2 + NX) * panel > budget && npan > 2) {
    seg = seg_plan();
    const size_t need = (size_t)(2 * ((npan + seg - 1) / seg) + seg + 2 + NX) * panel;
    if (need > budget)
      throw Error(TBK_ERR_OOM, "panel scratch budget of " + std::to_string(budget) +
                                   " bytes is below the checkpoint plan's " + std::to_string(need));
  }
  int nseg = (npan + seg - 1) / seg;
  // P(0 .. seg): segment panels (P(i) = y_{t0 - 1 + i}); checkpoints (y_{t0-2}, y_{t0-1}); E = y_{t1+1};
  // NB ybar panels; the probe panel of a batch
  auto plan_bytes = [&]() {
    if (prefix) return prefix_tail + (size_t)NX * panel;
    return panel * ((size_t)seg + 1 + (nseg <= 1 ? 0 : 2 * (size_t)nseg) + 1 + NX);
  };
  char* base = nullptr;
  try {
    base = (char*)scratch(ctx, WS_CHECKPOINTS, plan_bytes());
  } catch (const Error& e) {
    // the device could not map the all-stored plan after all: replay segments instead
    if (e.code != TBK_ERR_OOM || nseg > 1 || npan <= 2) throw;
    prefix = false;
    seg = seg_plan();
    nseg = (npan + seg - 1) / seg;
    base = (char*)scratch(ctx, WS_CHECKPOINTS, plan_bytes());
  }
  const bool all_stored = nseg <= 1;
  const size_t n_seg_pan = (size_t)seg + 1, n_ckpt = all_stored ? 0 : 2 * (size_t)nseg;
  // P(0 .. npan + 1) of the prefix plan at poff, the full-size panels after them
  auto P = [&](size_t i) -> void* {
    if (!prefix) return base + i * panel;
    if (i <= (size_t)npan + 1) return base + poff[i];
    return base + prefix_tail + (i - ((size_t)npan + 2)) * panel;
  };
  auto CK = [&](int sg, int which) { return P(n_seg_pan + 2 * (size_t)sg + which); };
  void* E = P(n_seg_pan + n_ckpt);
  auto YB = [&](int j) { return P(n_seg_pan + n_ckpt + 1 + (size_t)(j % NB)); };
  void* R0 = bt ? P(n_seg_pan + n_ckpt + 1 + NB) : const_cast<void*>(probe_panel);
  const BatchRows br = bt ? bt->br : BatchRows();
  if (bt) {
    // the probe block of every cluster, and ybar = 0 on the rows of clusters not yet started
    // (their first backward step then reduces to ybar_K = g_K)
    launch_batch_probe_panel(ctx, op, br, s, R0);
    for (int j = 0; j < NB; ++j) TBK_CUDA(cudaMemsetAsync(YB(j), 0, panel, ctx->stream));
  }
  auto forward_step = [&](int t, const void* yin, const void* yprev, void* yout, bool first_time) {
    HOp o = op;
    o.n_atoms = active(t);
    if (o.n_atoms <= 0) return;
    StepArgs a;
    a.seed = probe_seed;
    a.s = s;
    a.yin = t == 1 ? R0 : yin;
    a.cur_is_probe = t == 1 && !bt && !r_panel;
    a.alpha = t == 1 ? 1.0 : 2.0;
    if (t == 2) {
      if (bt || r_panel) a.yprev = R0; else a.c_r = -1.0;
    } else if (t >= 3) {
      a.yprev = const_cast<void*>(yprev);
    }
    a.yout = yout;
    a.err = err;
    a.batch = br;
    if (partials && first_time) {
      if (bt) {
        // per (atom, consumer warp) partial sums, reduced per cluster by the caller
        a.partials = partials + (size_t)(t - 1) * bt->pstride;
        a.per_task = 1;
      } else {
        a.partials = partials + (size_t)(t - 1) * nctas * 2;
      }
    }
    launch_step(ctx, o, a);
  };
  if (!all_stored) {
    void *cur = nullptr, *prv = nullptr;
    const int last = seg * (nseg - 1);
    for (int t = 1; t <= last; ++t) {
      void* out = t == 1 ? P(0) : (t == 2 ? P(1) : prv);
      forward_step(t, cur, prv, out, true);
      prv = cur;
      cur = out;
      if (t % seg == 0) {
        const int sg = t / seg;
        TBK_CUDA(cudaMemcpyAsync(CK(sg, 0), prv, panel, cudaMemcpyDeviceToDevice, ctx->stream));
        TBK_CUDA(cudaMemcpyAsync(CK(sg, 1), cur, panel, cudaMemcpyDeviceToDevice, ctx->stream));
      }
    }
  }
  int k = K;
  for (int sg = nseg - 1; sg >= -1 && k >= 0; --sg) {
    const int t0 = sg >= 0 ? 1 + seg * sg : 0;
    const int t1 = sg >= 0 ? std::min(npan, t0 + seg - 1) : 0;
    if (sg >= 0) {
      if (sg < nseg - 1) {
        // y_{t1+1} is the first panel of the segment just finished
        TBK_CUDA(cudaMemcpyAsync(E, P(1), panel, cudaMemcpyDeviceToDevice, ctx->stream));
      }
      const bool first_time = sg == nseg - 1;  // the last segment was never formed before
      int t = t0;
      if (sg > 0) {
        TBK_CUDA(cudaMemcpyAsync(P(0), CK(sg, 1), panel, cudaMemcpyDeviceToDevice, ctx->stream));
        forward_step(t0, P(0), CK(sg, 0), P(1), first_time);
        ++t;
      }
      for (; t <= t1; ++t) {
        const int i = t - t0 + 1;
        forward_step(t, t == 1 ? nullptr : P(i - 1), t >= 3 ? P(i - 2) : nullptr, P(i), first_time);
      }
    }
    if (!have_coefs) load_coefs();
    // y_j for j in [t0 - 1, t1 + 1] (nullptr = the probe block r = y_0, regenerated in the kernels)
    auto Y = [&](int j) -> const void* {
      if (j == 0) return r_panel ? R0 : nullptr;
      if (j == t1 + 1) return E;
      return P(j - t0 + 1);
    };
    for (; k >= t0; --k) {
      HOp o = op;
      o.n_atoms = active(std::max(k, 1));
      if (k == K && !bt) {
        // ybar_K = g_K (y_{K+1} does not enter)
        const int64_t n = op.n_rows * s;
        ybar_init<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
            op.n_rows, s, ca(K), (const float*)Y(K), cb(K), (const float*)Y(K - 1), probe_seed, (float*)YB(K));
        post_launch(ctx, "ybar_init");
        continue;
      }
      if (k >= 1) {
        // ybar_k = g_k + 2 H^ ybar_{k+1} - ybar_{k+2}; fused: and G += 2 y_k ybar_{k+1}^T on the pattern
        // (the probe coefficient .x scales the regenerated y_0; a stored y_0 streams as y_{k-1})
        const bool r_gen = k == 1 && !r_panel;
        const float4 cf = bt ? make_float4(0.f, 0.f, 0.f, 0.f)
                             : make_float4(r_gen ? cb(1) : 0.f, ca(k), r_gen ? 0.f : cb(k), cc(k));
        const float4* cfk = bt ? bt->cft + (size_t)k * bt->K.size() : nullptr;
        launch_fused(ctx, o, YB(k + 1), (k + 2 <= K || bt) ? YB(k + 2) : nullptr, YB(k), Y(k), cf, probe_seed, s,
                     2.0, (windowed || tensor) ? nullptr : Gacc, err, br, cfk,
                     (k >= 2 || r_panel) ? Y(k - 1) : nullptr, Y(k + 1));
        // G += 2 y_k ybar_{k+1}^T on the pattern, on the tensor cores
        if (tensor) launch_tc_sddmm(ctx, o, Y(k), YB(k + 1), s, 2.0, Gacc, err);
        if (windowed && (k - 1) % SDW == 0) {
          // G += 2 y_j ybar_{j+1}^T on the pattern for the window j = k .. min(k + SDW, K) - 1
          WindowPanels wp{};
          const int nw = std::min(SDW, K - k);
          for (int t = 0; t < nw; ++t) {
            wp.y[t] = (const float*)Y(k + t);
            wp.x[t] = (const float*)YB(k + t + 1);
          }
          launch_window(ctx, o, wp, nw, probe_seed, s, 2.0, Gacc, err, br, bt ? bt->d_K : nullptr, k);
        }
      } else if (windowed) {
        // G += y_0 ybar_1^T
        WindowPanels wp{};
        wp.y[0] = (const float*)Y(0);
        wp.x[0] = (const float*)YB(1);
        launch_window(ctx, o, wp, 1, probe_seed, s, 1.0, Gacc, err, br, bt ? bt->d_K : nullptr, 0);
      } else if (tensor && Y(0)) {
        // G += y_0 ybar_1^T with a stored probe block
        launch_tc_sddmm(ctx, o, Y(0), YB(1), s, 1.0, Gacc, err);
      } else {
        launch_fused(ctx, o, YB(1), nullptr, nullptr, Y(0), make_float4(0.f, 0.f, 0.f, 0.f), probe_seed, s,
                     1.0, Gacc, err, br, nullptr, nullptr, nullptr);
      }
    }
  }
}

}  // namespace tbk

using namespace tbk;

namespace tbk {
// The adjoint's outer-product schedule: TBK_WINDOWED or TBK_FUSED_ADJOINT when given, else what
// tbk_autotune measured for this shape, else fused.
int outer_schedule(const tbk_ctx* ctx, const HOp& op, int s, int flags) {
  if (flags & TBK_TC_OUTER) return 2;
  if (flags & TBK_WINDOWED) return 1;
  if (flags & TBK_FUSED_ADJOINT) return 0;
  const tbk_ctx::Tuned* t = find_tuned(ctx, op.n_rows, op.nnzb, s);
  return t ? t->windowed : 0;
}
}  // namespace tbk

extern "C" int tbk_density_and_forces(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model,
                                      const double* pos, const double* box, double emin,
                                      double emax, uint64_t probe_seed, int32_t n_probes,
                                      int32_t order, double mu, double kT, int32_t damping,
                                      int32_t flags, int64_t max_panel_bytes, double* G,
                                      double* forces) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG(G || forces, "nothing to compute: G and forces are both NULL");
  TBK_CHECK_ARG(order >= 1, "order must be >= 1");
  TBK_CHECK_ARG(n_probes >= 4 && n_probes % 4 == 0, "n_probes must be a positive multiple of 4");
  TBK_CHECK_ARG((flags & ~(TBK_FP64 | TBK_PLAIN_KERNEL | TBK_WINDOWED | TBK_FUSED_ADJOINT | TBK_TC_OUTER)) == 0, "unknown flag");
  const int plain = (flags & TBK_PLAIN_KERNEL) ? 1 : 0;
  TBK_CHECK_ARG(kT > 0.0, "kT must be positive");
  DeviceGuard dg(ctx);
  const int prec = (flags & TBK_FP64) ? TBK_FP64 : TBK_MIXED;
  DevModel M{};
  if (forces) {
    M = upload_model(ctx, model, box, WS_TABLE);
    TBK_CHECK_ARG(M.kind == TBK_MODEL_SK, "forces need the Slater-Koster model");
    TBK_CHECK_ARG(pos != nullptr, "pos is NULL");
  }
  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  HOp op = prepare_hop(ctx, H, emin, emax, prec, WS_HHAT, err);
  const int p = order, s = n_probes, BB = op.B * op.B;
  const bool fused = fused_eligible(op, s, plain);
  const double W = emax - emin;

  // coefficients c_k = d_k beta_k[g] (device, then host for the per-step scalars)
  double* dcoef = (double*)scratch(ctx, WS_COEF, sizeof(double) * (size_t)p);
  coefficients(ctx, TBK_FN_FREE, p, emin, emax, mu, kT, damping, dcoef);
  std::vector<double> c(p);
  TBK_CUDA(cudaMemcpyAsync(c.data(), dcoef, sizeof(double) * p, cudaMemcpyDeviceToHost, ctx->stream));

  // transpose map of the pattern
  int32_t* tr = (int32_t*)scratch(ctx, WS_TRANSPOSE, sizeof(int32_t) * (size_t)op.nnzb);
  transpose_map<<<ceil_div(op.n_atoms, 16), dim3(8, 16), 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, tr, err);
  post_launch(ctx, "transpose_map");

  double* Gacc = (double*)scratch(ctx, WS_GACC, sizeof(double) * (size_t)op.nnzb * BB * 2);
  double* Gsym = Gacc + (size_t)op.nnzb * BB;
  TBK_CUDA(cudaMemsetAsync(Gacc, 0, sizeof(double) * (size_t)op.nnzb * BB, ctx->stream));

  const size_t esz = prec == TBK_MIXED ? 4 : 8;
  const size_t panel = (size_t)op.n_rows * s * esz;
  double scale = 2.0 / (W * s);
  if (fused) {
    adjoint_doubling(ctx, op, probe_seed, s, p, [&]() { return c; }, nullptr, 0, max_panel_bytes, Gacc, err,
                       outer_schedule(ctx, op, s, flags), nullptr);
    scale = 2.0 / W;  // the 1/s of the moments is inside the source terms
  } else {
    // Panels y_1 .. y_{p-2} are needed in reverse order: all of them are kept when they fit the
    // budget, else segments of ~sqrt(2p) steps are replayed from checkpoints.
    const int npan = std::max(0, p - 2);  // y_1 .. y_{p-2}
    size_t budget = max_panel_bytes > 0 ? (size_t)max_panel_bytes : panel_budget(ctx, WS_CHECKPOINTS);
    int seg = std::max(1, npan);
    if ((size_t)(npan + 3) * panel > budget && npan > 2) {
      seg = std::max(2, (int)std::ceil(std::sqrt(2.0 * npan)));
      const size_t need = (size_t)(2 * ((npan + seg - 1) / seg) + seg + 3) * panel;
      if (need > budget)
        throw Error(TBK_ERR_OOM, "panel scratch budget of " + std::to_string(budget) +
                                     " bytes is below the checkpoint plan's " + std::to_string(need));
    }
    const int nseg = npan > 0 ? (npan + seg - 1) / seg : 0;
    const bool all_stored = nseg <= 1;
    // Scratch layout: P(0 .. seg) segment panels, P(seg+1 ..) checkpoints, then two b panels.
    // Segment sg covers y_j for j in [t0, t1], t0 = 1 + seg sg, t1 = min(p - 2, t0 + seg - 1),
    // and holds y_{t0 - 1 + i} at P(i).  Checkpoint sg (sg >= 1) is (y_{t0-2}, y_{t0-1}).
    const size_t n_seg_pan = (size_t)seg + 1;
    const size_t n_ckpt = all_stored ? 0 : 2 * (size_t)nseg;
    char* base = (char*)scratch(ctx, WS_CHECKPOINTS, panel * (n_seg_pan + n_ckpt + 2));
    auto P = [&](size_t i) { return (void*)(base + i * panel); };
    auto CK = [&](int sg, int which) { return P(n_seg_pan + 2 * (size_t)sg + which); };
    void* bcur = P(n_seg_pan + n_ckpt);
    void* bprev = P(n_seg_pan + n_ckpt + 1);

    // y_t from y_{t-1} (yin; the probe block when t == 1) and y_{t-2} (the probe when t == 2).
    auto forward_step = [&](int t, const void* yin, const void* yprev, void* yout) {
      StepArgs a;
      a.seed = probe_seed;
      a.s = s;
      a.yin = yin;
      a.cur_is_probe = t == 1;
      a.alpha = t == 1 ? 1.0 : 2.0;
      if (t == 2) a.c_r = -1.0;
      else if (t >= 3) a.yprev = const_cast<void*>(yprev);
      a.yout = yout;
      a.err = err;
      a.force_simple = plain;
      launch_step(ctx, op, a);
    };
    // Forward sweep to the last checkpoint, with two rotating panels.
    if (!all_stored) {
      void *cur = nullptr, *prv = nullptr;
      const int last = seg * (nseg - 1);
      for (int t = 1; t <= last; ++t) {
        void* out = t == 1 ? P(0) : (t == 2 ? P(1) : prv);
        forward_step(t, cur, prv, out);
        prv = cur;
        cur = out;
        if (t % seg == 0) {
          const int sg = t / seg;  // the segment starting at t0 = t + 1
          TBK_CUDA(cudaMemcpyAsync(CK(sg, 0), prv, panel, cudaMemcpyDeviceToDevice, ctx->stream));
          TBK_CUDA(cudaMemcpyAsync(CK(sg, 1), cur, panel, cudaMemcpyDeviceToDevice, ctx->stream));
        }
      }
    }
    // Backward sweep: b_{p-1} = c_{p-1} r, then for j = p-2 .. 0 add the y_j b_{j+1} term and
    // form b_j = c_j r + 2 H^ b_{j+1} - b_{j+2}.
    if (p >= 2) {
      launch_scaled_probe(ctx, op, bcur, c[p - 1], probe_seed, s);
      bool have_bprev = false;
      int j = p - 2;
      for (int sg = nseg - 1; sg >= -1 && j >= 0; --sg) {
        const int t0 = sg >= 0 ? 1 + seg * sg : 0;
        const int t1 = sg >= 0 ? std::min(npan, t0 + seg - 1) : 0;
        if (sg >= 0) {
          int t = t0;
          if (sg > 0) {
            TBK_CUDA(cudaMemcpyAsync(P(0), CK(sg, 1), panel, cudaMemcpyDeviceToDevice, ctx->stream));
            forward_step(t0, P(0), CK(sg, 0), P(1));
            ++t;
          }
          for (; t <= t1; ++t) {
            const int i = t - t0 + 1;
            forward_step(t, t == 1 ? nullptr : P(i - 1), t >= 3 ? P(i - 2) : nullptr, P(i));
          }
        }
        for (; j >= t0; --j) {
          const void* yj = j == 0 ? nullptr : P(j - t0 + 1);
          launch_sddmm(ctx, op, yj, j == 0, probe_seed, bcur, s, j == 0 ? 1.0 : 2.0, Gacc);
          if (j >= 1) {
            StepArgs a;
            a.seed = probe_seed;
            a.s = s;
            a.yin = bcur;
            a.alpha = 2.0;
            a.c_r = c[j];
            a.yprev = have_bprev ? bprev : nullptr;
            a.yout = bprev;
            a.err = err;
            a.force_simple = plain;
            launch_step(ctx, op, a);
            std::swap(bcur, bprev);
            have_bprev = true;
          }
        }
      }
    }
  }
  // symmetrise and scale: G = scale sym(Gacc)
  double* Gout = G ? G : Gsym;
  const int64_t tot = op.nnzb * BB;
  if (op.B == 9)
    symmetrize<9><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(op.nnzb, tr, Gacc, scale, Gout);
  else
    symmetrize<1><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(op.nnzb, tr, Gacc, scale, Gout);
  post_launch(ctx, "symmetrize");
  if (forces) {
    double* tq = (double*)scratch(ctx, WS_MISC, sizeof(double) * 3 * (size_t)op.nnzb);
    bond_terms<<<ceil_div(op.n_atoms, 8), dim3(4, 8), 0, ctx->stream>>>(M, pos, op.n_atoms, op.row_ptr,
                                                                        op.col, Gout, tq);
    post_launch(ctx, "bond_terms");
    gather_forces<<<ceil_div(op.n_atoms, 128), 128, 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col,
                                                                      tr, tq, forces);
    post_launch(ctx, "gather_forces");
  }
  int herr = 0;
  TBK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(herr);
  if (herr & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in the recurrence kernel expired");
  TBK_CHECK_ARG(herr == 0, "the block pattern is not symmetric");
  TBK_API_END
}

namespace tbk {
void fermi_enqueue(tbk_ctx* ctx, const double* moments, int order, double emin, double emax,
                   double n_electrons, double mu_fixed, double kT, int damping, double* tab,
                   double* rho, double* res);
int quad_nodes(int p);
}  // namespace tbk

namespace tbk {
// The one-call energies and forces on the doubled-moment adjoint (fused-eligible shapes): the
// adjoint's forward sweep over y_1 .. y_{p/2} also yields the moments, so no separate moment pass
// runs.  probe_panel / s_norm: a stored probe block and its sample count (NULL / 0: the
// Rademacher probes regenerated from probe_seed, s of them).
void energies_and_forces_doubled(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model, const double* pos,
                                 const double* box, double emin, double emax, uint64_t probe_seed, int s,
                                 int order, double n_electrons, double kT, int damping, int flags,
                                 int64_t max_panel_bytes, double* moments, double* observables, double* G,
                                 double* forces, const void* probe_panel, int s_norm) {
  const int prec = (flags & TBK_FP64) ? TBK_FP64 : TBK_MIXED;
  DevModel M{};
  if (forces) {
    M = upload_model(ctx, model, box, WS_TABLE);
    TBK_CHECK_ARG(M.kind == TBK_MODEL_SK, "forces need the Slater-Koster model");
    TBK_CHECK_ARG(pos != nullptr, "pos is NULL");
  }
  // err: bit 4 = a row has no diagonal block, bit 2 = a bounded wait expired, bit 1 = the pattern
  // is not symmetric; err[1] bit 1 = a panel outgrew ||r|| (the spectrum is not inside [emin, emax])
  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), ctx->stream));
  HOp op = prepare_hop(ctx, H, emin, emax, prec, WS_HHAT, err);
  const int p = order, BB = op.B * op.B;
  const int nrm = probe_panel && s_norm > 0 ? s_norm : s;
  const double W = emax - emin;
  int32_t* tr = (int32_t*)scratch(ctx, WS_TRANSPOSE, sizeof(int32_t) * (size_t)op.nnzb);
  launch_transpose_map(ctx, op.n_atoms, op.row_ptr, op.col, tr, err);
  double* Gacc = (double*)scratch(ctx, WS_GACC, sizeof(double) * (size_t)op.nnzb * BB * 2);
  double* Gsym = Gacc + (size_t)op.nnzb * BB;
  TBK_CUDA(cudaMemsetAsync(Gacc, 0, sizeof(double) * (size_t)op.nnzb * BB, ctx->stream));
  const int K = p / 2;
  const int nctas = step_grid_ctas(ctx, op, s);
  double* partials = (double*)scratch(ctx, WS_PARTIALS, sizeof(double) * 2 * (size_t)std::max(1, K) * nctas);
  const int M_nodes = quad_nodes(p);
  double* fbuf = (double*)scratch(ctx, WS_SEGMENT, sizeof(double) * ((size_t)2 * K + 64 + 5 * (size_t)M_nodes + 16 +
                                                                     (size_t)p + 8));
  double* sums = fbuf;
  double* tab = sums + 2 * (size_t)K + 64;
  double* rho = tab + 4 * (size_t)M_nodes;
  double* res = rho + M_nodes;
  double* mom = moments ? moments : res + 16;
  double* dcoef = (double*)scratch(ctx, WS_COEF, sizeof(double) * (size_t)p);
  auto after_forward = [&]() {
    // moments from the doubling identities, then mu, Omega, E, N, then c_k = d_k beta_k[g](mu)
    launch_moment_reduction(ctx, partials, nctas, K, p, nrm, op.n_rows, 0, sums, mom, err + 1);
    fermi_enqueue(ctx, mom, p, emin, emax, n_electrons, 0.0, kT, damping, tab, rho, res);
    double h[5];
    int herr[2] = {0, 0};
    TBK_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    TBK_CUDA(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    check_diagonal_flag(herr[0]);
    if ((herr[0] | herr[1]) & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in the recurrence kernel expired");
    TBK_CHECK_ARG(herr[0] == 0, "the block pattern is not symmetric");
    if (herr[1])
      throw Error(TBK_ERR_SPECTRUM, "a Chebyshev panel grew beyond ||r||: the spectrum of H is not "
                                    "inside [emin, emax]");
    if (h[4] != 0.0) throw Error(TBK_ERR_NOCONV, "n_electrons is outside the range of the estimated N(mu)");
    for (int i = 0; i < 4; ++i) observables[i] = h[i];
    coefficients(ctx, TBK_FN_FREE, p, emin, emax, h[0], kT, damping, dcoef);
    std::vector<double> c(p);
    TBK_CUDA(cudaMemcpyAsync(c.data(), dcoef, sizeof(double) * p, cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    return c;
  };
  adjoint_doubling(ctx, op, probe_seed, s, p, after_forward, partials, nctas, max_panel_bytes, Gacc, err,
                   outer_schedule(ctx, op, s, flags), nullptr, probe_panel, s_norm);
  double* Gout = G ? G : Gsym;
  const int64_t tot = op.nnzb * BB;
  symmetrize<9><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(op.nnzb, tr, Gacc, 2.0 / W, Gout);
  post_launch(ctx, "symmetrize");
  if (forces) {
    double* tq = (double*)scratch(ctx, WS_MISC, sizeof(double) * 3 * (size_t)op.nnzb);
    launch_forces(ctx, M, pos, op.n_atoms, op.row_ptr, op.col, tr, Gout, tq, forces);
  }
  int herr = 0;
  TBK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(herr);
  if (herr & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in the recurrence kernel expired");
  TBK_CHECK_ARG(herr == 0, "the block pattern is not symmetric");
}
}  // namespace tbk

// Energies and forces in one call: the adjoint's forward sweep over y_1 .. y_{p/2} also yields
// the (doubled) moments, so no separate moment pass is run.
extern "C" int tbk_energies_and_forces(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model,
                                       const double* pos, const double* box, double emin,
                                       double emax, uint64_t probe_seed, int32_t n_probes,
                                       int32_t order, double n_electrons, double kT,
                                       int32_t damping, int32_t flags, int64_t max_panel_bytes,
                                       double* moments, double* observables, double* G,
                                       double* forces) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr && observables != nullptr, "NULL argument");
  TBK_CHECK_ARG(order >= 1, "order must be >= 1");
  TBK_CHECK_ARG(n_probes >= 4 && n_probes % 4 == 0, "n_probes must be a positive multiple of 4");
  TBK_CHECK_ARG((flags & ~(TBK_FP64 | TBK_PLAIN_KERNEL | TBK_WINDOWED | TBK_FUSED_ADJOINT | TBK_TC_OUTER)) == 0, "unknown flag");
  TBK_CHECK_ARG(kT > 0.0 && n_electrons >= 0.0, "kT must be positive and n_electrons >= 0");
  DeviceGuard dg(ctx);
  const int prec = (flags & TBK_FP64) ? TBK_FP64 : TBK_MIXED;
  const int plain = (flags & TBK_PLAIN_KERNEL) ? 1 : 0;
  HOp shape;
  shape.B = H ? H->n_orb : 0;
  shape.prec = prec;
  if (!H || !fused_eligible(shape, n_probes, plain)) {
    // the separate calls give the same results for the other shapes and precisions
    double* mom = moments ? moments : (double*)scratch(ctx, WS_SEGMENT, sizeof(double) * (size_t)order);
    int rc = tbk_chebyshev_moments(ctx, H, emin, emax, probe_seed, n_probes, order,
                                   flags & ~(TBK_WINDOWED | TBK_FUSED_ADJOINT | TBK_TC_OUTER), mom);
    if (rc != TBK_OK) throw Error(rc, tbk_last_error());
    rc = tbk_fermi_level(ctx, mom, order, emin, emax, n_electrons, 0.0, kT, damping, observables);
    if (rc != TBK_OK) throw Error(rc, tbk_last_error());
    if (G || forces) {
      rc = tbk_density_and_forces(ctx, H, model, pos, box, emin, emax, probe_seed, n_probes, order,
                                  observables[0], kT, damping, flags, max_panel_bytes, G, forces);
      if (rc != TBK_OK) throw Error(rc, tbk_last_error());
    }
    return TBK_OK;
  }
  energies_and_forces_doubled(ctx, H, model, pos, box, emin, emax, probe_seed, n_probes, order, n_electrons,
                              kT, damping, flags, max_panel_bytes, moments, observables, G, forces, nullptr, 0);
  TBK_API_END
}
