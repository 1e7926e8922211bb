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
#include <vector>

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

static void launch_sddmm(tbk_ctx* ctx, const HOp& op, const void* y, int y_is_probe, uint64_t seed,
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

}  // namespace tbk

using namespace tbk;

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
  TBK_CHECK_ARG((flags & ~(TBK_FP64 | TBK_PLAIN_KERNEL)) == 0, "unknown flag");
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
  HOp op = prepare_hop(ctx, H, emin, emax, prec, WS_HHAT);
  const int p = order, s = n_probes, BB = op.B * op.B;
  const double W = emax - emin;

  // coefficients c_k = d_k beta_k[g] (device, then host for the per-step scalars)
  double* dcoef = (double*)scratch(ctx, WS_COEF, sizeof(double) * (size_t)p);
  coefficients(ctx, TBK_FN_FREE, p, emin, emax, mu, kT, damping, dcoef);
  std::vector<double> c(p);
  TBK_CUDA(cudaMemcpyAsync(c.data(), dcoef, sizeof(double) * p, cudaMemcpyDeviceToHost, ctx->stream));

  // transpose map of the pattern
  int32_t* tr = (int32_t*)scratch(ctx, WS_TRANSPOSE, sizeof(int32_t) * (size_t)op.nnzb);
  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  transpose_map<<<ceil_div(op.n_atoms, 16), dim3(8, 16), 0, ctx->stream>>>(op.n_atoms, op.row_ptr, op.col, tr, err);
  post_launch(ctx, "transpose_map");

  double* Gacc = (double*)scratch(ctx, WS_GACC, sizeof(double) * (size_t)op.nnzb * BB * 2);
  double* Gsym = Gacc + (size_t)op.nnzb * BB;
  TBK_CUDA(cudaMemsetAsync(Gacc, 0, sizeof(double) * (size_t)op.nnzb * BB, ctx->stream));

  const size_t esz = prec == TBK_MIXED ? 4 : 8;
  const size_t panel = (size_t)op.n_rows * s * esz;
  // Panels y_1 .. y_{p-2} are needed in reverse order: all of them are kept when they fit the
  // budget, else segments of ~sqrt(2p) steps are replayed from checkpoints.
  const int npan = std::max(0, p - 2);  // y_1 .. y_{p-2}
  size_t budget = (size_t)std::max<int64_t>(0, max_panel_bytes);
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    TBK_CUDA(cudaMemGetInfo(&fr, &tot));
    budget = (size_t)(0.6 * (double)fr);
  }
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
  // symmetrise and scale: G = (2/W)(1/s) sym(Gacc)
  double* Gout = G ? G : Gsym;
  const int64_t tot = op.nnzb * BB;
  const double scale = 2.0 / (W * s);
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
  if (herr & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in the recurrence kernel expired");
  TBK_CHECK_ARG(herr == 0, "the block pattern is not symmetric");
  TBK_API_END
}
