// f3: the local approximation of the sampled density and energy-density matrices (Sec. II.C.1,
// Eq. local_density, S = I).
//
// For each atom a, the region R_a = the atoms within r_max of a (the mask M_L(r_max) of the
// paper; a included) defines the local operator H_a = L_a^T H L_a.  All n_orb functions of a share
// its centre and so its region: one local problem per atom gives the n_orb columns of a, which
// are P~_L[:, a] = L_a p_f(H_a) L_a^T E_a and Q~_L[:, a] = L_a H_a p_f(H_a) L_a^T E_a, E_a the unit
// vectors of a's functions, p_f the order-term Chebyshev expansion of the Fermi function on the
// global bounds [emin, emax] (every local spectrum lies inside them: a principal submatrix's
// eigenvalues interlace H's).  The result is kept on the pattern M of H: block (b, a) of the output
// is rows b of column block a.  Columns come from different local problems, so the result is not
// symmetric.
//
// All local problems run together as one block-diagonal operator: the regions' atoms are listed
// one region after another (region a's atom i at merged index rs[a] + i), the local pattern is M
// restricted to each region, and each local block is a copy of the mapped global block
// (H^ of the global bounds restricted to the region is the region's own mapped operator).  X =
// p_f(H^_loc) E is formed by the backward (Clenshaw) form of the sum on the recurrence kernels,
// with the unit-vector source added by a scatter after each step; H X is one more product with
// the local copies of H itself.
#include <vector>

#include "cheb.cuh"
#include "scan.cuh"

namespace tbk {

// Position of value v in the ascending list c[lo .. hi), or -1.
__device__ __forceinline__ int find_in(const int32_t* __restrict__ c, int lo, int hi, int v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int x = c[mid];
    if (x == v) return mid;
    if (x < v) lo = mid + 1; else hi = mid;
  }
  return -1;
}

// Region of merged index t: the a with rs[a] <= t < rs[a + 1].
__device__ __forceinline__ int region_of(const int32_t* __restrict__ rs, int n_atoms, int64_t t) {
  int lo = 0, hi = n_atoms;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (rs[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Pass 1 (fill = false): cnt[t] = stored blocks of merged row t inside its region.  Pass 2 (fill):
// their local columns (merged indices) and global block indices, at lrp[t].
template <bool FILL>
__global__ void local_pattern(int n_atoms, int64_t n_loc, const int32_t* __restrict__ rs, const int32_t* __restrict__ rcol,
                              const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                              int32_t* __restrict__ cnt, const int64_t* __restrict__ lrp, int32_t* __restrict__ lcol,
                              int32_t* __restrict__ lblk) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_loc) return;
  const int a = region_of(rs, n_atoms, t);
  const int r0 = rs[a], r1 = rs[a + 1];
  const int g = rcol[t];
  int n = 0;
  int64_t o = FILL ? lrp[t] : 0;
  for (int k = rp[g]; k < rp[g + 1]; ++k) {
    const int j = find_in(rcol, r0, r1, col[k]);
    if (j < 0) continue;
    if (FILL) {
      lcol[o] = j;
      lblk[o] = k;
      ++o;
    }
    ++n;
  }
  if (!FILL) cnt[t] = n;
}

// The local copy of every mapped block: dst[k] = src[blk[k]] (BS elements each).
template <typename T>
__global__ void gather_blocks(int64_t nnz, int BS, const int32_t* __restrict__ blk, const T* __restrict__ src,
                              T* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnz * BS) return;
  const int64_t k = i / BS;
  dst[i] = src[(int64_t)blk[k] * BS + (i - k * BS)];
}

// own[a] = merged index of atom a inside its own region.
__global__ void own_index(int n_atoms, const int32_t* __restrict__ rs, const int32_t* __restrict__ rcol,
                          int32_t* __restrict__ own, int* __restrict__ err) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const int j = find_in(rcol, rs[a], rs[a + 1], a);
  if (j < 0) atomicOr(err, 1);
  own[a] = j < 0 ? rs[a] : j;
}

// panel[(own[a] B + c) S + c] += alpha for every atom a and c < B (the unit vectors E).
template <typename T>
__global__ void add_units(int n_atoms, int B, int S, const int32_t* __restrict__ own, double alpha,
                          T* __restrict__ panel) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_atoms * B) return;
  const int a = (int)(i / B), c = (int)(i - (int64_t)a * B);
  T* p = panel + ((int64_t)own[a] * B + c) * S + c;
  *p = (T)((double)*p + alpha);
}

// out[k][l][c] = X[(loc B + l) S + c] for every stored block k = (b, a) of M, loc = the merged
// index of b in a's region: rows b of column block a.
template <typename T>
__global__ void local_extract(int n_atoms, int B, int S, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const int32_t* __restrict__ rs, const int32_t* __restrict__ rcol,
                              const T* __restrict__ X, double* __restrict__ out, int* __restrict__ err) {
  const int b = blockIdx.x * blockDim.y + threadIdx.y;
  if (b >= n_atoms) return;
  for (int k = rp[b]; k < rp[b + 1]; ++k) {
    const int a = col[k];
    const int loc = find_in(rcol, rs[a], rs[a + 1], b);
    for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
      const int l = e / B, c = e - l * B;
      double v = 0.0;
      if (loc < 0) {
        if (e == 0) atomicOr(err, 1);
      } else {
        v = (double)X[((int64_t)loc * B + l) * S + c];
      }
      out[(int64_t)k * B * B + e] = v;
    }
  }
}

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_local_density(tbk_ctx* ctx, const tbk_bsr* H, const double* pos, const double* box,
                                 double r_max, double emin, double emax, int32_t order, double mu, double kT,
                                 int32_t damping, int32_t flags, double* P, double* Q) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr && H != nullptr && pos != nullptr, "NULL argument");
  TBK_CHECK_ARG(P || Q, "nothing to compute: P and Q are both NULL");
  TBK_CHECK_ARG(order >= 1, "order must be >= 1");
  TBK_CHECK_ARG(r_max > 0.0, "r_max must be positive");
  TBK_CHECK_ARG((flags & ~TBK_FP64) == 0, "unknown flag");
  TBK_CHECK_ARG(kT > 0.0, "kT must be positive");
  DeviceGuard dg(ctx);
  const int prec = (flags & TBK_FP64) ? TBK_FP64 : TBK_MIXED;
  const int n = H->n_atoms, B = H->n_orb, p = order;
  const int S = 4 * ((B + 3) / 4);                 // panel width: the B unit vectors, padded

  // 1. regions: the atoms within r_max of each atom (CSR, ascending)
  int32_t* rs = (int32_t*)scratch(ctx, WS_LOCAL0, sizeof(int32_t) * ((size_t)n + 1));
  int64_t n_loc = 0;
  int rc = tbk_build_neighbors(ctx, pos, n, box, r_max, rs, nullptr, 0, &n_loc);
  if (rc != TBK_OK) throw Error(rc, tbk_last_error());
  TBK_CHECK_ARG(n_loc < INT32_MAX, "the regions hold too many atoms");
  int32_t* rcol = (int32_t*)scratch(ctx, WS_LOCAL1, sizeof(int32_t) * (size_t)std::max<int64_t>(1, n_loc));
  rc = tbk_build_neighbors(ctx, pos, n, box, r_max, rs, rcol, n_loc, &n_loc);
  if (rc != TBK_OK) throw Error(rc, tbk_last_error());

  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  // 2. the local pattern: M restricted to each region, merged
  int32_t* cnt = (int32_t*)scratch(ctx, WS_LOCAL2, sizeof(int32_t) * (size_t)n_loc + sizeof(int32_t) * n + 64);
  int32_t* own = cnt + n_loc;
  local_pattern<false><<<ceil_div(n_loc, 256), 256, 0, ctx->stream>>>(n, n_loc, rs, rcol, H->row_ptr, H->col, cnt,
                                                                       nullptr, nullptr, nullptr);
  post_launch(ctx, "local_pattern");
  int64_t* lrp = (int64_t*)scratch(ctx, WS_LOCAL3, sizeof(int64_t) * ((size_t)n_loc + 1 + scan_tmp_elems(n_loc)));
  exclusive_scan_i32(ctx, cnt, lrp, n_loc, lrp + n_loc + 1);
  int64_t nnz_loc = 0;
  TBK_CUDA(cudaMemcpyAsync(&nnz_loc, lrp + n_loc, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  TBK_CHECK_ARG(nnz_loc < INT32_MAX, "the local operators hold too many blocks");
  int32_t* lrow = (int32_t*)scratch(ctx, WS_LOCAL4, sizeof(int32_t) * ((size_t)n_loc + 1 + 2 * (size_t)nnz_loc));
  int32_t* lcol = lrow + n_loc + 1;
  int32_t* lblk = lcol + nnz_loc;
  local_pattern<true><<<ceil_div(n_loc, 256), 256, 0, ctx->stream>>>(n, n_loc, rs, rcol, H->row_ptr, H->col, nullptr,
                                                                      lrp, lcol, lblk);
  post_launch(ctx, "local_pattern");
  {
    // the int32 row pointer of the merged operator
    std::vector<int64_t> h((size_t)n_loc + 1);
    TBK_CUDA(cudaMemcpyAsync(h.data(), lrp, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    std::vector<int32_t> h32(h.begin(), h.end());
    TBK_CUDA(cudaMemcpyAsync(lrow, h32.data(), sizeof(int32_t) * h32.size(), cudaMemcpyHostToDevice, ctx->stream));
    sync(ctx);
  }
  own_index<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(n, rs, rcol, own, err);
  post_launch(ctx, "own_index");

  // 3. local copies of the mapped blocks (H^ for X; H itself, the bounds [-1, 1], for H X)
  const size_t esz = prec == TBK_MIXED ? 4 : 8;
  const int BS = prec == TBK_MIXED ? (B == 1 ? Layout<float, 1>::BS : Layout<float, 9>::BS)
                                   : (B == 1 ? Layout<double, 1>::BS : Layout<double, 9>::BS);
  void* hv_loc = scratch(ctx, WS_SEGMENT, (size_t)nnz_loc * BS * esz);
  auto local_operator = [&](double lo, double hi) {
    HOp g = prepare_hop(ctx, H, lo, hi, prec, WS_HHAT, err);
    const int64_t tot = nnz_loc * BS;
    if (prec == TBK_MIXED)
      gather_blocks<float><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(nnz_loc, BS, lblk, (const float*)g.hv,
                                                                                  (float*)hv_loc);
    else
      gather_blocks<double><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(nnz_loc, BS, lblk, (const double*)g.hv,
                                                                                   (double*)hv_loc);
    post_launch(ctx, "gather_blocks");
    HOp o;
    o.n_atoms = (int)n_loc;
    o.B = B;
    o.prec = prec;
    o.nnzb = nnz_loc;
    o.n_rows = n_loc * B;
    o.row_ptr = lrow;
    o.col = lcol;
    o.hv = hv_loc;
    return o;
  };
  HOp op = local_operator(emin, emax);

  // 4. coefficients of p_f, then X = p_f(H^) E by the Clenshaw form with unit-vector sources
  double* dcoef = (double*)scratch(ctx, WS_COEF, sizeof(double) * (size_t)p);
  coefficients(ctx, TBK_FN_FERMI, p, emin, emax, mu, kT, damping, dcoef);
  std::vector<double> c(p);
  TBK_CUDA(cudaMemcpyAsync(c.data(), dcoef, sizeof(double) * p, cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  const size_t panel = (size_t)op.n_rows * S * esz;
  char* base = (char*)scratch(ctx, WS_CHECKPOINTS, 3 * panel);
  void* B1 = base;
  void* B2 = base + panel;
  void* X = base + 2 * panel;
  auto add_e = [&](void* pnl, double alpha) {
    if (alpha == 0.0) return;
    const int64_t tot = (int64_t)n * B;
    if (prec == TBK_MIXED)
      add_units<float><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(n, B, S, own, alpha, (float*)pnl);
    else
      add_units<double><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(n, B, S, own, alpha, (double*)pnl);
    post_launch(ctx, "add_units");
  };
  auto step = [&](const HOp& o, const void* yin, void* yprev, void* yout, double alpha) {
    StepArgs a;
    a.yin = yin;
    a.yprev = yprev;
    a.yout = yout;
    a.alpha = alpha;
    a.s = S;
    a.err = err;
    a.force_simple = 1;
    launch_step(ctx, o, a);
  };
  TBK_CUDA(cudaMemsetAsync(X, 0, panel, ctx->stream));
  if (p == 1) {
    add_e(X, c[0]);
  } else {
    TBK_CUDA(cudaMemsetAsync(B1, 0, panel, ctx->stream));
    add_e(B1, c[p - 1]);                           // b_{p-1} = alpha_{p-1} E
    void *bk1 = B1, *bk2 = nullptr;
    for (int k = p - 2; k >= 1; --k) {
      void* out = bk2 ? bk2 : B2;
      step(op, bk1, bk2, out, 2.0);                // 2 H^ b_{k+1} - b_{k+2}
      add_e(out, c[k]);                            // + alpha_k E
      bk2 = bk1;
      bk1 = out;
    }
    step(op, bk1, bk2, X, 1.0);                    // X = H^ b_1 - b_2 + alpha_0 E
    add_e(X, c[0]);
  }
  const dim3 eb(32, 8);
  auto extract = [&](const void* Y, double* out) {
    if (prec == TBK_MIXED)
      local_extract<float><<<ceil_div(n, 8), eb, 0, ctx->stream>>>(n, B, S, H->row_ptr, H->col, rs, rcol,
                                                                   (const float*)Y, out, err);
    else
      local_extract<double><<<ceil_div(n, 8), eb, 0, ctx->stream>>>(n, B, S, H->row_ptr, H->col, rs, rcol,
                                                                    (const double*)Y, out, err);
    post_launch(ctx, "local_extract");
  };
  if (P) extract(X, P);
  if (Q) {
    HOp h1 = local_operator(-1.0, 1.0);
    step(h1, X, nullptr, B1, 1.0);                 // H X
    extract(B1, Q);
  }
  int herr = 0;
  TBK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(herr);
  TBK_CHECK_ARG(herr == 0, "a stored block of H joins atoms farther apart than r_max");
  TBK_API_END
}
