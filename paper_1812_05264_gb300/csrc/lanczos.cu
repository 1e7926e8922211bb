// a3: spectral bounds [e_min, e_max] of H by FP64 Lanczos (the paper maps the spectral interval
// onto [-1, 1] before the Chebyshev expansion, Sec. II.B.1).  The Lanczos scalars stay on the
// device; the host reads the tridiagonal matrix once at the end and takes its extreme
// eigenvalues (Sturm bisection) and eigenvector end components (inverse iteration).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace tbk {

// w = H v - beta * vprev (beta read from the device; vprev may be NULL), and per-CTA partial
// sums of w . v.  One thread per orbital row.
__device__ __forceinline__ void lz_spmv_cta(int cta, int n_atoms, int B, const int32_t* __restrict__ row_ptr,
                                            const int32_t* __restrict__ col, const double* __restrict__ H,
                                            const double* __restrict__ v, const double* __restrict__ vprev,
                                            const double* __restrict__ beta, double* __restrict__ w,
                                            double* __restrict__ part) {
  __shared__ double red[32];
  const int64_t n = (int64_t)n_atoms * B;
  const int64_t row = (int64_t)cta * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (row < n) {
    const int a = (int)(row / B), i = (int)(row - (int64_t)a * B);
    double acc = 0.0;
    for (int k = row_ptr[a]; k < row_ptr[a + 1]; ++k) {
      const int b = col[k];
      const double* h = H + (int64_t)k * B * B + i * B;
      for (int l = 0; l < B; ++l) acc += h[l] * v[(int64_t)b * B + l];
    }
    if (vprev) acc -= (*beta) * vprev[row];
    w[row] = acc;
    d = acc * v[row];
  }
  double t = tbk_block_sum(d, red);
  if (threadIdx.x == 0) part[cta] = t;
}

__global__ void lz_spmv(int n_atoms, int B, const int32_t* __restrict__ row_ptr,
                        const int32_t* __restrict__ col, const double* __restrict__ H,
                        const double* __restrict__ v, const double* __restrict__ vprev,
                        const double* __restrict__ beta, double* __restrict__ w,
                        double* __restrict__ part) {
  lz_spmv_cta(blockIdx.x, n_atoms, B, row_ptr, col, H, v, vprev, beta, w, part);
}

// w -= alpha v; per-CTA partial sums of w . w.
__device__ __forceinline__ void lz_orth_cta(int cta, int64_t n, const double* __restrict__ v,
                                            const double* __restrict__ alpha, double* __restrict__ w,
                                            double* __restrict__ part) {
  __shared__ double red[32];
  const int64_t i = (int64_t)cta * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (i < n) {
    double x = w[i] - (*alpha) * v[i];
    w[i] = x;
    d = x * x;
  }
  double t = tbk_block_sum(d, red);
  if (threadIdx.x == 0) part[cta] = t;
}

__global__ void lz_orth(int64_t n, const double* __restrict__ v, const double* __restrict__ alpha,
                        double* __restrict__ w, double* __restrict__ part) {
  lz_orth_cta(blockIdx.x, n, v, alpha, w, part);
}

// out = sum(part) (take_sqrt: sqrt of it), single block, fixed order.
__device__ __forceinline__ void lz_reduce_block(const double* __restrict__ part, int m, int take_sqrt,
                                                double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
  double t = tbk_block_sum(s, red);
  if (threadIdx.x == 0) *out = take_sqrt ? sqrt(t) : t;
}

__global__ void lz_reduce(const double* __restrict__ part, int m, int take_sqrt, double* __restrict__ out) {
  lz_reduce_block(part, m, take_sqrt, out);
}

// v_next = w / beta (written over w).
__global__ void lz_scale(int64_t n, const double* __restrict__ beta, double* __restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double b = *beta;
  if (i < n) w[i] = b > 0.0 ? w[i] / b : 0.0;
}

__global__ void lz_start(int64_t n, uint64_t seed, double* __restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (double)tbk_probe_sign(seed, i, 0) / sqrt((double)n);
}

// ---- many clusters: the same kernels, blockIdx.y = cluster ---------------------------------
struct LzJob {
  int n_atoms, B, nb, m;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* H;
  double* vecs;  // vp, v, w (n each), part (nb), alpha (m + 2), beta (m + 2)
  int64_t n;
  uint64_t seed;
};

__device__ __forceinline__ void lz_ptrs(const LzJob& j, int step, double*& vp, double*& v, double*& w) {
  // the rotation vp <- v, v <- w, w <- old vp of the single-cluster loop, by step parity mod 3
  double* base[3] = {j.vecs, j.vecs + j.n, j.vecs + 2 * j.n};
  vp = base[step % 3];
  v = base[(step + 1) % 3];
  w = base[(step + 2) % 3];
}

__global__ void lzb_start(const LzJob* __restrict__ jobs) {
  const LzJob j = jobs[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < j.n) j.vecs[j.n + i] = (double)tbk_probe_sign(j.seed, i, 0) / sqrt((double)j.n);
}

__global__ void lzb_spmv(const LzJob* __restrict__ jobs, int step) {
  const LzJob j = jobs[blockIdx.y];
  if (step >= j.m || (int)blockIdx.x >= j.nb) return;
  double *vp, *v, *w;
  lz_ptrs(j, step, vp, v, w);
  double* part = j.vecs + 3 * j.n;
  double* beta = part + j.nb + (j.m + 2);
  lz_spmv_cta(blockIdx.x, j.n_atoms, j.B, j.row_ptr, j.col, j.H, v, step ? vp : nullptr, beta + step, w, part);
}

__global__ void lzb_reduce(const LzJob* __restrict__ jobs, int step, int take_sqrt) {
  const LzJob j = jobs[blockIdx.y];
  if (step >= j.m) return;
  double* part = j.vecs + 3 * j.n;
  double* alpha = part + j.nb;
  double* beta = alpha + (j.m + 2);
  lz_reduce_block(part, j.nb, take_sqrt, take_sqrt ? beta + step + 1 : alpha + step);
}

__global__ void lzb_orth(const LzJob* __restrict__ jobs, int step) {
  const LzJob j = jobs[blockIdx.y];
  if (step >= j.m || (int)blockIdx.x >= j.nb) return;
  double *vp, *v, *w;
  lz_ptrs(j, step, vp, v, w);
  double* part = j.vecs + 3 * j.n;
  lz_orth_cta(blockIdx.x, j.n, v, part + j.nb + step, w, part);
}

__global__ void lzb_scale(const LzJob* __restrict__ jobs, int step) {
  const LzJob j = jobs[blockIdx.y];
  if (step >= j.m) return;
  double *vp, *v, *w;
  lz_ptrs(j, step, vp, v, w);
  const double* beta = j.vecs + 3 * j.n + j.nb + (j.m + 2);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double b = beta[step + 1];
  if (i < j.n) w[i] = b > 0.0 ? w[i] / b : 0.0;
}

// ---- host: tridiagonal eigen-analysis -------------------------------------------------------

// Number of eigenvalues of the tridiagonal (a, b) below x (Sturm sequence).
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double q = 1.0;
  const double tiny = 1e-300;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    q = (a[i] - x) - (i ? bb / q : 0.0);
    if (q == 0.0) q = -tiny;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// k-th smallest eigenvalue (0-based) by bisection.
static double tri_eig(const std::vector<double>& a, const std::vector<double>& b, int k) {
  const size_t m = a.size();
  double lo = INFINITY, hi = -INFINITY;
  for (size_t i = 0; i < m; ++i) {
    const double r = (i ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  const double scale = std::max(fabs(lo), fabs(hi)) + 1e-300;
  for (int it = 0; it < 200 && hi - lo > 4e-16 * scale; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, mid) > k) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// |last component| of the unit eigenvector of the tridiagonal for eigenvalue theta, by three
// steps of inverse iteration with a slightly shifted theta (Gaussian elimination with partial
// pivoting on the tridiagonal system).
static double tri_last_component(const std::vector<double>& a, const std::vector<double>& b, double theta) {
  const int m = (int)a.size();
  if (m == 1) return 1.0;
  double scale = 0.0;
  for (int i = 0; i < m; ++i) scale = std::max(scale, fabs(a[i]) + (i < m - 1 ? fabs(b[i]) : 0.0));
  const double sigma = theta + 1e-10 * (scale + 1e-300);
  std::vector<double> z(m, 1.0 / std::sqrt((double)m));
  for (int rep = 0; rep < 3; ++rep) {
    // rows: dl (sub), d (diag), du (super), du2 (fill-in)
    std::vector<double> dl(m, 0.0), d(m), du(m, 0.0), du2(m, 0.0), rhs = z;
    for (int i = 0; i < m; ++i) {
      d[i] = a[i] - sigma;
      if (i < m - 1) { du[i] = b[i]; dl[i] = b[i]; }
    }
    for (int i = 0; i < m - 1; ++i) {
      if (fabs(d[i]) >= fabs(dl[i])) {
        if (d[i] == 0.0) d[i] = 1e-300;
        const double f = dl[i] / d[i];
        d[i + 1] -= f * du[i];
        if (i < m - 2) du2[i] = 0.0;
        rhs[i + 1] -= f * rhs[i];
      } else {
        // swap rows i and i+1, then eliminate: the pivot row gains a second superdiagonal
        const double f = d[i] / dl[i];
        const double old_dnext = d[i + 1], old_du = du[i];
        d[i] = dl[i];
        du[i] = old_dnext;
        d[i + 1] = old_du - f * old_dnext;
        if (i < m - 2) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du2[i];
        }
        std::swap(rhs[i], rhs[i + 1]);
        rhs[i + 1] -= f * rhs[i];
      }
    }
    if (d[m - 1] == 0.0) d[m - 1] = 1e-300;
    std::vector<double> x(m);
    x[m - 1] = rhs[m - 1] / d[m - 1];
    if (m >= 2) x[m - 2] = (rhs[m - 2] - du[m - 2] * x[m - 1]) / d[m - 2];
    for (int i = m - 3; i >= 0; --i) x[i] = (rhs[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / d[i];
    double nrm = 0.0;
    for (double v : x) nrm += v * v;
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return 1.0;
    for (int i = 0; i < m; ++i) z[i] = x[i] / nrm;
  }
  return fabs(z[m - 1]);
}

void bounds_from_tridiagonal(const std::vector<double>& ha, const std::vector<double>& hb, int m,
                             double rel_margin, double* emin, double* emax);

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_spectral_bounds(tbk_ctx* ctx, const tbk_bsr* H, int32_t steps,
                                   double rel_margin, uint64_t seed, double* emin, double* emax) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && H && emin && emax, "NULL argument");
  TBK_CHECK_ARG(H->n_orb == 1 || H->n_orb == 9, "n_orb must be 1 or 9");
  TBK_CHECK_ARG(H->n_atoms >= 1 && H->row_ptr && H->col && H->val, "empty or NULL matrix");
  TBK_CHECK_ARG(steps >= 1 && steps <= 10000, "steps must be in [1, 10000]");
  TBK_CHECK_ARG(rel_margin >= 0.0 && std::isfinite(rel_margin), "rel_margin must be >= 0");
  DeviceGuard dg(ctx);
  const int64_t n = (int64_t)H->n_atoms * H->n_orb;
  const int m = (int)std::min<int64_t>(steps, n);
  const int nb = ceil_div(n, 256);
  double* vecs = (double*)scratch(ctx, WS_LANCZOS, sizeof(double) * (size_t)(3 * n + nb + 2 * (m + 2)));
  double *vp = vecs, *v = vecs + n, *w = vecs + 2 * n;
  double* part = vecs + 3 * n;
  double* alpha = part + nb;          // alpha[j], j < m
  double* beta = alpha + (m + 2);     // beta[j]: beta[0] = 0, beta[j+1] = ||w_j||
  TBK_CUDA(cudaMemsetAsync(beta, 0, sizeof(double) * (m + 2), ctx->stream));
  lz_start<<<nb, 256, 0, ctx->stream>>>(n, seed, v);
  post_launch(ctx, "lz_start");
  for (int j = 0; j < m; ++j) {
    lz_spmv<<<nb, 256, 0, ctx->stream>>>(H->n_atoms, H->n_orb, H->row_ptr, H->col, H->val, v,
                                         j ? vp : nullptr, beta + j, w, part);
    post_launch(ctx, "lz_spmv");
    lz_reduce<<<1, 256, 0, ctx->stream>>>(part, nb, 0, alpha + j);
    post_launch(ctx, "lz_reduce");
    lz_orth<<<nb, 256, 0, ctx->stream>>>(n, v, alpha + j, w, part);
    post_launch(ctx, "lz_orth");
    lz_reduce<<<1, 256, 0, ctx->stream>>>(part, nb, 1, beta + j + 1);
    post_launch(ctx, "lz_reduce");
    lz_scale<<<nb, 256, 0, ctx->stream>>>(n, beta + j + 1, w);
    post_launch(ctx, "lz_scale");
    double* t = vp;  // rotate: vprev <- v, v <- w, w <- old vprev
    vp = v;
    v = w;
    w = t;
  }
  std::vector<double> ha(m), hb(m + 1);
  TBK_CUDA(cudaMemcpyAsync(ha.data(), alpha, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(hb.data(), beta, sizeof(double) * (m + 1), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  bounds_from_tridiagonal(ha, hb, m, rel_margin, emin, emax);
  TBK_API_END
}

namespace tbk {
// Extreme Ritz values of the Lanczos tridiagonal (alpha ha[0..m), beta hb[1..m]) widened by their
// residual norms, then by rel_margin of the width on each side.
void bounds_from_tridiagonal(const std::vector<double>& ha, const std::vector<double>& hb, int m,
                             double rel_margin, double* emin, double* emax) {
  // Stop at the first (numerically) vanishing beta: the Krylov space is invariant there.
  int mm = m;
  double scale = 0.0;
  for (int j = 0; j < m; ++j) scale = std::max(scale, fabs(ha[j]) + fabs(hb[j + 1]));
  for (int j = 1; j < m; ++j)
    if (hb[j] <= 1e-14 * (scale + 1e-300)) { mm = j; break; }
  std::vector<double> a(ha.begin(), ha.begin() + mm), b(hb.begin() + 1, hb.begin() + mm);
  for (double x : a) TBK_CHECK_ARG(std::isfinite(x), "Lanczos produced a non-finite value");
  const double tmin = tri_eig(a, b, 0), tmax = tri_eig(a, b, mm - 1);
  const double bm = hb[mm];  // residual coupling of the last Lanczos vector
  const double rmin = fabs(bm) * tri_last_component(a, b, tmin);
  const double rmax = fabs(bm) * tri_last_component(a, b, tmax);
  double lo = tmin - rmin, hi = tmax + rmax;
  const double width = std::max(hi - lo, 1e-12 * std::max(1.0, std::max(fabs(lo), fabs(hi))));
  *emin = lo - rel_margin * width;
  *emax = hi + rel_margin * width;
  if (!(*emax > *emin)) *emax = *emin + 1e-12;
}
}  // namespace tbk

extern "C" int tbk_batched_spectral_bounds(tbk_ctx* ctx, int32_t n_clusters, const tbk_bsr* H,
                                           int32_t steps, double rel_margin, uint64_t seed,
                                           double* emin, double* emax) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && H && emin && emax, "NULL argument");
  TBK_CHECK_ARG(n_clusters >= 1, "n_clusters must be >= 1");
  TBK_CHECK_ARG(steps >= 1 && steps <= 10000, "steps must be in [1, 10000]");
  TBK_CHECK_ARG(rel_margin >= 0.0 && std::isfinite(rel_margin), "rel_margin must be >= 0");
  DeviceGuard dg(ctx);
  std::vector<LzJob> jobs(n_clusters);
  size_t tot = 0;
  int nb_max = 1, m_max = 1;
  for (int c = 0; c < n_clusters; ++c) {
    TBK_CHECK_ARG(H[c].n_orb == 1 || H[c].n_orb == 9, "n_orb must be 1 or 9");
    TBK_CHECK_ARG(H[c].n_atoms >= 1 && H[c].row_ptr && H[c].col && H[c].val, "empty or NULL matrix");
    LzJob& j = jobs[c];
    j.n_atoms = H[c].n_atoms;
    j.B = H[c].n_orb;
    j.n = (int64_t)j.n_atoms * j.B;
    j.m = (int)std::min<int64_t>(steps, j.n);
    j.nb = ceil_div(j.n, 256);
    j.row_ptr = H[c].row_ptr;
    j.col = H[c].col;
    j.H = H[c].val;
    j.seed = seed;
    j.vecs = nullptr;
    tot += (size_t)(3 * j.n + j.nb + 2 * (j.m + 2));
    nb_max = std::max(nb_max, j.nb);
    m_max = std::max(m_max, j.m);
  }
  double* vecs = (double*)scratch(ctx, WS_LANCZOS, sizeof(double) * tot);
  LzJob* d_jobs = (LzJob*)scratch(ctx, WS_MISC, sizeof(LzJob) * (size_t)n_clusters);
  size_t off = 0;
  for (int c = 0; c < n_clusters; ++c) {
    LzJob& j = jobs[c];
    j.vecs = vecs + off;
    off += (size_t)(3 * j.n + j.nb + 2 * (j.m + 2));
    // beta[0] = 0 (the first step has no previous vector)
    TBK_CUDA(cudaMemsetAsync(j.vecs + 3 * j.n + j.nb + (j.m + 2), 0, sizeof(double) * (j.m + 2), ctx->stream));
  }
  TBK_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(LzJob) * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  const dim3 g(nb_max, n_clusters), g1(1, n_clusters);
  lzb_start<<<g, 256, 0, ctx->stream>>>(d_jobs);
  post_launch(ctx, "lzb_start");
  for (int step = 0; step < m_max; ++step) {
    lzb_spmv<<<g, 256, 0, ctx->stream>>>(d_jobs, step);
    post_launch(ctx, "lzb_spmv");
    lzb_reduce<<<g1, 256, 0, ctx->stream>>>(d_jobs, step, 0);
    post_launch(ctx, "lzb_reduce");
    lzb_orth<<<g, 256, 0, ctx->stream>>>(d_jobs, step);
    post_launch(ctx, "lzb_orth");
    lzb_reduce<<<g1, 256, 0, ctx->stream>>>(d_jobs, step, 1);
    post_launch(ctx, "lzb_reduce");
    lzb_scale<<<g, 256, 0, ctx->stream>>>(d_jobs, step);
    post_launch(ctx, "lzb_scale");
  }
  std::vector<std::vector<double>> ha(n_clusters), hb(n_clusters);
  for (int c = 0; c < n_clusters; ++c) {
    const LzJob& j = jobs[c];
    ha[c].resize(j.m);
    hb[c].resize(j.m + 1);
    const double* alpha = j.vecs + 3 * j.n + j.nb;
    TBK_CUDA(cudaMemcpyAsync(ha[c].data(), alpha, sizeof(double) * j.m, cudaMemcpyDeviceToHost, ctx->stream));
    TBK_CUDA(cudaMemcpyAsync(hb[c].data(), alpha + (j.m + 2), sizeof(double) * (j.m + 1), cudaMemcpyDeviceToHost,
                             ctx->stream));
  }
  sync(ctx);
  for (int c = 0; c < n_clusters; ++c)
    bounds_from_tridiagonal(ha[c], hb[c], jobs[c].m, rel_margin, emin + c, emax + c);
  TBK_API_END
}
