// a4: Chebyshev coefficients by Chebyshev-Gauss quadrature (Sec. II.B.1) and a8: chemical
// potential and observables from the moments (Sec. II.A Eqs. free_energy and density_matrix,
// with the traces replaced by the probe moments of Sec. II.C.2).
//
// With M nodes t_j = pi (j + 1/2)/M, x_j = cos t_j, e_j = emin (1 - x_j)/2 + emax (1 + x_j)/2:
//   alpha_k[h] = (2 - delta_k0)/M sum_j h(e_j) cos(k t_j),
// so any series sum_k d_k alpha_k[h] mu_k equals sum_j h(e_j) rho_j with the node weights
//   rho_j = (1/M) sum_k (2 - delta_k0) d_k mu_k cos(k t_j).
// The chemical-potential bisection therefore needs rho once and O(M) work per halving.
// cos(k t_j) = cos(pi m / (2M)) with m = k (2j + 1) mod 4M, read from a table of 4M entries.
#include <cmath>

#include "common.cuh"

namespace tbk {

__device__ __forceinline__ double fermi_fn(double e, double mu, double kT) {
  const double z = (e - mu) / kT;
  if (z > 0.0) {
    const double ez = exp(-z);
    return 2.0 * ez / (1.0 + ez);
  }
  return 2.0 / (1.0 + exp(z));
}
__device__ __forceinline__ double free_fn(double e, double mu, double kT) {
  const double u = -(e - mu) / kT;
  return -2.0 * kT * (fmax(u, 0.0) + log1p(exp(-fabs(u))));
}
__device__ __forceinline__ double node_energy(int j, int M, double emin, double emax) {
  const double x = cospi((j + 0.5) / M);
  return emin * (1.0 - x) * 0.5 + emax * (1.0 + x) * 0.5;
}

__device__ __forceinline__ void cos_entry(int m, int M, double* __restrict__ tab) {
  if (m < 4 * M) tab[m] = cospi((double)m / (2.0 * M));
}

__global__ void cos_table(int M, double* __restrict__ tab) {
  cos_entry(blockIdx.x * blockDim.x + threadIdx.x, M, tab);
}

__device__ __forceinline__ double damp_factor(int k, int p, int damping) {
  if (damping != TBK_DAMP_JACKSON) return 1.0;
  // Jackson kernel (Weisse et al., Rev. Mod. Phys. 78, 275 (2006), Eq. 71) with N = p
  const double q = M_PI / (p + 1);
  return ((p - k + 1) * cos(q * k) + sin(q * k) / tan(q)) / (p + 1);
}

// h_j = h(e_j) at the M quadrature nodes, once (the coefficient blocks all read them).
__global__ void node_values(int fn, int M, double emin, double emax, double mu, double kT,
                            double* __restrict__ hv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double e = node_energy(j, M, emin, emax);
  double h;
  if (fn == TBK_FN_FREE) h = free_fn(e, mu, kT);
  else {
    h = fermi_fn(e, mu, kT);
    if (fn == TBK_FN_ENERGY) h *= e;
  }
  hv[j] = h;
}

// One block per coefficient k.
__global__ void coeff_kernel(int p, int M, int damping, const double* __restrict__ tab,
                             const double* __restrict__ hv, double* __restrict__ out) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  double s = 0.0, c = 0.0;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const double h = hv[j];
    const int64_t m = ((int64_t)k * (2 * j + 1)) % (4 * (int64_t)M);
    const double y = h * tab[m] - c, t = s + y;
    c = (t - s) - y;
    s = t;
  }
  const double tot = tbk_block_sum(s, red);
  if (threadIdx.x == 0) out[k] = (k == 0 ? 1.0 : 2.0) / M * tot * damp_factor(k, p, damping);
}

// rho_j, one thread per node, fixed order over k.
__device__ __forceinline__ void rho_node(int j, const double* __restrict__ mom, int p, int M, int damping,
                                         const double* __restrict__ tab, double* __restrict__ rho) {
  if (j >= M) return;
  double s = 0.0, c = 0.0;
  const int64_t step = 2 * j + 1, period = 4 * (int64_t)M;
  int64_t m = 0;
  for (int k = 0; k < p; ++k) {
    const double w = (k == 0 ? 1.0 : 2.0) * damp_factor(k, p, damping) * mom[k];
    const double y = w * tab[m] - c, t = s + y;
    c = (t - s) - y;
    s = t;
    m += step;
    if (m >= period) m -= period;
  }
  rho[j] = s / M;
}

__global__ void rho_kernel(const double* __restrict__ mom, int p, int M, int damping,
                           const double* __restrict__ tab, double* __restrict__ rho) {
  rho_node(blockIdx.x * blockDim.x + threadIdx.x, mom, p, M, damping, tab, rho);
}

// One block: bisection for N(mu) = n_e (skipped when n_e < 0), then Omega, E, N.
// out = {mu, Omega, E, N, status} with status 1 when the bracket has no sign change.
__device__ void fermi_solve(const double* __restrict__ rho, int M, double emin, double emax,
                            double n_e, double mu_fixed, double kT, double* __restrict__ out) {
  __shared__ double red[32];
  __shared__ double bc;
  auto count = [&](double mu) {
    double s = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x)
      s += fermi_fn(node_energy(j, M, emin, emax), mu, kT) * rho[j];
    double t = tbk_block_sum(s, red);
    if (threadIdx.x == 0) bc = t;
    __syncthreads();
    t = bc;
    __syncthreads();
    return t;
  };
  double mu = mu_fixed;
  double status = 0.0;
  if (n_e >= 0.0) {
    double lo = emin, hi = emax;
    const double W = emax - emin;
    if (count(lo) > n_e || count(hi) < n_e) status = 1.0;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (count(mid) < n_e) lo = mid; else hi = mid;
      if (hi - lo < 1e-13 * W) break;
    }
    mu = 0.5 * (lo + hi);
  }
  double so = 0.0, se = 0.0, sn = 0.0;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const double e = node_energy(j, M, emin, emax);
    const double f = fermi_fn(e, mu, kT);
    so += free_fn(e, mu, kT) * rho[j];
    se += e * f * rho[j];
    sn += f * rho[j];
  }
  const double to = tbk_block_sum(so, red);
  __syncthreads();
  const double te = tbk_block_sum(se, red);
  __syncthreads();
  const double tn = tbk_block_sum(sn, red);
  if (threadIdx.x == 0) {
    out[0] = mu;
    out[1] = to;
    out[2] = te;
    out[3] = tn;
    out[4] = status;
  }
}

__global__ void fermi_kernel(const double* __restrict__ rho, int M, double emin, double emax,
                             double n_e, double mu_fixed, double kT, double* __restrict__ out) {
  fermi_solve(rho, M, emin, emax, n_e, mu_fixed, kT, out);
}

// ---- many clusters in three launches (blockIdx.y / blockIdx.x = cluster) ----

__global__ void cos_table_batched(const FermiJob* __restrict__ jobs, double* __restrict__ buf) {
  const FermiJob j = jobs[blockIdx.y];
  cos_entry(blockIdx.x * blockDim.x + threadIdx.x, j.M, buf + j.tab_off);
}

__global__ void rho_batched(const FermiJob* __restrict__ jobs, const double* __restrict__ mom, int damping,
                            double* __restrict__ buf) {
  const FermiJob j = jobs[blockIdx.y];
  rho_node(blockIdx.x * blockDim.x + threadIdx.x, mom + j.mom_off, j.p, j.M, damping, buf + j.tab_off,
           buf + j.rho_off);
}

__global__ void fermi_batched(const FermiJob* __restrict__ jobs, const double* __restrict__ buf,
                              double* __restrict__ res) {
  const FermiJob j = jobs[blockIdx.x];
  fermi_solve(buf + j.rho_off, j.M, j.emin, j.emax, j.n_e, 0.0, j.kT, res + 8 * (int64_t)blockIdx.x);
}

int quad_nodes(int p) { return std::max(4 * p, 256); }

void fermi_enqueue_batched(tbk_ctx* ctx, int n, const FermiJob* d_jobs, int M_max, const double* moments,
                           int damping, double* buf, double* res) {
  cos_table_batched<<<dim3(ceil_div(4 * (int64_t)M_max, 256), n), 256, 0, ctx->stream>>>(d_jobs, buf);
  post_launch(ctx, "cos_table_batched");
  rho_batched<<<dim3(ceil_div(M_max, 128), n), 128, 0, ctx->stream>>>(d_jobs, moments, damping, buf);
  post_launch(ctx, "rho_batched");
  fermi_batched<<<n, 1024, 0, ctx->stream>>>(d_jobs, buf, res);
  post_launch(ctx, "fermi_batched");
}

// cos table of 4M doubles in WS_NODES, followed by `extra` doubles of room for the caller.
const double* make_cos_table(tbk_ctx* ctx, int M, size_t extra = 0) {
  double* tab = (double*)scratch(ctx, WS_NODES, sizeof(double) * (4 * (size_t)M + extra));
  cos_table<<<ceil_div(4 * (int64_t)M, 256), 256, 0, ctx->stream>>>(M, tab);
  post_launch(ctx, "cos_table");
  return tab;
}

void coefficients(tbk_ctx* ctx, int fn, int p, double emin, double emax, double mu, double kT,
                  int damping, double* out) {
  TBK_CHECK_ARG(p >= 1 && p <= (1 << 22), "order out of range");
  TBK_CHECK_ARG(fn == TBK_FN_FERMI || fn == TBK_FN_ENERGY || fn == TBK_FN_FREE, "unknown function");
  TBK_CHECK_ARG(damping == TBK_DAMP_NONE || damping == TBK_DAMP_JACKSON, "unknown damping");
  TBK_CHECK_ARG(kT > 0.0 && std::isfinite(kT), "kT must be positive");
  TBK_CHECK_ARG(emax > emin, "need emax > emin");
  const int M = quad_nodes(p);
  const double* tab = make_cos_table(ctx, M, (size_t)M);
  double* hv = const_cast<double*>(tab) + 4 * (size_t)M;
  node_values<<<ceil_div(M, 256), 256, 0, ctx->stream>>>(fn, M, emin, emax, mu, kT, hv);
  post_launch(ctx, "node_values");
  coeff_kernel<<<p, 256, 0, ctx->stream>>>(p, M, damping, tab, hv, out);
  post_launch(ctx, "coeff_kernel");
}

// Enqueue the chemical-potential solve for one moment vector without synchronising: tab (4M
// doubles), rho (M doubles) and res (5 doubles: mu, Omega, E, N, status) are device buffers.
void fermi_enqueue(tbk_ctx* ctx, const double* moments, int order, double emin, double emax,
                   double n_electrons, double mu_fixed, double kT, int damping, double* tab,
                   double* rho, double* res) {
  TBK_CHECK_ARG(order >= 1 && order <= (1 << 22), "order out of range");
  TBK_CHECK_ARG(kT > 0.0 && std::isfinite(kT), "kT must be positive");
  TBK_CHECK_ARG(emax > emin, "need emax > emin");
  const int M = quad_nodes(order);
  cos_table<<<ceil_div(4 * (int64_t)M, 256), 256, 0, ctx->stream>>>(M, tab);
  post_launch(ctx, "cos_table");
  rho_kernel<<<ceil_div(M, 128), 128, 0, ctx->stream>>>(moments, order, M, damping, tab, rho);
  post_launch(ctx, "rho_kernel");
  fermi_kernel<<<1, 1024, 0, ctx->stream>>>(rho, M, emin, emax, n_electrons, mu_fixed, kT, res);
  post_launch(ctx, "fermi_kernel");
}

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_chebyshev_coefficients(tbk_ctx* ctx, int32_t fn, int32_t order, double emin,
                                          double emax, double mu, double kT, int32_t damping,
                                          double* out) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && out, "NULL argument");
  DeviceGuard dg(ctx);
  coefficients(ctx, fn, order, emin, emax, mu, kT, damping, out);
  TBK_API_END
}

extern "C" int tbk_fermi_level(tbk_ctx* ctx, const double* moments, int32_t order, double emin,
                               double emax, double n_electrons, double mu_fixed, double kT,
                               int32_t damping, double* out) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && moments && out, "NULL argument");
  TBK_CHECK_ARG(order >= 1 && order <= (1 << 22), "order out of range");
  TBK_CHECK_ARG(kT > 0.0 && std::isfinite(kT), "kT must be positive");
  TBK_CHECK_ARG(emax > emin, "need emax > emin");
  TBK_CHECK_ARG(damping == TBK_DAMP_NONE || damping == TBK_DAMP_JACKSON, "unknown damping");
  DeviceGuard dg(ctx);
  const int M = quad_nodes(order);
  const double* tab = make_cos_table(ctx, M);
  double* rho = (double*)scratch(ctx, WS_COEF, sizeof(double) * ((size_t)M + 8));
  double* res = rho + M;
  rho_kernel<<<ceil_div(M, 128), 128, 0, ctx->stream>>>(moments, order, M, damping, tab, rho);
  post_launch(ctx, "rho_kernel");
  fermi_kernel<<<1, 1024, 0, ctx->stream>>>(rho, M, emin, emax, n_electrons, mu_fixed, kT, res);
  post_launch(ctx, "fermi_kernel");
  double h[5];
  TBK_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  for (int i = 0; i < 4; ++i) out[i] = h[i];
  if (h[4] != 0.0)
    throw Error(TBK_ERR_NOCONV, "n_electrons is outside the range of the estimated N(mu) on [emin, emax]");
  TBK_API_END
}
