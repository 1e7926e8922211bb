// f4: the rational (pole) approximation of the sampled density and energy-density matrices
// with CGLS solves (Sec. II.B.2, Eq. rational_fit, Eq. rational_PQ with S = I).
//
// Poles and residues: the continued-fraction expansion of the Fermi function (Ozaki, Phys. Rev. B
// 75, 035123 (2007)): the positive eigenvalues b_p of the 2N x 2N symmetric tridiagonal matrix with
// off-diagonal 1/(2 sqrt((2m-1)(2m+1))) and the first components v_p of their eigenvectors give
// 1/(1 + e^u) = 1/2 + sum_p R_p [1/(u - i z_p) + 1/(u + i z_p)], z_p = 1/b_p, R_p = -v_p^2/(4 b_p^2),
// so that f(x) = 2/(1 + e^{(x-mu)/kT}) = 1 + 2 Re sum_p w_p/(x - zeta_p), zeta_p = mu + i kT z_p,
// w_p = 2 kT R_p (the residue-pole form of Eq. rational_fit plus the expansion's constant 1).
// The eigenproblem is solved on the host by the Jacobi rotation method (FP64, a few hundred rows).
//
// With X = f_r(H) R = R + 2 Re sum_p w_p g_p and (H - zeta_p) g_p = R (one complex system per pole
// and probe column), the estimates are M o P~ = (1/s) M o (X R^T), M o Q~ = (1/s) M o (H X R^T)
// (Eq. random_density).  Each system is solved by CGLS (CG on the normal equations, which keeps the
// structure of CG for the indefinite complex-shifted matrix), every probe column with its own step
// lengths; the poles run from the farthest from mu to the nearest, each solve starting from the
// previous pole's solution, as the paper orders them.  FP64 throughout: the condition numbers reach
// max|eps - mu| / (pi kT).  A complex panel is a real panel of 2s columns (real parts, then
// imaginary parts, per row), so H applies to it with the recurrence's FP64 block product (H mapped on
// the bounds [-1, 1], for which H^ = H), and the shift, the column norms and the updates are
// elementwise kernels.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cheb.cuh"
#include "model.cuh"

namespace tbk {
void launch_forces(tbk_ctx* ctx, const DevModel& M, const double* pos, int n_atoms, const int32_t* row_ptr,
                   const int32_t* col, const int32_t* tr, const double* G, double* tq, double* F);

// Symmetric eigenproblem by cyclic Jacobi rotations (host, FP64): eigenvalues in w, eigenvectors in
// the columns of V (row-major n x n).
static void jacobi_eigh(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a(i, i);
}

// (z_p, R_p), ascending z_p, of the continued-fraction expansion with n_pairs pole pairs.
void cfe_poles(int n_pairs, std::vector<double>& z, std::vector<double>& R) {
  const int m = 2 * n_pairs;
  std::vector<double> B((size_t)m * m, 0.0), w, V;
  for (int k = 1; k < m; ++k) {
    const double v = 1.0 / (2.0 * std::sqrt((2.0 * k - 1.0) * (2.0 * k + 1.0)));
    B[(size_t)(k - 1) * m + k] = B[(size_t)k * m + k - 1] = v;
  }
  jacobi_eigh(m, B, w, V);
  std::vector<std::pair<double, double>> zr;
  for (int i = 0; i < m; ++i)
    if (w[i] > 0) {
      const double v0 = V[i];  // row 0, column i
      zr.push_back({1.0 / w[i], -v0 * v0 / (4.0 * w[i] * w[i])});
    }
  std::sort(zr.begin(), zr.end());
  z.clear();
  R.clear();
  for (auto& e : zr) {
    z.push_back(e.first);
    R.push_back(e.second);
  }
}

// out = Hv - z v on complex panels (n_rows x 2s: real parts in columns [0, s), imaginary in
// [s, 2s)); Hv may alias out.
__global__ void shift_panel(int64_t n_rows, int s, double zr, double zi, const double* Hv,
                            const double* __restrict__ v, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows * s) return;
  const int64_t row = i / s;
  const int j = (int)(i - row * s);
  const int64_t ir = row * 2 * s + j, ii = ir + s;
  const double vr = v[ir], vi = v[ii];
  out[ir] = Hv[ir] - (zr * vr - zi * vi);
  out[ii] = Hv[ii] - (zr * vi + zi * vr);
}

// Per-column partial sums of |x_j|^2 over row blocks: part[rb * s + j] (fixed order within a block).
constexpr int NRM_BLOCKS = 152;
__global__ void col_norm_part(int64_t n_rows, int s, int64_t rpb, const double* __restrict__ x,
                              double* __restrict__ part) {
  const int rb = blockIdx.x;
  const int64_t r0 = rb * rpb, r1 = min(n_rows, r0 + rpb);
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      const double a = x[r * 2 * s + j], b = x[r * 2 * s + s + j];
      acc += a * a + b * b;
    }
    part[(int64_t)rb * s + j] = acc;
  }
}
__global__ void col_norm_reduce(int nrb, int s, const double* __restrict__ part, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  double acc = 0.0;
  for (int rb = 0; rb < nrb; ++rb) acc += part[(int64_t)rb * s + j];
  out[j] = acc;
}

// CGLS updates with per-column real coefficients: alpha_j = gamma_j / delta_j (0 when delta_j = 0).
__global__ void cgls_update_xr(int64_t n_rows, int s, const double* __restrict__ gamma,
                               const double* __restrict__ delta, const double* __restrict__ p,
                               const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows * 2 * s) return;
  const int j = (int)(i % (2 * s)) % s;
  const double a = delta[j] > 0.0 ? gamma[j] / delta[j] : 0.0;
  x[i] += a * p[i];
  r[i] -= a * q[i];
}
// p = sv + beta p, beta_j = gnew_j / gamma_j; then gamma <- gnew (by the caller's swap).
__global__ void cgls_update_p(int64_t n_rows, int s, const double* __restrict__ gnew,
                              const double* __restrict__ gamma, const double* __restrict__ sv,
                              double* __restrict__ p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows * 2 * s) return;
  const int j = (int)(i % (2 * s)) % s;
  const double b = gamma[j] > 0.0 ? gnew[j] / gamma[j] : 0.0;
  p[i] = sv[i] + b * p[i];
}
// X += 2 Re(w g) (X real n_rows x s, g complex).
__global__ void accumulate_pole(int64_t n_rows, int s, double wr, double wi, const double* __restrict__ g,
                                double* __restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows * s) return;
  const int64_t row = i / s;
  const int j = (int)(i - row * s);
  X[i] += 2.0 * (wr * g[row * 2 * s + j] - wi * g[row * 2 * s + s + j]);
}
// y -= x (panels of n elements).
__global__ void sub_panel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] -= x[i];
}
// complex panel c = real panel y (imaginary parts zero); or c = 0 when y is NULL.
__global__ void to_complex(int64_t n_rows, int s, const double* __restrict__ y, double* __restrict__ c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows * s) return;
  const int64_t row = i / s;
  const int j = (int)(i - row * s);
  c[row * 2 * s + j] = y ? y[i] : 0.0;
  c[row * 2 * s + s + j] = 0.0;
}

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_rational_density(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model, const double* pos,
                                    const double* box, uint64_t probe_seed, int32_t n_probes, double mu, double kT,
                                    int32_t n_pairs, double tol, int32_t max_iter, int32_t flags, double* P,
                                    double* Q, double* forces, double* info) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr && H != nullptr, "NULL argument");
  TBK_CHECK_ARG(P || Q || forces, "nothing to compute: P, Q and forces are all NULL");
  TBK_CHECK_ARG(n_probes >= 4 && n_probes <= 4096 && n_probes % 4 == 0,
                "n_probes must be a multiple of 4 in [4, 4096]");
  TBK_CHECK_ARG(n_pairs >= 1 && n_pairs <= 256, "n_pairs must be in [1, 256]");
  TBK_CHECK_ARG(tol > 0.0 && max_iter >= 1, "tol must be positive and max_iter >= 1");
  TBK_CHECK_ARG(flags == TBK_FP64, "the rational solves run in FP64 (flags = TBK_FP64)");
  TBK_CHECK_ARG(kT > 0.0, "kT must be positive");
  DeviceGuard dg(ctx);
  DevModel Mdl{};
  if (forces) {
    Mdl = upload_model(ctx, model, box, WS_TABLE);
    TBK_CHECK_ARG(Mdl.kind == TBK_MODEL_SK, "forces need the Slater-Koster model");
    TBK_CHECK_ARG(pos != nullptr, "pos is NULL");
  }
  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  // H itself: the mapped operator of the bounds [-1, 1]
  HOp op = prepare_hop(ctx, H, -1.0, 1.0, TBK_FP64, WS_HHAT, err);
  const int s = n_probes, BB = op.B * op.B;
  const int64_t nr = op.n_rows;
  const size_t rp_bytes = (size_t)nr * s * 8, cp_bytes = 2 * rp_bytes;
  // panels: R, X (real); g, r, sv, p, q (complex)
  char* base = (char*)scratch(ctx, WS_CHECKPOINTS, 2 * rp_bytes + 5 * cp_bytes);
  double* R = (double*)base;
  double* X = (double*)(base + rp_bytes);
  double* g = (double*)(base + 2 * rp_bytes);
  double* r = g + 2 * nr * s;
  double* sv = r + 2 * nr * s;
  double* pp = sv + 2 * nr * s;
  double* q = pp + 2 * nr * s;
  const int64_t rpb = (nr + NRM_BLOCKS - 1) / NRM_BLOCKS;
  const int nrb = (int)((nr + rpb - 1) / rpb);
  double* nb = (double*)scratch(ctx, WS_MISC, sizeof(double) * ((size_t)nrb * s + 8 * (size_t)s));
  double* part = nb;
  double* gamma = part + (size_t)nrb * s;
  double* delta = gamma + s;
  double* gnew = delta + s;
  double* rn = gnew + s;
  double* bn = rn + s;
  launch_scaled_probe(ctx, op, R, 1.0, probe_seed, s);
  TBK_CUDA(cudaMemcpyAsync(X, R, rp_bytes, cudaMemcpyDeviceToDevice, ctx->stream));

  const unsigned gr = (unsigned)((nr * s + 255) / 256), gc = (unsigned)((nr * 2 * s + 255) / 256);
  auto norms = [&](const double* x, double* out) {
    col_norm_part<<<nrb, 128, 0, ctx->stream>>>(nr, s, rpb, x, part);
    col_norm_reduce<<<ceil_div(s, 128), 128, 0, ctx->stream>>>(nrb, s, part, out);
    post_launch(ctx, "col_norms");
  };
  // out = (H - z) v on complex panels (out != v)
  auto apply = [&](const double* v, double zr, double zi, double* out) {
    StepArgs a;
    a.yin = v;
    a.yout = out;
    a.alpha = 1.0;
    a.s = 2 * s;
    a.err = err;
    a.force_simple = 1;
    launch_step(ctx, op, a);
    shift_panel<<<gr, 256, 0, ctx->stream>>>(nr, s, zr, zi, out, v, out);
    post_launch(ctx, "shift_panel");
  };
  std::vector<double> zp, Rp;
  cfe_poles(n_pairs, zp, Rp);
  to_complex<<<gr, 256, 0, ctx->stream>>>(nr, s, nullptr, g);
  post_launch(ctx, "to_complex");
  // ||b_j|| (b = R) once
  to_complex<<<gr, 256, 0, ctx->stream>>>(nr, s, R, q);
  post_launch(ctx, "to_complex");
  norms(q, bn);
  std::vector<double> hb(s), hr(s);
  TBK_CUDA(cudaMemcpyAsync(hb.data(), bn, sizeof(double) * s, cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  int64_t total_iter = 0;
  double worst = 0.0;
  for (int k = n_pairs - 1; k >= 0; --k) {
    const double zr = mu, zi = kT * zp[k];
    const double wr = 2.0 * kT * Rp[k], wi = 0.0;
    // r = b - A g (g: the previous pole's solution), sv = A^H r, p = sv, gamma = ||sv||^2
    apply(g, zr, zi, q);
    to_complex<<<gr, 256, 0, ctx->stream>>>(nr, s, R, r);
    post_launch(ctx, "to_complex");
    sub_panel<<<gc, 256, 0, ctx->stream>>>(nr * 2 * s, q, r);
    post_launch(ctx, "sub_panel");
    apply(r, zr, -zi, sv);
    TBK_CUDA(cudaMemcpyAsync(pp, sv, cp_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    norms(sv, gamma);
    int it = 0;
    for (; it < max_iter; ++it) {
      if (it % 8 == 0) {
        // convergence: every column's relative residual below tol
        norms(r, rn);
        TBK_CUDA(cudaMemcpyAsync(hr.data(), rn, sizeof(double) * s, cudaMemcpyDeviceToHost, ctx->stream));
        sync(ctx);
        double mx = 0.0;
        for (int j = 0; j < s; ++j) mx = std::max(mx, std::sqrt(hr[j] / std::max(hb[j], 1e-300)));
        if (mx < tol) break;
      }
      apply(pp, zr, zi, q);
      norms(q, delta);
      cgls_update_xr<<<gc, 256, 0, ctx->stream>>>(nr, s, gamma, delta, pp, q, g, r);
      post_launch(ctx, "cgls_update_xr");
      apply(r, zr, -zi, sv);
      norms(sv, gnew);
      cgls_update_p<<<gc, 256, 0, ctx->stream>>>(nr, s, gnew, gamma, sv, pp);
      post_launch(ctx, "cgls_update_p");
      std::swap(gamma, gnew);
    }
    total_iter += it;
    norms(r, rn);
    TBK_CUDA(cudaMemcpyAsync(hr.data(), rn, sizeof(double) * s, cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    for (int j = 0; j < s; ++j) worst = std::max(worst, std::sqrt(hr[j] / std::max(hb[j], 1e-300)));
    accumulate_pole<<<gr, 256, 0, ctx->stream>>>(nr, s, wr, wi, g, X);
    post_launch(ctx, "accumulate_pole");
  }
  if (info) {
    info[0] = (double)total_iter;
    info[1] = worst;
  }
  // sampled products with the probe block
  auto sampled = [&](const double* Y, double* out) {
    TBK_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * (size_t)op.nnzb * BB, ctx->stream));
    launch_sddmm(ctx, op, Y, 0, probe_seed, R, s, 1.0 / s, out);
  };
  double* Pacc = P ? P : (double*)scratch(ctx, WS_GACC, sizeof(double) * (size_t)op.nnzb * BB);
  if (P || forces) sampled(X, Pacc);
  if (forces) {
    int32_t* tr = (int32_t*)scratch(ctx, WS_TRANSPOSE, sizeof(int32_t) * (size_t)op.nnzb);
    launch_transpose_map(ctx, op.n_atoms, op.row_ptr, op.col, tr, err);
    double* Gs = (double*)scratch(ctx, WS_SEGMENT, sizeof(double) * (size_t)op.nnzb * BB);
    launch_symmetrize(ctx, op.nnzb, op.B, tr, Pacc, 1.0, Gs);
    double* tq = (double*)scratch(ctx, WS_LOCAL0, sizeof(double) * 3 * (size_t)op.nnzb);
    launch_forces(ctx, Mdl, pos, op.n_atoms, op.row_ptr, op.col, tr, Gs, tq, forces);
  }
  if (Q) {
    // H X, in the first complex panel's memory (a real panel of s columns)
    StepArgs a;
    a.yin = X;
    a.yout = g;
    a.alpha = 1.0;
    a.s = s;
    a.err = err;
    a.force_simple = 1;
    launch_step(ctx, op, a);
    sampled(g, Q);
  }
  int herr = 0;
  TBK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(herr);
  TBK_CHECK_ARG(herr == 0, "the block pattern is not symmetric");
  if (worst > tol)
    throw Error(TBK_ERR_NOCONV, "CGLS did not reach the tolerance in max_iter iterations (relative residual " +
                                    std::to_string(worst) + ")");
  TBK_API_END
}
