// f2: the direct random estimates of the sampled density and energy-density matrices
// (Eq. poly_PQ with S = I; Eq. random_density):
//   M o P~ = (1/s) M o (X R^T),   M o Q~ = (1/s) M o (H X R^T),   X = p_f(H^) R = sum_k alpha_k C_k(H^) R,
// with alpha_k the (damped) Chebyshev coefficients of the Fermi function at a given mu and kT
// (Sec. II.B.1), R the s Rademacher probes and M the block pattern of H.  Unlike the adjoint's
// dOmega/dH these estimates are not symmetric; they are returned as computed.
//
// X comes from the backward (Clenshaw) form of the same sum, on the recurrence kernels unchanged:
//   b_{p-1} = alpha_{p-1} r,  b_k = alpha_k r + 2 H^ b_{k+1} - b_{k+2}  (k = p-2 .. 1),
//   X = alpha_0 r + H^ b_1 - b_2,
// p - 1 block products on two panels (each step is the fused step y_out = c H^ y_in + c_r r - y_prev
// with the probe regenerated in the kernel).  H X is one more product with H itself (H mapped with
// the bounds [-1, 1], for which H^ = H).  The two sampled products M o (X R^T) and M o (H X R^T)
// run on the tensor-core kernel for FP32 9x9 blocks (else on the plain outer-product kernel) with
// the probe block written once as a panel.
#include <vector>

#include "cheb.cuh"
#include "model.cuh"

namespace tbk {
void launch_forces(tbk_ctx* ctx, const DevModel& M, const double* pos, int n_atoms, const int32_t* row_ptr,
                   const int32_t* col, const int32_t* tr, const double* G, double* tq, double* F);
}  // namespace tbk

using namespace tbk;

extern "C" int tbk_direct_density(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model, const double* pos,
                                  const double* box, double emin, double emax, uint64_t probe_seed,
                                  int32_t n_probes, int32_t order, double mu, double kT, int32_t damping,
                                  int32_t flags, double* P, double* Q, double* forces) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr && H != nullptr, "NULL argument");
  TBK_CHECK_ARG(P || Q || forces, "nothing to compute: P, Q and forces are all NULL");
  TBK_CHECK_ARG(order >= 1, "order must be >= 1");
  TBK_CHECK_ARG(n_probes >= 4 && n_probes % 4 == 0, "n_probes must be a positive multiple of 4");
  TBK_CHECK_ARG((flags & ~(TBK_FP64 | TBK_PLAIN_KERNEL)) == 0, "unknown flag");
  TBK_CHECK_ARG(kT > 0.0, "kT must be positive");
  DeviceGuard dg(ctx);
  const int prec = (flags & TBK_FP64) ? TBK_FP64 : TBK_MIXED;
  DevModel Mdl{};
  if (forces) {
    Mdl = upload_model(ctx, model, box, WS_TABLE);
    TBK_CHECK_ARG(Mdl.kind == TBK_MODEL_SK, "forces need the Slater-Koster model");
    TBK_CHECK_ARG(pos != nullptr, "pos is NULL");
  }
  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  HOp op = prepare_hop(ctx, H, emin, emax, prec, WS_HHAT, err);
  const int p = order, s = n_probes, BB = op.B * op.B;
  const size_t esz = prec == TBK_MIXED ? 4 : 8;
  const size_t panel = (size_t)op.n_rows * s * esz;
  const int plain = (flags & TBK_PLAIN_KERNEL) ? 1 : 0;

  // coefficients alpha_k[f] (damped), to the host for the per-step scalars
  double* dcoef = (double*)scratch(ctx, WS_COEF, sizeof(double) * (size_t)p);
  coefficients(ctx, TBK_FN_FERMI, p, emin, emax, mu, kT, damping, dcoef);
  std::vector<double> c(p);
  TBK_CUDA(cudaMemcpyAsync(c.data(), dcoef, sizeof(double) * p, cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);

  // panels: two Clenshaw panels, X, the probe block
  char* base = (char*)scratch(ctx, WS_CHECKPOINTS, 4 * panel);
  void* B1 = base;
  void* B2 = base + panel;
  void* X = base + 2 * panel;
  void* R = base + 3 * panel;
  launch_scaled_probe(ctx, op, R, 1.0, probe_seed, s);

  auto step = [&](const void* yin, void* yprev, void* yout, double alpha, double c_r) {
    StepArgs a;
    a.yin = yin;
    a.yprev = yprev;
    a.yout = yout;
    a.alpha = alpha;
    a.c_r = c_r;
    a.seed = probe_seed;
    a.s = s;
    a.err = err;
    a.force_simple = plain;
    launch_step(ctx, op, a);
  };
  if (p == 1) {
    launch_scaled_probe(ctx, op, X, c[0], probe_seed, s);
  } else {
    // b_{p-1} in B1; then b_k alternates between B2 and B1 (b_k overwrites b_{k+2} in place)
    launch_scaled_probe(ctx, op, B1, c[p - 1], probe_seed, s);
    void *bk1 = B1, *bk2 = nullptr;        // b_{k+1}, b_{k+2}
    for (int k = p - 2; k >= 1; --k) {
      void* out = bk2 ? bk2 : B2;
      step(bk1, bk2, out, 2.0, c[k]);
      bk2 = bk1;
      bk1 = out;
    }
    // X = alpha_0 r + H^ b_1 - b_2
    step(bk1, bk2, X, 1.0, c[0]);
  }

  const bool mixed9 = prec == TBK_MIXED && op.B == 9 && !plain;
  const bool tc = mixed9 && tc_sddmm_eligible(ctx, op, s, tc_sddmm_max_row(ctx, op));
  auto sampled = [&](const void* Y, double* out) {
    TBK_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * (size_t)op.nnzb * BB, ctx->stream));
    if (tc) launch_tc_sddmm(ctx, op, Y, R, s, 1.0 / s, out, err);
    else launch_sddmm(ctx, op, Y, 0, probe_seed, R, s, 1.0 / s, out);
  };
  double* Pacc = P ? P : (double*)scratch(ctx, WS_GACC, sizeof(double) * (size_t)op.nnzb * BB * 2);
  if (P || forces) sampled(X, Pacc);
  if (forces) {
    // Hellmann-Feynman forces of the estimate, from its symmetric part
    int32_t* tr = (int32_t*)scratch(ctx, WS_TRANSPOSE, sizeof(int32_t) * (size_t)op.nnzb);
    launch_transpose_map(ctx, op.n_atoms, op.row_ptr, op.col, tr, err);
    double* Gs = (double*)scratch(ctx, WS_SEGMENT, sizeof(double) * (size_t)op.nnzb * BB);
    launch_symmetrize(ctx, op.nnzb, op.B, tr, Pacc, 1.0, Gs);
    double* tq = (double*)scratch(ctx, WS_MISC, sizeof(double) * 3 * (size_t)op.nnzb);
    launch_forces(ctx, Mdl, pos, op.n_atoms, op.row_ptr, op.col, tr, Gs, tq, forces);
  }
  if (Q) {
    // H X: H itself is H^ for the bounds [-1, 1]
    HOp h1 = prepare_hop(ctx, H, -1.0, 1.0, prec, WS_HHAT, err);
    void* HX = B1;
    StepArgs a;
    a.yin = X;
    a.yout = HX;
    a.alpha = 1.0;
    a.seed = probe_seed;
    a.s = s;
    a.err = err;
    a.force_simple = plain;
    launch_step(ctx, h1, a);
    sampled(HX, Q);
  }
  int herr = 0;
  TBK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(herr);
  if (herr & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in a recurrence kernel expired");
  TBK_CHECK_ARG(herr == 0, "the block pattern is not symmetric");
  TBK_API_END
}
