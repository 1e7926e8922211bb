// f1: the multi-colour probe ensemble (Sec. II.C.3) on the recurrence and the adjoint.
//
// The basis functions are split into colours such that two functions of one colour sit farther
// apart than a colouring radius: atom a has the Welsh-Powell colour c(a) (Sec. II.E, computed by
// tbk_welsh_powell on the neighbour pattern at that radius) and its orbital o the function colour
// c(a) n_orb + o, so q = n_colors n_orb function colours.  One sample of the ensemble has q
// columns; column k is nonzero exactly on the functions of colour k, with random signs there.  The
// mean of R_i R_i^T over samples is I, and only matrix elements between distinct functions of one
// colour enter the sampling error, so a local observable's variance drops with the radius.
//
// Probe block: column i q + k of sample i holds the sign of the plain Rademacher entry (row, i)
// (tbk_probe_sign) on the rows of colour k and zero elsewhere; columns from n_samples q up to the
// panel width are zero.  The estimator divides by the number of samples, not by the columns:
//   mu_k = (1/n_samples) sum_columns r^T C_k(H^) r.
// The block is written once as a panel in the recurrence precision and read where the probe
// enters (the first two forward steps, the source and outer product of the last two backward
// steps); every other step is the plain recurrence on the panel width, with the same kernels.
#include "cheb.cuh"

namespace tbk {

// out[row, col] of the coloured probe block (n_rows x S, row-major); *bad |= 1 if a colour is
// outside [0, n_colors).
template <typename T>
__global__ void colored_probe_panel(int64_t n_rows, int n_orb, int S, int q, int n_samples, int n_colors,
                                    uint64_t seed, const int32_t* __restrict__ atom_color, T* __restrict__ out,
                                    int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows * S) return;
  const int64_t row = i / S;
  const int c = (int)(i - row * S);
  const int ac = __ldg(atom_color + row / n_orb);
  T v = (T)0;
  if (ac < 0 || ac >= n_colors) {
    if (c == 0) atomicOr(bad, 1);
  } else {
    const int sample = c / q, k = c - sample * q;
    const int fc = ac * n_orb + (int)(row % n_orb);
    if (sample < n_samples && k == fc) v = (T)tbk_probe_sign(seed, (uint64_t)row, (uint64_t)sample);
  }
  out[i] = v;
}

// Validate the ensemble's arguments and write its probe block into scratch; returns the panel.
static void* colored_block(tbk_ctx* ctx, const tbk_bsr* H, int prec, uint64_t seed, const int32_t* atom_color,
                           int n_colors, int n_samples, int n_columns) {
  TBK_CHECK_ARG(H != nullptr, "H is NULL");
  TBK_CHECK_ARG(atom_color != nullptr, "atom_color is NULL");
  TBK_CHECK_ARG(H->n_orb == 1 || H->n_orb == 9, "n_orb must be 1 or 9");
  TBK_CHECK_ARG(H->n_atoms >= 1, "empty matrix");
  TBK_CHECK_ARG(n_colors >= 1 && n_samples >= 1, "n_colors and n_samples must be >= 1");
  const int64_t q = (int64_t)n_colors * H->n_orb;
  TBK_CHECK_ARG(q * n_samples <= n_columns, "n_columns is below n_samples * n_colors * n_orb");
  TBK_CHECK_ARG(n_columns % 4 == 0, "n_columns must be a multiple of 4");
  const int64_t n_rows = (int64_t)H->n_atoms * H->n_orb;
  const size_t esz = prec == TBK_MIXED ? 4 : 8;
  const size_t bytes = (size_t)n_rows * n_columns * esz;
  unsigned char* buf = (unsigned char*)scratch(ctx, WS_PROBES, bytes + 256);
  int* bad = (int*)(buf + bytes);
  TBK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
  const int64_t n = n_rows * n_columns;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (prec == TBK_MIXED)
    colored_probe_panel<float><<<grid, 256, 0, ctx->stream>>>(n_rows, H->n_orb, n_columns, (int)q, n_samples,
                                                              n_colors, seed, atom_color, (float*)buf, bad);
  else
    colored_probe_panel<double><<<grid, 256, 0, ctx->stream>>>(n_rows, H->n_orb, n_columns, (int)q, n_samples,
                                                               n_colors, seed, atom_color, (double*)buf, bad);
  post_launch(ctx, "colored_probe_panel");
  int hbad = 0;
  TBK_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  TBK_CHECK_ARG(hbad == 0, "an atom colour is outside [0, n_colors)");
  return buf;
}

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_colored_moments(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax,
                                   uint64_t probe_seed, const int32_t* atom_color, int32_t n_colors,
                                   int32_t n_samples, int32_t n_columns, int32_t order, int32_t flags,
                                   double* moments) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG(moments != nullptr, "moments is NULL");
  TBK_CHECK_ARG((flags & ~(TBK_FP64 | TBK_PLAIN_KERNEL)) == 0, "unknown flag");
  DeviceGuard dg(ctx);
  const int prec = (flags & TBK_FP64) ? TBK_FP64 : TBK_MIXED;
  const void* R0 = colored_block(ctx, H, prec, probe_seed, atom_color, n_colors, n_samples, n_columns);
  moments_sweep(ctx, H, emin, emax, probe_seed, n_columns, order, flags, moments, nullptr, R0, n_samples);
  TBK_API_END
}

extern "C" int tbk_colored_energies_and_forces(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model,
                                               const double* pos, const double* box, double emin, double emax,
                                               uint64_t probe_seed, const int32_t* atom_color, int32_t n_colors,
                                               int32_t n_samples, int32_t n_columns, int32_t order,
                                               double n_electrons, double kT, int32_t damping, int32_t flags,
                                               int64_t max_panel_bytes, double* moments, double* observables,
                                               double* G, double* forces) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr && observables != nullptr, "NULL argument");
  TBK_CHECK_ARG(order >= 1, "order must be >= 1");
  TBK_CHECK_ARG((flags & ~(TBK_WINDOWED | TBK_FUSED_ADJOINT | TBK_TC_OUTER)) == 0,
                "unknown flag (the coloured adjoint runs in mixed precision)");
  TBK_CHECK_ARG(kT > 0.0 && n_electrons >= 0.0, "kT must be positive and n_electrons >= 0");
  TBK_CHECK_ARG(H != nullptr, "H is NULL");
  HOp shape;
  shape.B = H->n_orb;
  shape.prec = TBK_MIXED;
  TBK_CHECK_ARG(fused_eligible(shape, n_columns, 0),
                "the coloured adjoint needs 9x9 blocks and n_columns of 128, 256 or 512");
  DeviceGuard dg(ctx);
  const void* R0 = colored_block(ctx, H, TBK_MIXED, probe_seed, atom_color, n_colors, n_samples, n_columns);
  energies_and_forces_doubled(ctx, H, model, pos, box, emin, emax, probe_seed, n_columns, order, n_electrons,
                              kT, damping, flags, max_panel_bytes, moments, observables, G, forces, R0,
                              n_samples);
  TBK_API_END
}
