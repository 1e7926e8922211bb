// The mapped operator H^ = (2H - (emax + emin) I)/(emax - emin) (Sec. II.B.1) in the layout the
// recurrence kernels read, and the fused block-SpMM step shared by the forward recurrence
// (moments) and the adjoint (Clenshaw) passes.
#pragma once
#include <functional>
#include <vector>

#include "common.cuh"

namespace tbk {

// Stored block of the mapped operator.  FP32 9x9 blocks are column-major: column l holds
// H^[0..8][l] padded to 12 floats, so a column is three 16-byte vectors and adjacent rows (i, i+1)
// form the float pairs of the packed f32x2 FMAs.  FP64 9x9 blocks are row-major with rows padded
// to 10 doubles.  RS is the padded stride of the leading index, BS the elements per block.
template <typename T, int B>
struct Layout {
  static constexpr bool COLMAJOR = B == 9 && sizeof(T) == 4;
  static constexpr int RS = B == 1 ? 1 : (sizeof(T) == 4 ? 12 : 10);
  static constexpr int BS = B * RS;
};

struct HOp {
  int n_atoms = 0, B = 0, prec = 0;  // prec: TBK_MIXED or TBK_FP64
  int64_t nnzb = 0, n_rows = 0;
  const int32_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const void* hv = nullptr;          // mapped blocks, Layout<T,B>
};

// Error-word bit set by the kernels that map H when a row stores no diagonal block (a, a): the
// shift of H^ = (2H - (emax + emin) I) / W lives on the diagonal blocks, so such a pattern is
// rejected rather than mapped wrongly.
constexpr int ERR_NO_DIAGONAL = 4;
inline void check_diagonal_flag(int herr) {
  if (herr & ERR_NO_DIAGONAL)
    throw Error(TBK_ERR_ARG, "a row of H stores no diagonal block; every row must hold its block (a, a)");
}

// Validate a tbk_bsr and build H^ in scratch slot `slot` with precision `prec`; a row without
// its diagonal block sets ERR_NO_DIAGONAL in *err (device).
HOp prepare_hop(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, int prec, Slot slot, int* err);

// One fused step over all rows and probes:
//   y_out = alpha * (H^ y_in) + c_r * r - y_prev
// where y_in is a panel or (cur_is_probe) the probe block r regenerated from the seed, and the
// y_prev term is present only when `yprev` is not NULL.  `yout` may equal `yprev` (in-place
// update: each element is read and then written by the same thread).
// With `partials` not NULL the CTA writes two FP64 partial sums at partials + 2 * cta:
//   [0] = sum y_out . y_in   (or sum y_out . r when `direct`),   [1] = sum y_out . y_out.
// Batched operators (many clusters merged block-diagonally): per-atom cluster index, per-cluster
// probe seed and first atom, so that each cluster's probes are those of a standalone run.
struct BatchRows {
  const int32_t* atom_cl = nullptr;
  const uint64_t* seed = nullptr;
  const int32_t* atom0 = nullptr;
};

struct StepArgs {
  const void* yin = nullptr;
  void* yprev = nullptr;
  void* yout = nullptr;
  int cur_is_probe = 0;
  double alpha = 2.0;
  double c_r = 0.0;
  uint64_t seed = 0;
  int s = 0;
  int direct = 0;
  double* partials = nullptr;
  int* err = nullptr;       // device flag raised (= 2) when a bounded wait expires
  int force_simple = 0;     // use the plain load/FMA kernel even where the TMA-fed one applies
  // TMA-fed kernel only: per-cluster probes, and partial sums per (atom, consumer warp) at
  // partials + 2 (a * CW + warp) instead of per CTA (CW = consumer warps, bulk_consumer_warps).
  BatchRows batch;
  int per_task = 0;
  int use_tc = 0;           // tensor-core (tcgen05) step where it applies
};
// Consumer warps of the TMA-fed step kernel for this operator and probe count (0 = not used).
int bulk_consumer_warps(const HOp& op, int s);
// CTAs a step launches for this operator and probe count.
int step_grid_ctas(tbk_ctx* ctx, const HOp& op, int s);
void launch_step(tbk_ctx* ctx, const HOp& op, const StepArgs& a);
// panel = c * r (probe block) for all rows.
void launch_scaled_probe(tbk_ctx* ctx, const HOp& op, void* panel, double c, uint64_t seed, int s);

// Allocation-free building blocks: bytes of the mapped operator, building it into caller
// memory, and the per-step partial-sum reduction into moments (flag bit 1 = spectrum error).
size_t mapped_h_bytes(const tbk_bsr* H, int prec);
HOp prepare_hop_into(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, int prec, void* dst, int* err);
void launch_moment_reduction(tbk_ctx* ctx, const double* partials, int nctas, int K, int order, int s,
                             int64_t n_rows, int direct, double* sums, double* moments, int* flag);

// ---- the adjoint of the doubled moments (adjoint.cu) ----
// A batch of clusters merged into one block-diagonal operator, sorted by K = order/2 descending:
// step t runs on the atoms of the clusters with K >= t (a prefix of the merged rows).
struct AdjBatch {
  BatchRows br;              // atom -> cluster, per-cluster probe seed and first atom (device)
  std::vector<int> K;        // per sorted cluster
  std::vector<int> n_at;     // atoms per sorted cluster
  const float4* cft = nullptr;  // device, (K_max + 1) x n_clusters: (probe, y_k, y_{k-1}, y_{k+1})
                                // coefficients of the source g_k of step k, zero past K_c
  int64_t pstride = 0;          // doubles of moment partials per forward step (per atom and warp)
  const int32_t* d_K = nullptr;  // device, K per sorted cluster (windowed outer products)
};
// Gacc += the unscaled gradient sum_k 2 y_k ybar_{k+1}^T + y_0 ybar_1^T on the pattern (scale 2/W
// afterwards).  Single system: get_coefs() returns c_0 .. c_{p-1} once y_1 .. y_{p/2} exist
// (with partials != NULL those forward steps also write their moment partial sums).  Batch: bt
// gives the per-cluster tables; p is unused; get_coefs, when given, is called once the forward
// sweep is done and fills bt->cft (its return value is ignored); partials, when given, receive
// per (atom, warp) sums of every forward step at partials + (t - 1) bt->pstride.
// probe_panel (single system only): the probe block y_0 stored as a panel (s columns) instead of
// regenerated from the seed, for probe ensembles other than plain Rademacher signs; s_norm: the
// number of samples the estimator divides by (0 = s).
// sched: where the outer products run: 0 inside each fused backward step, 1 summed over windows of
// steps by their own kernel, 2 on the tensor cores by a kernel after each backward step (single
// system, 9x9 blocks; falls back to 0 where the tensor-core kernel does not apply).
void adjoint_doubling(tbk_ctx* ctx, const HOp& op, uint64_t probe_seed, int s, int p,
                      const std::function<std::vector<double>()>& get_coefs, double* partials, int nctas,
                      int64_t max_panel_bytes, double* Gacc, int* err, int sched, const AdjBatch* bt,
                      const void* probe_panel = nullptr, int s_norm = 0);
// The tensor-core sampled outer products (tc_sddmm.cu): the longest block row of the pattern,
// whether the kernel takes this operator, and one launch Gacc += w y x^T on the pattern.
int tc_sddmm_max_row(tbk_ctx* ctx, const HOp& op);
bool tc_sddmm_eligible(tbk_ctx* ctx, const HOp& op, int s, int max_row);
void launch_tc_sddmm(tbk_ctx* ctx, const HOp& op, const void* y, const void* x, int s, double w, double* Gacc,
                     int* err);
// Pieces of the adjoint reused by the direct estimates (adjoint.cu): Chebyshev coefficients into
// device memory; Gacc += w sum_probes y[a rows] b[b rows]^T on every stored block (y or b FP32/FP64
// panels of the operator's precision; y_is_probe: y is the probe block regenerated from seed);
// the transpose map of a symmetric pattern; G = scale (Gacc + Gacc^T) / 2 blockwise.
void coefficients(tbk_ctx* ctx, int fn, int p, double emin, double emax, double mu, double kT,
                  int damping, double* out);
void launch_sddmm(tbk_ctx* ctx, const HOp& op, const void* y, int y_is_probe, uint64_t seed,
                  const void* b, int s, double w, double* Gacc);
void launch_transpose_map(tbk_ctx* ctx, int n_atoms, const int32_t* row_ptr, const int32_t* col,
                          int32_t* tr, int* err);
void launch_symmetrize(tbk_ctx* ctx, int64_t nnzb, int B, const int32_t* tr, const double* Gacc, double scale,
                       double* G);
// The adjoint's outer-product schedule for a call: the flag if one is given, else the tuned choice
// for this shape, else fused (0).
int outer_schedule(const tbk_ctx* ctx, const HOp& op, int s, int flags);
// The moments sweep of tbk_chebyshev_moments (per_probe: also each probe's moments).  With
// probe_panel the probe block y_0 is read from that panel (s columns, the precision of the
// recurrence) and the moments divide by s_norm samples; flags may not ask for direct moments then.
void moments_sweep(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, uint64_t probe_seed,
                   int32_t n_probes, int32_t order, int32_t flags, double* moments, double* per_probe,
                   const void* probe_panel = nullptr, int s_norm = 0);
// The one-call energies and forces of the doubled-moment adjoint (mixed, 9x9, s = 128/256/512),
// with the probe block regenerated from probe_seed or read from probe_panel (s_norm samples).
void energies_and_forces_doubled(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model, const double* pos,
                                 const double* box, double emin, double emax, uint64_t probe_seed, int s,
                                 int order, double n_electrons, double kT, int damping, int flags,
                                 int64_t max_panel_bytes, double* moments, double* observables, double* G,
                                 double* forces, const void* probe_panel, int s_norm);
bool fused_eligible(const HOp& op, int s, int plain);
void launch_batch_probe_panel(tbk_ctx* ctx, const HOp& op, const BatchRows& br, int s, void* out);

}  // namespace tbk
