/*
 * tbk.h -- C ABI of libtbk, a GB300 (sm_103a) implementation of the Chebyshev random-probe
 * path of arXiv 1812.05264 ("Assessment of localized and randomized algorithms for
 * electronic structure"): a Chebyshev expansion of the Fermi-Dirac and free-energy functions
 * of a block-sparse orthogonal tight-binding Hamiltonian, applied to a block of Rademacher
 * probe vectors, giving the grand potential, band energy, electron count, the sampled
 * density matrix on the sparsity pattern and Hellmann-Feynman forces.
 *
 * Conventions (all entry points):
 *  - Every call returns a tbk_status (0 = TBK_OK).  On failure tbk_last_error() returns a
 *    message for the calling thread; no exception, exit or trap crosses the ABI.
 *  - "device" pointers are CUDA global-memory addresses on the context's device; "host"
 *    pointers are ordinary CPU memory.  Inputs are owned by the caller and not retained after
 *    the call returns; outputs go into caller-allocated buffers of the stated size.
 *  - Work is enqueued on the context's stream.  Calls that return values in host memory
 *    synchronise that stream before returning; the others are asynchronous.
 *  - Energies are in the units of the model (eV for the Slater-Koster model), lengths in the
 *    units of the positions (Angstrom).
 *  - Block-sparse matrices use BSR with square n_orb x n_orb blocks (n_orb = 1 or 9): row_ptr
 *    (int32, n_atoms + 1), col (int32, nnzb, ascending within a row, the diagonal block
 *    present: a call that maps H to H^ fails with TBK_ERR_ARG on a row without it), values FP64
 *    row-major per block (nnzb * n_orb * n_orb).  Row i of a dense
 *    vector block is orbital i = n_orb * atom + orbital-in-atom; probe panels are row-major
 *    (n_rows x s, probe index fastest).
 *  - The library allocates its own scratch (panels, partial sums, checkpoints) from the
 *    context on first use and keeps it for later calls; tbk_destroy frees it.
 */
#ifndef TBK_H
#define TBK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TBK_OK = 0,
  TBK_ERR_ARG = -1,       /* invalid argument (null pointer, size, inconsistent shapes) */
  TBK_ERR_CUDA = -2,      /* a CUDA runtime call or kernel launch failed */
  TBK_ERR_OOM = -3,       /* device scratch could not be allocated */
  TBK_ERR_SPECTRUM = -4,  /* a recurrence left [-1, 1]: spectral bounds too narrow */
  TBK_ERR_NOCONV = -5,    /* bisection lost its sign change */
  TBK_ERR_TIMEOUT = -6    /* a bounded device-side wait gave up */
} tbk_status;

/* Precision / algorithm flags of the recurrence. */
#define TBK_MIXED 0            /* FP32 panels and FP32 mapped H, FP64 moment sums (default) */
#define TBK_FP64 1             /* FP64 panels and FP64 mapped H throughout */
#define TBK_MOMENTS_DIRECT 2   /* mu_k = <r, y_k> for every k instead of the doubling identity */
#define TBK_PLAIN_KERNEL 4     /* use the plain load/FMA step kernel instead of the TMA-fed one */
#define TBK_NO_GRAPH 8         /* batched calls: enqueue the kernels directly, no CUDA graph */
#define TBK_TENSOR_CORES 16    /* mixed mode: recurrence steps on the tensor cores (tcgen05, TF32 x3) */
#define TBK_WINDOWED 32        /* adjoint: outer products summed over windows of 4 steps by their own
                                  kernel instead of inside each backward step */
#define TBK_FUSED_ADJOINT 64   /* adjoint: outer products inside each backward step, whatever
                                  tbk_autotune chose */
#define TBK_TC_OUTER 128       /* adjoint (mixed, 9x9 blocks): outer products on the tensor cores
                                  (tcgen05, TF32 split three ways), one sampled-product kernel after
                                  each backward step */

/* Damping of the Chebyshev series. */
#define TBK_DAMP_NONE 0
#define TBK_DAMP_JACKSON 1

/* Which function the coefficients expand (tbk_chebyshev_coefficients). */
#define TBK_FN_FERMI 0         /* f(e) = 2 / (1 + exp((e - mu)/kT)) */
#define TBK_FN_ENERGY 1        /* e f(e) */
#define TBK_FN_FREE 2          /* g(e) = -2 kT ln(1 + exp(-(e - mu)/kT)) */

/* Tight-binding models (tbk_model.kind). */
#define TBK_MODEL_SK 1         /* Slater-Koster s/p/d two-centre blocks (n_orb = 9) */
#define TBK_MODEL_TABLE 2      /* blocks looked up by bond displacement (lattice models) */

typedef struct tbk_ctx tbk_ctx;

/* Model parameters of tbk_assemble_H.  Plain data; pointers are read during the call only. */
typedef struct {
  int32_t kind;              /* TBK_MODEL_SK or TBK_MODEL_TABLE */
  int32_t n_orb;             /* 9 for SK; 1 or 9 for TABLE */
  /* SK: bond integrals ss_sigma, sp_sigma, sd_sigma, pp_sigma, pp_pi, pd_sigma, pd_pi,
     dd_sigma, dd_pi, dd_delta, each scaled by exp(-sk_decay (r / sk_r0 - 1)); on-site
     energies of the s, p and d orbitals. */
  double sk_V[10];
  double sk_r0;
  double sk_decay;
  double onsite_spd[3];
  /* TABLE: n_disp bond displacements (host, n_disp x 3) and their blocks (host,
     n_disp x n_orb x n_orb); a bond matches an entry when every component differs by at
     most disp_tol.  Every off-diagonal neighbour pair must match exactly one entry. */
  int32_t n_disp;
  const double* disp;
  const double* disp_blocks;
  double disp_tol;
  /* Optional per-site on-site diagonal energies (device, n_atoms x n_orb), added to the
     diagonal blocks of either model; NULL for none. */
  const double* onsite_site;
} tbk_model;

/* A block-sparse matrix on the device (see the conventions above). */
typedef struct {
  int32_t n_atoms;
  int32_t n_orb;
  int64_t nnzb;
  const int32_t* row_ptr;    /* device, n_atoms + 1 */
  const int32_t* col;        /* device, nnzb */
  const double* val;         /* device, nnzb * n_orb * n_orb */
} tbk_bsr;

/* ---- context ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device` that enqueues on `stream` (a cudaStream_t; NULL =
   the legacy default stream).  *out receives the handle. */
int tbk_create(tbk_ctx** out, int device, void* stream);
/* Free the context and all its device scratch. */
int tbk_destroy(tbk_ctx* ctx);
/* Message of the last failed call on this thread ("" if none).  Valid until the next call. */
const char* tbk_last_error(void);
/* Number of kernel launches this context has issued (for launch accounting). */
int64_t tbk_launch_count(tbk_ctx* ctx);

/* Test of the bounded waits: the next TMA-fed recurrence step launched on ctx gets a producer
   that copies nothing, so its consumers' waits run out (each gives up after 2 s of wall time)
   and the call that launched it returns TBK_ERR_TIMEOUT.  Nothing faults; the context stays
   usable and the next calls compute normally.  Host-side only. */
int tbk_test_stall_next_step(tbk_ctx* ctx);
/* The same test for the fused adjoint step (the TMA-fed Clenshaw step with the sampled outer
   products): the next such launch on ctx gets a producer that copies nothing; its consumers give
   up after 2 s, the adjoint call returns TBK_ERR_TIMEOUT, and the context stays usable.  Host-side
   only. */
int tbk_test_stall_next_adjoint(tbk_ctx* ctx);

/* tbk_autotune: time, on this operator (9x9 blocks, mixed precision) with n_probes a multiple
   of 128, the probe chunk (128, 256 or 512 probes) per task of the TMA-fed recurrence step and
   the adjoint's outer-product schedule (fused into each backward step, or windows of 4 steps),
   and keep the faster of each in the context for every later call on an operator of the same
   shape (rows, stored blocks) and probe count.  The outer-product schedules timed are: fused into
   each backward step, windows of 4 steps, and the tensor cores after each step (TBK_TC_OUTER,
   where it applies).  All choices give the same results up to FP32 summation order.  choice:
   host, 2 ints {probes per task, schedule (0 fused, 1 windowed, 2 tensor cores)}.  Runs a few
   dozen kernels on scratch panels; synchronises the stream. */
int tbk_autotune(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, int32_t n_probes,
                 int32_t* choice);

/* Kernel families that tbk_kernel_timer can bracket with CUDA events. */
#define TBK_KERNEL_NONE 0
#define TBK_KERNEL_STEP 1     /* one recurrence step y_{k+1} = 2 H^ y_k - y_{k-1} (Eq. cheb_rec) */
#define TBK_KERNEL_BACKWARD 2 /* one adjoint step ybar_k = g_k + 2 H^ ybar_{k+1} - ybar_{k+2} */
#define TBK_KERNEL_WINDOW 3   /* the sampled outer products sum y_j ybar_{j+1}^T of a few steps */
/* Select the kernel families whose launches on ctx's stream are from now on bracketed by pairs
   of CUDA events: mask = sum of (1 << TBK_KERNEL_*) (0 switches timing off); earlier pairs are
   forgotten.  Launches captured into CUDA graphs are not bracketed.  Host-side only. */
int tbk_kernel_timer(tbk_ctx* ctx, int32_t mask);
/* Synchronise ctx's stream and return, for one family TBK_KERNEL_*, the summed device time
   (milliseconds) and the number of its bracketed launches since the last tbk_kernel_timer call.
   total_ms, launches: host pointers. */
int tbk_kernel_timer_read(tbk_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches);

/* ---- a1: neighbour list (Sec. II.A mask M; Sec. II.E uniform-cube cell lists) ---------- */

/* Pairs (i, j) with |r_j - r_i|^2 <= cutoff^2, self included, as CSR with ascending columns.
   r^2 is evaluated in FP64 as ((dx*dx) + (dy*dy)) + (dz*dz) with one rounding per operation;
   with a periodic box the displacement is the minimum image dx - L rint(dx / L).
   pos: device, n_atoms x 3 FP64.  box: host, 3 FP64 box lengths, or NULL for an open
   cluster (a periodic box must be longer than 2 cutoffs in every direction).
   row_ptr: device, n_atoms + 1 int32, always written.  col: device int32 of col_capacity
   entries, or NULL to count only.  *nnzb (host) receives the number of pairs; if col is not
   NULL and col_capacity < *nnzb the call fails with TBK_ERR_ARG and col is untouched.
   Synchronises the stream. */
int tbk_build_neighbors(tbk_ctx* ctx, const double* pos, int32_t n_atoms, const double* box,
                        double cutoff, int32_t* row_ptr, int32_t* col, int64_t col_capacity,
                        int64_t* nnzb);

/* tbk_batched_build_neighbors: tbk_build_neighbors for n_clusters open clusters in one call,
   with every pass run once over the atoms of all clusters; the same patterns, bit for bit.
   Host arrays: pos (device pointers, n_atoms[c] x 3 FP64 each), n_atoms (each >= 1), row_ptr
   (device pointers, n_atoms[c] + 1 int32 each, always written), col (device pointers with
   col_capacity[c] int32 each; the array may be NULL to count only), nnzb (out, pairs per
   cluster).  If a col entry is NULL or smaller than its cluster's pairs, the call fails with
   TBK_ERR_ARG after writing nnzb and row_ptr, and no col is touched.  Synchronises the stream
   twice. */
int tbk_batched_build_neighbors(tbk_ctx* ctx, int32_t n_clusters, const double* const* pos,
                                const int32_t* n_atoms, double cutoff, int32_t* const* row_ptr,
                                int32_t* const* col, const int64_t* col_capacity, int64_t* nnzb);

/* Welsh-Powell colouring of the atoms (Sec. II.E), for the multi-colour probe ensemble of
   Sec. II.C.3: the vertices are listed by non-increasing degree (equal degrees in index order),
   and each takes the smallest colour that none of its earlier-listed neighbours has.  This is
   the same colouring as building one colour class at a time down the list.  Two atoms of one
   colour are never neighbours in the graph.  Pass the pattern tbk_build_neighbors returns at
   the colouring radius (copied to the host), so that atoms of one colour are farther apart
   than that radius.  Host only: no context, no device memory, no stream.
   row_ptr: host, n_atoms + 1 int32, non-decreasing from 0.  col: host, row_ptr[n_atoms] int32
   in [0, n_atoms), strictly ascending within a row; self entries are ignored, and a pair must
   appear in both rows.  color: host, n_atoms int32, receives 0 .. *n_colors - 1.  *n_colors
   (host) receives the number of colours.  Bad sizes or indices, unsorted rows or a pair listed
   in one row only give TBK_ERR_ARG with color untouched.  O(n_atoms + nnz). */
int tbk_welsh_powell(int32_t n_atoms, const int32_t* row_ptr, const int32_t* col, int32_t* color,
                     int32_t* n_colors);

/* ---- a2: Hamiltonian assembly (Sec. II.A, Slater-Koster form of the NRL model) --------- */

/* Fill H (device, nnzb * n_orb^2 FP64) for the pattern (row_ptr, col) of n_atoms atoms at pos
   (device FP64 n_atoms x 3; box as in tbk_build_neighbors).  Off-diagonal block (a, b) is the
   model's block for the bond d = R_b - R_a; diagonal blocks carry the on-site energies. */
int tbk_assemble_H(tbk_ctx* ctx, const tbk_model* model, const double* pos, int32_t n_atoms,
                   const double* box, const int32_t* row_ptr, const int32_t* col, int64_t nnzb,
                   double* H);

/* ---- a3: spectral bounds (Sec. II.B.1 spectral interval [e_min, e_max]) ----------------- */

/* FP64 Lanczos with `steps` iterations from a Rademacher start vector drawn from `seed`.  The
   bounds are the extreme Ritz values widened by their residual norms, then by rel_margin times
   the width on each side.  emin, emax: host.  Synchronises the stream. */
int tbk_spectral_bounds(tbk_ctx* ctx, const tbk_bsr* H, int32_t steps, double rel_margin,
                        uint64_t seed, double* emin, double* emax);
/* tbk_batched_spectral_bounds: tbk_spectral_bounds for every cluster of a batch (host array H
   of n_clusters matrices), the Lanczos steps of all clusters in one launch per kernel and step;
   each cluster gets the bounds tbk_spectral_bounds gives it alone.  emin, emax: host,
   n_clusters each.  Synchronises the stream once. */
int tbk_batched_spectral_bounds(tbk_ctx* ctx, int32_t n_clusters, const tbk_bsr* H, int32_t steps,
                                double rel_margin, uint64_t seed, double* emin, double* emax);

/* ---- a4: Chebyshev coefficients (Sec. II.B.1) ------------------------------------------- */

/* out (device, order FP64) = the first `order` Chebyshev coefficients of fn on [emin, emax]
   by max(4 order, 256)-point Chebyshev-Gauss quadrature, times the damping factors. */
int tbk_chebyshev_coefficients(tbk_ctx* ctx, int32_t fn, int32_t order, double emin,
                               double emax, double mu, double kT, int32_t damping, double* out);

/* ---- a5-a7: fused recurrence and moments (Sec. II.B.1 Eq. poly_PQ; Sec. II.C.2) -------- */

/* moments (device, order FP64) = (1/s) sum_i r_i^T C_k(H^) r_i for k < order, with
   H^ = (2H - (emax + emin) I)/(emax - emin) and s = n_probes Rademacher probes r_i whose entry
   (row, j) is the sign of the top bit of SplitMix64 output number (row 2^32 + j + 1) of a stream
   seeded with probe_seed.  The probes are regenerated inside the kernels and never stored.
   flags: TBK_MIXED or TBK_FP64, optionally | TBK_MOMENTS_DIRECT | TBK_PLAIN_KERNEL |
   TBK_TENSOR_CORES.  n_probes must be a multiple of 4; in mixed mode with 9x9 blocks and
   n_probes a multiple of 128 the steps stream neighbour tiles through shared memory with bulk
   (TMA) copies, and with TBK_TENSOR_CORES the block products run as tcgen05 TF32 MMAs with a
   three-way split (head x head + head x rest + rest x head, FP32 accuracy).  TBK_ERR_TIMEOUT
   reports an expired bounded wait inside those kernels.  Fails with TBK_ERR_SPECTRUM if a panel grows beyond the bound that holds
   when the spectrum of H^ lies in [-1, 1]. */
int tbk_chebyshev_moments(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax,
                          uint64_t probe_seed, int32_t n_probes, int32_t order, int32_t flags,
                          double* moments);

/* Per-probe moments (Sec. II.C.2: the random-probe estimate is the mean of independent
   single-probe estimates, so their spread gives its statistical error, which falls as
   1/sqrt(n_probes)).  per_probe (device, order x n_probes FP64, k-major:
   per_probe[k * n_probes + i]) = r_i^T C_k(H^) r_i, whose mean over i is the moment mu_k;
   moments (device, order FP64, or NULL) receives tbk_chebyshev_moments' result from the same
   sweep.  Arguments, flags, probes and errors are those of tbk_chebyshev_moments.  After every
   recurrence step a column-dot kernel reads the new panel and the previous one, and the
   doubling identities (or, with TBK_MOMENTS_DIRECT, r_i . y_k) give each probe's moments:
   about 2/3 more panel traffic than tbk_chebyshev_moments.  The per-probe sums are added in a
   fixed order; repeated calls give identical results.  The standard error of an observable
   sum_k c_k mu_k is the standard deviation over i of sum_k c_k per_probe[k][i] divided by
   sqrt(n_probes). */
int tbk_chebyshev_probe_moments(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax,
                                uint64_t probe_seed, int32_t n_probes, int32_t order, int32_t flags,
                                double* moments, double* per_probe);

/* ---- a8: chemical potential and observables (Sec. II.A Eqs. free_energy, density_matrix)

   From the moments of tbk_chebyshev_moments: N(mu) = sum_k d_k alpha_k[f] mu_k with damping
   factors d_k is solved for N(mu) = n_electrons by bisection on [emin, emax] (stopping when
   the bracket is narrower than 1e-13 (emax - emin) or after 200 halvings; result = midpoint).
   out (host, 4 FP64) = {mu, Omega, E, N} with Omega = sum d_k beta_k[g] mu_k and
   E = sum d_k alpha_k[e f] mu_k.  If n_electrons < 0 the bisection is skipped and mu_fixed is
   used.  moments: device.  Synchronises the stream. */
int tbk_fermi_level(tbk_ctx* ctx, const double* moments, int32_t order, double emin,
                    double emax, double n_electrons, double mu_fixed, double kT,
                    int32_t damping, double* out);

/* ---- a9-a10: sampled density matrix and forces (Sec. II.D Eq. polynomial_response) -----

   The analytic derivative of the probe estimate Omega^ = (1/s) sum_i r_i^T q(H^) r_i,
   q = sum_k d_k beta_k[g] C_k, with the bounds held fixed:
     G = dOmega^/dH = (2/W)(1/s) sum_i sum_{j<order-1} y_ij x_ij^T on the pattern of H,
     y_ij = C_j(H^) r_i,  x_ij = (2 - delta_j0) sum_{k>j} d_k beta_k U_{k-j-1}(H^) r_i,
   returned symmetrised, G_ab <- (G_ab + G_ba^T)/2.  In mixed precision with 9x9 blocks and
   n_probes 128, 256 or 512 the same gradient is taken through the doubled moments
   mu_2k = 2<y_k, y_k>/s - mu_0, mu_2k-1 = 2<y_k, y_k-1>/s - mu_1, which needs y_j only up to
   j = order/2.  The panels y_j are recomputed from checkpoints when they do not fit in
   max_panel_bytes of scratch (0 = what the device has free, less a reserve).
   G: device, nnzb * n_orb^2 FP64, or NULL.  forces: device, n_atoms x 3 FP64, or NULL;
   F_c = -sum_ab <G_ab, dH_ab/dR_c> needs model->kind == TBK_MODEL_SK and pos (device) / box as
   in tbk_assemble_H.  flags: TBK_MIXED or TBK_FP64, optionally | TBK_PLAIN_KERNEL |
   TBK_WINDOWED, TBK_FUSED_ADJOINT or TBK_TC_OUTER (all give the same G up to FP32 summation
   order; without any, the schedule tbk_autotune chose for this shape, else fused). */
int tbk_density_and_forces(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model,
                           const double* pos, const double* box, double emin, double emax,
                           uint64_t probe_seed, int32_t n_probes, int32_t order, double mu,
                           double kT, int32_t damping, int32_t flags, int64_t max_panel_bytes,
                           double* G, double* forces);

/* tbk_energies_and_forces: tbk_chebyshev_moments + tbk_fermi_level + tbk_density_and_forces in
   one call, for the same results.  In mixed precision with 9x9 blocks and n_probes 128, 256 or
   512 the forward sweep of the adjoint produces the moments as it goes, so no separate moment
   pass runs.  moments: device, order doubles, or NULL.  observables: host, 4 doubles {mu, Omega,
   E, N}.  G, forces as in tbk_density_and_forces (either may be NULL).  flags: TBK_MIXED or
   TBK_FP64, optionally | TBK_PLAIN_KERNEL | TBK_WINDOWED | TBK_FUSED_ADJOINT | TBK_TC_OUTER.
   Synchronises the stream. */
int tbk_energies_and_forces(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model,
                            const double* pos, const double* box, double emin, double emax,
                            uint64_t probe_seed, int32_t n_probes, int32_t order,
                            double n_electrons, double kT, int32_t damping, int32_t flags,
                            int64_t max_panel_bytes, double* moments, double* observables,
                            double* G, double* forces);

/* ---- a11: batches of clusters ------------------------------------------------------------

   tbk_batched_moments: the moments of n_clusters independent clusters (each with its own H,
   spectral interval, probe seed and order) in one launch per recurrence step.  The clusters'
   mapped operators are merged block-diagonally, sorted by step count so that the clusters still
   running form a prefix of the rows; each cluster keeps its own probe stream, so its moments
   equal those of tbk_chebyshev_moments on it alone (mixed precision).  H: host array of
   n_clusters descriptors (9x9 blocks).  emin, emax, seeds, orders: host arrays.  moments:
   device, sum(orders) doubles, cluster c at offset sum_{c' < c} orders[c'].  n_probes: a
   multiple of 128.  flags: 0 or TBK_MOMENTS_DIRECT, optionally | TBK_NO_GRAPH.  The step
   sequence is captured into a CUDA graph on the first call and replayed while the arguments
   stay the same.  Synchronises the stream. */
int tbk_batched_moments(tbk_ctx* ctx, int32_t n_clusters, const tbk_bsr* H, const double* emin,
                        const double* emax, const uint64_t* seeds, int32_t n_probes,
                        const int32_t* orders, int32_t flags, double* moments);

/* tbk_batched_fermi_level: tbk_fermi_level for every cluster of a batch (moments laid out as
   tbk_batched_moments writes them); host arrays orders, emin, emax, n_electrons, kT; out: host,
   4 doubles {mu, Omega, E, N} per cluster.  Synchronises the stream once. */
int tbk_batched_fermi_level(tbk_ctx* ctx, int32_t n_clusters, const double* moments,
                            const int32_t* orders, const double* emin, const double* emax,
                            const double* n_electrons, const double* kT, int32_t damping,
                            double* out);

/* tbk_batched_density_and_forces: tbk_density_and_forces for every cluster of a batch, with
   the backward sweep of all clusters in one launch per step (merged operator as in
   tbk_batched_moments; each cluster joins the sweep at its own order).  Host arrays: H, pos
   (device pointers, n_atoms x 3 each; open clusters), emin, emax, seeds, orders, mu, kT, G and
   forces (device pointers or NULL entries; either array may be NULL).  n_probes 128, 256 or 512
   for the one-launch path; other shapes run the clusters one after another.  flags: 0 (mixed),
   optionally TBK_WINDOWED.  max_panel_bytes as in tbk_density_and_forces: the one-launch path
   keeps every panel y_j when they fit, each stored with only the rows of the clusters still
   running at step j - 1, else it replays full-size panels from checkpoints.  Synchronises the
   stream. */
int tbk_batched_density_and_forces(tbk_ctx* ctx, int32_t n_clusters, const tbk_bsr* H,
                                   const tbk_model* model, const double* const* pos,
                                   const double* emin, const double* emax, const uint64_t* seeds,
                                   int32_t n_probes, const int32_t* orders, const double* mu,
                                   const double* kT, int32_t damping, int32_t flags,
                                   int64_t max_panel_bytes, double* const* G,
                                   double* const* forces);

/* tbk_batched_energies_and_forces: tbk_batched_moments + tbk_batched_fermi_level +
   tbk_batched_density_and_forces in one call, for the same results.  On the one-launch path the
   forward sweep of the batched adjoint produces every cluster's moments as it goes, so no
   separate moment pass runs.  n_electrons: host, per cluster.  moments: device, laid out as
   tbk_batched_moments writes them, or NULL.  observables: host, 4 doubles {mu, Omega, E, N}
   per cluster.  G, forces as in tbk_batched_density_and_forces (either may be NULL).  n_probes
   a multiple of 128; flags: 0 (mixed), optionally TBK_WINDOWED.  Synchronises the stream. */
int tbk_batched_energies_and_forces(tbk_ctx* ctx, int32_t n_clusters, const tbk_bsr* H,
                                    const tbk_model* model, const double* const* pos,
                                    const double* emin, const double* emax, const uint64_t* seeds,
                                    int32_t n_probes, const int32_t* orders,
                                    const double* n_electrons, const double* kT, int32_t damping,
                                    int32_t flags, int64_t max_panel_bytes, double* moments,
                                    double* observables, double* const* G, double* const* forces);

/* ---- f1: the multi-colour probe ensemble (Sec. II.C.3; colours from Sec. II.E) ----------

   The basis functions are split into colours so that two functions of one colour sit farther
   apart than a colouring radius: atom a has colour atom_color[a] in [0, n_colors) (e.g. from
   tbk_welsh_powell on the pattern at that radius) and its orbital o the function colour
   atom_color[a] * n_orb + o, q = n_colors * n_orb colours in all.  Sample i of the ensemble has q
   columns: column i q + k is nonzero exactly on the functions of colour k, where its entry is the
   plain probe sign of (row, i) (the Rademacher entry of tbk_chebyshev_moments for probe i).  The
   panel has n_columns >= n_samples q columns (a multiple of 4; the ones past n_samples q are zero,
   so a width of 128, 256 or 512 takes the TMA-fed and fused kernels), and the estimator divides by
   the number of samples: mu_k = (1/n_samples) sum_columns r^T C_k(H^) r.  Its mean over samples is
   the trace of C_k(H^); only matrix elements between distinct functions of one colour enter its
   variance (Eq. sampling_error with the ensemble's deviation matrix).  The probe block is written
   once into library scratch in the recurrence precision and read where the probe enters.
   atom_color: device, n_atoms int32; a colour outside [0, n_colors) gives TBK_ERR_ARG. */

/* tbk_colored_moments: the moments of tbk_chebyshev_moments (doubled; flags TBK_MIXED or TBK_FP64,
   optionally | TBK_PLAIN_KERNEL) for the multi-colour ensemble.  moments: device, order FP64. */
int tbk_colored_moments(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, uint64_t probe_seed,
                        const int32_t* atom_color, int32_t n_colors, int32_t n_samples, int32_t n_columns,
                        int32_t order, int32_t flags, double* moments);

/* tbk_colored_energies_and_forces: tbk_energies_and_forces (one call: moments from the adjoint's
   forward sweep, mu, Omega, E, N, the sampled density matrix G = dOmega^/dH on the pattern and the
   forces) for the multi-colour ensemble.  Mixed precision with 9x9 blocks and n_columns of 128, 256
   or 512 (the doubled-moment adjoint); flags 0, TBK_WINDOWED, TBK_FUSED_ADJOINT or
   TBK_TC_OUTER.  Other
   arguments and outputs as in tbk_energies_and_forces.  Synchronises the stream. */
int tbk_colored_energies_and_forces(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model,
                                    const double* pos, const double* box, double emin, double emax,
                                    uint64_t probe_seed, const int32_t* atom_color, int32_t n_colors,
                                    int32_t n_samples, int32_t n_columns, int32_t order,
                                    double n_electrons, double kT, int32_t damping, int32_t flags,
                                    int64_t max_panel_bytes, double* moments, double* observables,
                                    double* G, double* forces);

/* ---- f2: direct random estimates of the sampled density matrices (Eq. poly_PQ, S = I;
   Eq. random_density) -----------------------------------------------------------------------

   tbk_direct_density: at a given chemical potential mu and temperature kT,
     P (device, nnzb * n_orb^2 FP64, or NULL) = M o P~,  P~ = (1/s) X R^T,
     Q (device, same size, or NULL)           = M o Q~,  Q~ = (1/s) H X R^T,
   with X = sum_{k < order} d_k alpha_k[f] C_k(H^) R (f the Fermi function of tbk_fermi_level at
   mu, kT; d_k the damping factors), R the n_probes Rademacher probes of tbk_chebyshev_moments
   and M the block pattern of H.  Blocks are laid out as H's values; the estimates are not
   symmetric and are returned as computed.  forces (device, n_atoms x 3 FP64, or NULL): the
   Hellmann-Feynman forces -sum_ab <P_ab, dH_ab/dR_c> from the symmetric part of M o P~ (needs
   model->kind == TBK_MODEL_SK, pos and box as in tbk_assemble_H).  X is formed by the backward
   (Clenshaw) form of the sum: order - 1 fused block products.  flags: TBK_MIXED or TBK_FP64,
   optionally | TBK_PLAIN_KERNEL.  Synchronises the stream. */
int tbk_direct_density(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model, const double* pos,
                       const double* box, double emin, double emax, uint64_t probe_seed,
                       int32_t n_probes, int32_t order, double mu, double kT, int32_t damping,
                       int32_t flags, double* P, double* Q, double* forces);

/* ---- f3: the local approximation (Sec. II.C.1, Eq. local_density, S = I) ----------------

   tbk_local_density: for every atom a, the region R_a of the atoms within r_max of a (the mask
   M_L(r_max), pairs at exactly r_max included, as tbk_build_neighbors counts them) gives the
   local operator H_a = H restricted to R_a; the n_orb columns of a of
     P~_L = L_a p_f(H_a) L_a^T E_a   and   Q~_L = L_a H_a p_f(H_a) L_a^T E_a
   (E_a the unit vectors of a's functions, p_f the order-term Chebyshev expansion of the Fermi
   function at mu, kT on [emin, emax] with damping, as tbk_chebyshev_coefficients gives it) are
   kept on the pattern of H: block (b, a) of P (device, nnzb * n_orb^2 FP64, or NULL) holds rows b
   of column block a, likewise Q.  The result is not symmetric (each column comes from its own
   local problem).  Every stored block (b, a) of H must join atoms at most r_max apart
   (TBK_ERR_ARG otherwise).  pos: device, n_atoms x 3 FP64; box as in tbk_build_neighbors.  All
   local problems run as one block-diagonal operator (order - 1 block products).  flags:
   TBK_MIXED or TBK_FP64.  Synchronises the stream. */
int tbk_local_density(tbk_ctx* ctx, const tbk_bsr* H, const double* pos, const double* box, double r_max,
                      double emin, double emax, int32_t order, double mu, double kT, int32_t damping,
                      int32_t flags, double* P, double* Q);

/* ---- f4: the rational (pole) approximation with CGLS solves (Sec. II.B.2, Eq. rational_fit,
   Eq. rational_PQ with S = I) -----------------------------------------------------------------

   tbk_rational_density: f(x) = 2 / (1 + exp((x - mu)/kT)) is replaced by the n_pairs-pole-pair
   continued-fraction expansion of the Fermi function (Ozaki, Phys. Rev. B 75, 035123 (2007)),
     f_r(x) = 1 + 2 Re sum_p w_p / (x - zeta_p),   zeta_p = mu + i kT z_p,  w_p = 2 kT R_p,
   with z_p = 1/b_p and R_p = -v_p^2/(4 b_p^2) from the positive eigenvalues b_p and the first
   eigenvector components v_p of the 2 n_pairs square tridiagonal matrix with off-diagonal
   1/(2 sqrt((2m-1)(2m+1))).  Then X = f_r(H) R = R + 2 Re sum_p w_p g_p with (H - zeta_p) g_p = R
   for the n_probes Rademacher probes R of tbk_chebyshev_moments, each system solved by CGLS to a
   relative residual below tol in every probe column (at most max_iter iterations per pole; the
   poles from the farthest from mu to the nearest, each solve started from the previous one), and
     P (device, nnzb * n_orb^2, or NULL) = M o (X R^T)/s,  Q (same, or NULL) = M o (H X R^T)/s,
   forces (device, n_atoms x 3, or NULL) from the symmetric part of M o P~ as in
   tbk_direct_density.  info (host, 2 doubles, or NULL): {CGLS iterations over all poles, the
   largest final relative residual}.  n_probes a multiple of 4; n_pairs in [1, 256]; flags must
   be TBK_FP64 (the systems' condition numbers reach max|eps - mu|/(pi kT)).  TBK_ERR_NOCONV
   when a solve stops above tol (the outputs are still written).  Synchronises the stream. */
int tbk_rational_density(tbk_ctx* ctx, const tbk_bsr* H, const tbk_model* model, const double* pos,
                         const double* box, uint64_t probe_seed, int32_t n_probes, double mu, double kT,
                         int32_t n_pairs, double tol, int32_t max_iter, int32_t flags, double* P,
                         double* Q, double* forces, double* info);

/* ---- allocation-free variant of tbk_chebyshev_moments ------------------------------------

   No counterpart in the paper: this entry point exists for callers that cannot allocate device
   memory while they run (latency-bounded loops where an allocation may block on the device,
   embedders whose device memory is budgeted by a framework that owns every allocation, drivers
   that forbid allocation between set-up and shutdown).  It computes exactly what
   tbk_chebyshev_moments computes, with the same kernels, but takes all of its scratch from one
   static device array of 64 MiB (TBK_NOALLOC_SCRATCH_BYTES) that is part of the library and
   stays reserved on every GPU that loads the library until the process exits.  The call
   allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
   - Arguments, layout, ownership and errors are those of tbk_chebyshev_moments; in addition a
     problem whose scratch (mapped H, two panels, per-step partial sums) exceeds the static size
     fails with TBK_ERR_ARG and a message giving the bytes it would need.
   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
     that device current; make that first call before any stream capture.  Under CUDA's lazy
     module loading (the default) that first call is also the one that loads the library's
     module and so commits the 64 MiB on the device: it can fail for lack of device memory, and
     only the calls after it allocate nothing.  The address is kept per device for the life of
     the process, so the device's primary context must stay alive between calls (no
     cudaDeviceReset), and calls must run under that primary context.
   - The context's kernel timer (tbk_kernel_timer) is switched off for the duration of the call:
     timing would create CUDA events.
   - Every call on a device shares the one array and leaves its contents behind (the call clears
     what must start at zero).  Calls whose work overlaps on the GPU -- on different streams, or
     from different host threads -- race on the array and give wrong results. */
#define TBK_NOALLOC_SCRATCH_BYTES (64u << 20)
int tbk_chebyshev_moments_noalloc(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax,
                                  uint64_t probe_seed, int32_t n_probes, int32_t order,
                                  int32_t flags, double* moments);

#ifdef __cplusplus
}
#endif

#endif /* TBK_H */
