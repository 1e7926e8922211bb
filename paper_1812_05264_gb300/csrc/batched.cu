// a11: many clusters of uneven size and temperature in one launch per recurrence step.
//
// The clusters' mapped operators (each with its own spectral interval) are merged block-
// diagonally into one operator, with clusters sorted by their number of steps so that the
// clusters still running at step j are a prefix of the rows: step j processes that prefix only.
// Every cluster keeps its own probe stream (seed and cluster-local row index), so its moments are
// those of a standalone run.  Partial sums are written per (atom, warp) and reduced per cluster in
// a fixed order.  After the first call the whole step sequence is replayed from a CUDA graph
// while the inputs (pointers, sizes, bounds, seeds, orders) stay the same.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "cheb.cuh"

namespace tbk {

void fermi_enqueue(tbk_ctx* ctx, const double* moments, int order, double emin, double emax,
                   double n_electrons, double mu_fixed, double kT, int damping, double* tab,
                   double* rho, double* res);
int quad_nodes(int p);

// Copy cluster c into the merged operator: rows shifted by a_off, blocks by b_off, mapped block
// values (column-major FP32, as the step kernels read them).
__global__ void merge_cluster(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ H, double shift, double inv, int a_off,
                              int b_off, int cl, int last, int32_t* __restrict__ m_row_ptr,
                              int32_t* __restrict__ m_col, float* __restrict__ m_hv,
                              int32_t* __restrict__ atom_cl, int* __restrict__ err) {
  // blockDim (8, 16): the 8 lanes of a row are 8 consecutive lanes of one warp
  const int a = blockIdx.x * blockDim.y + threadIdx.y;
  if (a >= n) return;
  bool has_diag = false;
  if (threadIdx.x == 0) {
    m_row_ptr[a_off + a] = b_off + row_ptr[a];
    atom_cl[a_off + a] = cl;
    if (last && a == n - 1) m_row_ptr[a_off + n] = b_off + row_ptr[n];
  }
  for (int k = row_ptr[a] + threadIdx.x; k < row_ptr[a + 1]; k += blockDim.x) {
    const int b = col[k];
    m_col[b_off + k] = a_off + b;
    const bool diag = b == a;
    has_diag |= diag;
    float* out = m_hv + (int64_t)(b_off + k) * Layout<float, 9>::BS;
    for (int l = 0; l < 9; ++l)          // column l
      for (int i = 0; i < 12; ++i) {     // row i (padded to 12)
        double v = 0.0;
        if (i < 9) {
          v = H[(int64_t)k * 81 + i * 9 + l];
          if (diag && i == l) v -= shift;
          v *= inv;
        }
        out[l * 12 + i] = (float)v;
      }
  }
  if (!__any_sync(0xFFu << (8 * (threadIdx.y & 3)), has_diag) && threadIdx.x == 0) atomicOr(err, ERR_NO_DIAGONAL);
}

// y0 = r for every merged row (cluster probe streams).
__global__ void batch_probe_panel(int64_t n_rows, int s, const int32_t* __restrict__ atom_cl,
                                  const uint64_t* __restrict__ seeds, const int32_t* __restrict__ atom0,
                                  float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows * s) return;
  const int64_t row = i / s;
  const int p = (int)(i - row * s);
  const int a = (int)(row / 9);
  const int cl = atom_cl[a];
  y[i] = tbk_probe_sign(seeds[cl], row - (int64_t)9 * atom0[cl], p);
}

// sums[(ci K + j) 2 + c] = sum over the atoms of sorted cluster ci of step j's partials.
__global__ void batch_reduce(const double* __restrict__ partials, int64_t stride, int cw,
                             const int32_t* __restrict__ a_off, const int32_t* __restrict__ n_at,
                             const int32_t* __restrict__ ksteps, int K, double* __restrict__ sums) {
  const int j = blockIdx.x, ci = blockIdx.y;
  if (j >= ksteps[ci]) return;
  __shared__ double sh[2][256];
  const double* p = partials + (int64_t)j * stride;
  const int64_t e0 = (int64_t)a_off[ci] * cw, e1 = e0 + (int64_t)n_at[ci] * cw;
  double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    double y = p[2 * e] - c0, t = s0 + y;
    c0 = (t - s0) - y;
    s0 = t;
    y = p[2 * e + 1] - c1;
    t = s1 + y;
    c1 = (t - s1) - y;
    s1 = t;
  }
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[((int64_t)ci * K + j) * 2] = sh[0][0];
    sums[((int64_t)ci * K + j) * 2 + 1] = sh[1][0];
  }
}

// Moments of sorted cluster ci (same identities as the single-cluster path), written at its
// offset in the caller's (unsorted) output; flag bit 1 on a panel norm above ||r||.
__global__ void batch_finish(const double* __restrict__ sums, int K, const int32_t* __restrict__ ksteps,
                             const int32_t* __restrict__ orders, const int64_t* __restrict__ out_off,
                             const int32_t* __restrict__ n_at, int s, int direct,
                             double* __restrict__ mom, int* __restrict__ flag) {
  const int ci = blockIdx.x;
  const int Kc = ksteps[ci], order = orders[ci];
  const double* S = sums + (int64_t)ci * K * 2;
  double* out = mom + out_off[ci];
  const double mu0 = 9.0 * n_at[ci], inv_s = 1.0 / s;
  const double mu1 = Kc >= 1 ? S[0] * inv_s : 0.0;
  for (int k = threadIdx.x; k < order; k += blockDim.x) {
    double v;
    if (k == 0) v = mu0;
    else if (direct) v = S[2 * (k - 1)] * inv_s;
    else if (k == 1) v = mu1;
    else if ((k & 1) == 0) v = 2.0 * S[2 * (k / 2 - 1) + 1] * inv_s - mu0;
    else v = 2.0 * S[2 * ((k + 1) / 2 - 1)] * inv_s - mu1;
    out[k] = v;
  }
  for (int j = threadIdx.x; j < Kc; j += blockDim.x) {
    const double e = S[2 * j + 1] * inv_s, o = S[2 * j];
    if (!(e <= mu0 * (1.0 + 1e-3)) || !isfinite(o)) atomicOr(flag, 1);
  }
}

struct BatchGraph {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  int64_t kernels = 0;  // kernel launches recorded in the graph
};

static BatchGraph& batch_graph(tbk_ctx* ctx) {
  // one cached graph per context (the context's address identifies it)
  static std::vector<std::pair<tbk_ctx*, BatchGraph*>> cache;
  for (auto& e : cache)
    if (e.first == ctx) return *e.second;
  cache.emplace_back(ctx, new BatchGraph());
  return *cache.back().second;
}

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_batched_moments(tbk_ctx* ctx, int32_t n_clusters, const tbk_bsr* H,
                                   const double* emin, const double* emax, const uint64_t* seeds,
                                   int32_t n_probes, const int32_t* orders, int32_t flags,
                                   double* moments) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && H && emin && emax && seeds && orders && moments, "NULL argument");
  TBK_CHECK_ARG(n_clusters >= 1, "n_clusters must be >= 1");
  TBK_CHECK_ARG((flags & ~(TBK_MOMENTS_DIRECT | TBK_NO_GRAPH)) == 0,
                "batched moments run in mixed precision; unknown or unsupported flag");
  TBK_CHECK_ARG(n_probes >= 128 && n_probes % 128 == 0, "batched moments need n_probes a multiple of 128");
  DeviceGuard dg(ctx);
  const int direct = (flags & TBK_MOMENTS_DIRECT) ? 1 : 0;
  const int s = n_probes;
  // ---- host plan: sort clusters by step count (descending) ----
  std::vector<int> K(n_clusters), idx(n_clusters);
  int64_t tot_atoms = 0, tot_blocks = 0, tot_mom = 0;
  std::vector<int64_t> out_off_u(n_clusters);
  for (int c = 0; c < n_clusters; ++c) {
    const tbk_bsr& h = H[c];
    TBK_CHECK_ARG(h.n_orb == 9, "batched moments need 9x9 blocks");
    TBK_CHECK_ARG(h.n_atoms >= 1 && h.nnzb >= h.n_atoms && h.row_ptr && h.col && h.val, "empty or NULL cluster");
    TBK_CHECK_ARG(orders[c] >= 1, "order must be >= 1");
    TBK_CHECK_ARG(std::isfinite(emin[c]) && std::isfinite(emax[c]) && emax[c] > emin[c], "need emax > emin");
    K[c] = direct ? orders[c] - 1 : orders[c] / 2;
    idx[c] = c;
    out_off_u[c] = tot_mom;
    tot_mom += orders[c];
    tot_atoms += h.n_atoms;
    tot_blocks += h.nnzb;
  }
  TBK_CHECK_ARG(tot_blocks < INT32_MAX && tot_atoms * 9 < INT32_MAX, "batch too large for int32 indices");
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return K[x] > K[y]; });
  const int Kmax = K[idx[0]];
  std::vector<int32_t> a_off(n_clusters), n_at(n_clusters), ks(n_clusters), ord(n_clusters);
  std::vector<int64_t> b_off(n_clusters), out_off(n_clusters);
  std::vector<uint64_t> sd(n_clusters);
  int64_t ao = 0, bo = 0;
  for (int ci = 0; ci < n_clusters; ++ci) {
    const int c = idx[ci];
    a_off[ci] = (int32_t)ao;
    b_off[ci] = bo;
    n_at[ci] = H[c].n_atoms;
    ks[ci] = K[c];
    ord[ci] = orders[c];
    out_off[ci] = out_off_u[c];
    sd[ci] = seeds[c];
    ao += H[c].n_atoms;
    bo += H[c].nnzb;
  }
  // ---- device buffers ----
  HOp op;
  op.B = 9;
  op.prec = TBK_MIXED;
  op.n_atoms = (int)tot_atoms;
  op.nnzb = tot_blocks;
  op.n_rows = tot_atoms * 9;
  const int cw = bulk_consumer_warps(op, s);
  TBK_CHECK_ARG(cw > 0, "no TMA-fed step kernel for this probe count");
  const size_t panel = (size_t)op.n_rows * s * 4;
  const int64_t pstride = tot_atoms * cw * 2;   // doubles per step of partials
  char* meta = (char*)scratch(ctx, WS_TABLE, 64 * (size_t)n_clusters + 4096);
  int32_t* d_aoff = (int32_t*)meta;
  int32_t* d_nat = d_aoff + n_clusters;
  int32_t* d_ks = d_nat + n_clusters;
  int32_t* d_ord = d_ks + n_clusters;
  int32_t* d_atom0 = d_ord + n_clusters;      // first merged atom of sorted cluster ci
  uint64_t* d_seed = (uint64_t*)(((uintptr_t)(d_atom0 + n_clusters) + 15) & ~(uintptr_t)15);
  int64_t* d_out = (int64_t*)(d_seed + n_clusters);
  int32_t* m_row_ptr = (int32_t*)scratch(ctx, WS_CELLS, sizeof(int32_t) * (size_t)(2 * tot_atoms + 1) + 64);
  int32_t* atom_cl = m_row_ptr + tot_atoms + 1;
  int32_t* m_col = (int32_t*)scratch(ctx, WS_CELLS2, sizeof(int32_t) * (size_t)tot_blocks + 64);
  float* m_hv = (float*)scratch(ctx, WS_HHAT, sizeof(float) * (size_t)tot_blocks * Layout<float, 9>::BS);
  char* panels = (char*)scratch(ctx, WS_PANEL0, 2 * panel);
  double* partials = (double*)scratch(ctx, WS_PARTIALS, sizeof(double) * (size_t)std::max(1, Kmax) * pstride);
  double* sums = (double*)scratch(ctx, WS_MISC, sizeof(double) * 2 * (size_t)std::max(1, Kmax) * n_clusters + 64);
  int* flag = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemcpyAsync(d_aoff, a_off.data(), 4 * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_nat, n_at.data(), 4 * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_ks, ks.data(), 4 * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_ord, ord.data(), 4 * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_atom0, a_off.data(), 4 * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_seed, sd.data(), 8 * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_out, out_off.data(), 8 * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  op.row_ptr = m_row_ptr;
  op.col = m_col;
  op.hv = m_hv;
  BatchRows br;
  br.atom_cl = atom_cl;
  br.seed = d_seed;
  br.atom0 = d_atom0;
  // active atoms before step j: prefix over clusters with K >= j
  auto active = [&](int j) {
    int64_t r = 0;
    for (int ci = 0; ci < n_clusters && ks[ci] >= j; ++ci) r += n_at[ci];
    return (int)r;
  };

  auto enqueue = [&]() {
    for (int ci = 0; ci < n_clusters; ++ci) {
      const int c = idx[ci];
      const double shift = 0.5 * (emax[c] + emin[c]), inv = 2.0 / (emax[c] - emin[c]);
      merge_cluster<<<ceil_div(n_at[ci], 16), dim3(8, 16), 0, ctx->stream>>>(
          n_at[ci], H[c].row_ptr, H[c].col, H[c].val, shift, inv, a_off[ci], (int)b_off[ci], ci,
          ci == n_clusters - 1, m_row_ptr, m_col, m_hv, atom_cl, flag);
      post_launch(ctx, "merge_cluster");
    }
    char* A = panels;
    char* Bq = panels + panel;
    batch_probe_panel<<<(unsigned)((op.n_rows * s + 255) / 256), 256, 0, ctx->stream>>>(
        op.n_rows, s, atom_cl, d_seed, d_atom0, (float*)A);
    post_launch(ctx, "batch_probe_panel");
    void *cur = A, *prev = nullptr;
    for (int j = 1; j <= Kmax; ++j) {
      HOp opj = op;
      opj.n_atoms = active(j);
      StepArgs a;
      a.seed = 0;
      a.s = s;
      a.direct = direct;
      a.partials = partials + (size_t)(j - 1) * pstride;
      a.err = flag;
      a.batch = br;
      a.per_task = 1;
      if (j == 1) {
        a.yin = A;       // y_0 = r
        a.alpha = 1.0;
        a.yout = Bq;
        prev = A;
        cur = Bq;
      } else {
        a.yin = cur;
        a.yprev = prev;
        a.yout = prev;
        a.alpha = 2.0;
        std::swap(cur, prev);
      }
      launch_step(ctx, opj, a);
    }
    if (Kmax >= 1) {
      batch_reduce<<<dim3(Kmax, n_clusters), 256, 0, ctx->stream>>>(partials, pstride, cw, d_aoff,
                                                                      d_nat, d_ks, Kmax, sums);
      post_launch(ctx, "batch_reduce");
    }
    batch_finish<<<n_clusters, 256, 0, ctx->stream>>>(sums, std::max(1, Kmax), d_ks, d_ord, d_out,
                                                      d_nat, s, direct, moments, flag);
    post_launch(ctx, "batch_finish");
  };

  const bool graph = !(flags & TBK_NO_GRAPH);
  if (!graph) {
    enqueue();
  } else {
    BatchGraph& bg = batch_graph(ctx);
    std::vector<uint64_t> key = {(uint64_t)n_clusters, (uint64_t)s, (uint64_t)direct, (uint64_t)(uintptr_t)moments,
                                 (uint64_t)(uintptr_t)panels, (uint64_t)(uintptr_t)partials,
                                 (uint64_t)(uintptr_t)m_hv, (uint64_t)(uintptr_t)meta};
    for (int c = 0; c < n_clusters; ++c) {
      uint64_t e0, e1;
      memcpy(&e0, &emin[c], 8);
      memcpy(&e1, &emax[c], 8);
      for (uint64_t v : {(uint64_t)(uintptr_t)H[c].row_ptr, (uint64_t)(uintptr_t)H[c].col,
                         (uint64_t)(uintptr_t)H[c].val, (uint64_t)H[c].n_atoms, (uint64_t)H[c].nnzb,
                         e0, e1, seeds[c], (uint64_t)orders[c]})
        key.push_back(v);
    }
    if (!bg.exec || bg.key != key) {
      if (bg.exec) {
        cudaGraphExecDestroy(bg.exec);
        bg.exec = nullptr;
      }
      if (!bg.cap) TBK_CUDA(cudaStreamCreateWithFlags(&bg.cap, cudaStreamNonBlocking));
      // capture on a private stream (the context's stream may be the legacy default stream)
      sync(ctx);
      cudaStream_t user = ctx->stream;
      ctx->stream = bg.cap;
      cudaGraph_t g = nullptr;
      const int64_t l0 = ctx->launches;
      cudaError_t e = cudaStreamBeginCapture(bg.cap, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        try {
          enqueue();
        } catch (...) {
          cudaStreamEndCapture(bg.cap, &g);
          if (g) cudaGraphDestroy(g);
          ctx->stream = user;
          throw;
        }
        e = cudaStreamEndCapture(bg.cap, &g);
      }
      ctx->stream = user;
      bg.kernels = ctx->launches - l0;
      ctx->launches = l0;  // counted when the graph runs
      TBK_CUDA(e);
      e = cudaGraphInstantiate(&bg.exec, g, 0);
      cudaGraphDestroy(g);
      TBK_CUDA(e);
      bg.key = key;
    }
    TBK_CUDA(cudaGraphLaunch(bg.exec, ctx->stream));
    ctx->launches += bg.kernels;
  }
  int hflag = 0;
  TBK_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(hflag);
  if (hflag & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in the recurrence kernel expired");
  if (hflag) throw Error(TBK_ERR_SPECTRUM, "a Chebyshev panel of some cluster grew beyond ||r||");
  TBK_API_END
}

extern "C" int tbk_batched_fermi_level(tbk_ctx* ctx, int32_t n_clusters, const double* moments,
                                       const int32_t* orders, const double* emin, const double* emax,
                                       const double* n_electrons, const double* kT, int32_t damping,
                                       double* out) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && moments && orders && emin && emax && n_electrons && kT && out, "NULL argument");
  TBK_CHECK_ARG(n_clusters >= 1, "n_clusters must be >= 1");
  TBK_CHECK_ARG(damping == TBK_DAMP_NONE || damping == TBK_DAMP_JACKSON, "unknown damping");
  DeviceGuard dg(ctx);
  std::vector<FermiJob> jobs(n_clusters);
  size_t need = 0;
  int64_t moff = 0;
  int M_max = 1;
  for (int c = 0; c < n_clusters; ++c) {
    TBK_CHECK_ARG(orders[c] >= 1 && orders[c] <= (1 << 22), "order out of range");
    TBK_CHECK_ARG(kT[c] > 0.0 && std::isfinite(kT[c]) && emax[c] > emin[c], "bad kT or bounds");
    FermiJob& j = jobs[c];
    j.M = quad_nodes(orders[c]);
    j.p = orders[c];
    j.emin = emin[c];
    j.emax = emax[c];
    j.n_e = n_electrons[c];
    j.kT = kT[c];
    j.mom_off = moff;
    j.tab_off = (int64_t)need;
    j.rho_off = j.tab_off + 4 * (int64_t)j.M;
    need += 5 * (size_t)j.M + 8;
    moff += orders[c];
    M_max = std::max(M_max, j.M);
  }
  double* buf = (double*)scratch(ctx, WS_COEF, sizeof(double) * need);
  double* res = (double*)scratch(ctx, WS_NODES, sizeof(double) * 8 * (size_t)n_clusters + sizeof(FermiJob) * n_clusters + 64);
  FermiJob* d_jobs = (FermiJob*)(res + 8 * (size_t)n_clusters);
  TBK_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(FermiJob) * n_clusters, cudaMemcpyHostToDevice, ctx->stream));
  fermi_enqueue_batched(ctx, n_clusters, d_jobs, M_max, moments, damping, buf, res);
  std::vector<double> h(8 * (size_t)n_clusters);
  TBK_CUDA(cudaMemcpyAsync(h.data(), res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  bool bad = false;
  for (int c = 0; c < n_clusters; ++c) {
    for (int i = 0; i < 4; ++i) out[4 * c + i] = h[8 * c + i];
    bad = bad || h[8 * c + 4] != 0.0;
  }
  if (bad) throw Error(TBK_ERR_NOCONV, "n_electrons is outside the estimated N(mu) range for some cluster");
  TBK_API_END
}

// ---- batched adjoint and forces -------------------------------------------------------------

#include "model.cuh"

namespace tbk {

void coefficients(tbk_ctx* ctx, int fn, int p, double emin, double emax, double mu, double kT,
                  int damping, double* out);
bool fused_eligible(const HOp& op, int s, int plain);
void launch_fused(tbk_ctx* ctx, const HOp& op, const void* bin, const void* bprev, void* bout,
                  const void* ypan, float4 cf, uint64_t seed, int s, double w, double* Gacc,
                  int* err, const BatchRows& batch, const float4* cf_cl, const void* ym1,
                  const void* yp1);
void launch_transpose_map(tbk_ctx* ctx, int n_atoms, const int32_t* row_ptr, const int32_t* col,
                          int32_t* tr, int* err);
void launch_symmetrize_batched(tbk_ctx* ctx, int n_atoms, const int32_t* row_ptr, const int32_t* tr,
                               const int32_t* atom_cl, const double* scale_cl, const double* Gacc,
                               double* G);
void launch_forces(tbk_ctx* ctx, const DevModel& M, const double* pos, int n_atoms, const int32_t* row_ptr,
                   const int32_t* col, const int32_t* tr, const double* G, double* tq, double* F);

void launch_batch_probe_panel(tbk_ctx* ctx, const HOp& op, const BatchRows& br, int s, void* out) {
  batch_probe_panel<<<(unsigned)((op.n_rows * s + 255) / 256), 256, 0, ctx->stream>>>(
      op.n_rows, s, br.atom_cl, br.seed, br.atom0, (float*)out);
  post_launch(ctx, "batch_probe_panel");
}

}  // namespace tbk

namespace tbk {

// The adjoint of the doubled moments over a merged batch of clusters.  mu != NULL: chemical
// potentials given (tbk_batched_density_and_forces).  mu == NULL: the forward sweep also yields
// the moments, then mu, Omega, E, N of every cluster are solved for before the backward sweep
// (tbk_batched_energies_and_forces; moments / observables receive them).
static void batched_adjoint(tbk_ctx* ctx, int ncl, const tbk_bsr* H, const tbk_model* model,
                            const double* const* pos, const double* emin, const double* emax,
                            const uint64_t* seeds, int s, const int32_t* orders, const double* mu,
                            const double* n_electrons, const double* kT, int damping,
                            int64_t max_panel_bytes, double* moments, double* observables,
                            double* const* G, double* const* forces, bool windowed) {
  HOp op;
  op.B = 9;
  op.prec = TBK_MIXED;
  DevModel Mdl{};
  if (forces) {
    Mdl = upload_model(ctx, model, nullptr, WS_TABLE);
    TBK_CHECK_ARG(Mdl.kind == TBK_MODEL_SK, "forces need the Slater-Koster model");
  }
  // ---- plan: sort by K = order/2 (descending); cluster c needs y_1 .. y_{K_c} ----
  std::vector<int> idx(ncl);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return orders[x] / 2 > orders[y] / 2; });
  std::vector<int32_t> a_off(ncl), n_at(ncl), pc(ncl), ks(ncl);
  std::vector<int64_t> b_off(ncl), out_off(ncl), out_off_u(ncl);
  std::vector<uint64_t> sd(ncl);
  std::vector<double> scale(ncl);
  int64_t ao = 0, bo = 0, mo = 0;
  int pmax = 1;
  for (int c = 0; c < ncl; ++c) {
    out_off_u[c] = mo;
    mo += orders[c];
  }
  for (int ci = 0; ci < ncl; ++ci) {
    const int c = idx[ci];
    TBK_CHECK_ARG(H[c].n_atoms >= 1 && H[c].row_ptr && H[c].col && H[c].val, "empty or NULL cluster");
    TBK_CHECK_ARG(orders[c] >= 1 && emax[c] > emin[c] && kT[c] > 0.0, "bad order, bounds or kT");
    a_off[ci] = (int32_t)ao;
    b_off[ci] = bo;
    n_at[ci] = H[c].n_atoms;
    pc[ci] = orders[c];
    ks[ci] = orders[c] / 2;
    out_off[ci] = out_off_u[c];
    sd[ci] = seeds[c];
    scale[ci] = 2.0 / (emax[c] - emin[c]);
    ao += H[c].n_atoms;
    bo += H[c].nnzb;
    pmax = std::max(pmax, orders[c]);
  }
  TBK_CHECK_ARG(bo < INT32_MAX && ao * 9 < INT32_MAX, "batch too large for int32 indices");
  const int Kmax = ks[0];
  op.n_atoms = (int)ao;
  op.nnzb = bo;
  op.n_rows = ao * 9;
  // ---- device metadata, merged operator and positions ----
  char* meta = (char*)scratch(ctx, WS_TABLE, 128 * (size_t)ncl + 4096);
  // (WS_TABLE also holds the uploaded model table only for TABLE models; SK needs none)
  int32_t* d_atom0 = (int32_t*)meta;
  int32_t* d_nat = d_atom0 + ncl;
  int32_t* d_ks = d_nat + ncl;
  int32_t* d_ord = d_ks + ncl;
  uint64_t* d_seed = (uint64_t*)(((uintptr_t)(d_ord + ncl) + 15) & ~(uintptr_t)15);
  double* d_scale = (double*)(d_seed + ncl);
  int64_t* d_out = (int64_t*)(d_scale + ncl);
  TBK_CUDA(cudaMemcpyAsync(d_atom0, a_off.data(), 4 * ncl, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_nat, n_at.data(), 4 * ncl, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_ks, ks.data(), 4 * ncl, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_ord, pc.data(), 4 * ncl, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_seed, sd.data(), 8 * ncl, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_scale, scale.data(), 8 * ncl, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_out, out_off.data(), 8 * ncl, cudaMemcpyHostToDevice, ctx->stream));
  int32_t* m_row_ptr = (int32_t*)scratch(ctx, WS_CELLS, sizeof(int32_t) * (size_t)(2 * ao + 1) + 64);
  int32_t* atom_cl = m_row_ptr + ao + 1;
  int32_t* m_col = (int32_t*)scratch(ctx, WS_CELLS2, sizeof(int32_t) * (size_t)bo + 64);
  float* m_hv = (float*)scratch(ctx, WS_HHAT, sizeof(float) * (size_t)bo * Layout<float, 9>::BS);
  double* m_pos = (double*)scratch(ctx, WS_CELLS3, sizeof(double) * 3 * (size_t)ao + 64);
  // err: bit 4 = a row has no diagonal block, bit 2 = a bounded wait expired, bit 1 = a pattern is
  // not symmetric; err[1] bit 1 = a panel outgrew ||r|| (the spectrum is not inside [emin, emax])
  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), ctx->stream));
  for (int ci = 0; ci < ncl; ++ci) {
    const int c = idx[ci];
    const double shift = 0.5 * (emax[c] + emin[c]), inv = 2.0 / (emax[c] - emin[c]);
    merge_cluster<<<ceil_div(n_at[ci], 16), dim3(8, 16), 0, ctx->stream>>>(
        n_at[ci], H[c].row_ptr, H[c].col, H[c].val, shift, inv, a_off[ci], (int)b_off[ci], ci,
        ci == ncl - 1, m_row_ptr, m_col, m_hv, atom_cl, err);
    post_launch(ctx, "merge_cluster");
    if (forces)
      TBK_CUDA(cudaMemcpyAsync(m_pos + 3 * (size_t)a_off[ci], pos[c], sizeof(double) * 3 * n_at[ci],
                               cudaMemcpyDeviceToDevice, ctx->stream));
  }
  op.row_ptr = m_row_ptr;
  op.col = m_col;
  op.hv = m_hv;
  BatchRows br;
  br.atom_cl = atom_cl;
  br.seed = d_seed;
  br.atom0 = d_atom0;
  // (not WS_NODES: coefficients() keeps its cosine table there)
  float4* d_cft = (float4*)scratch(ctx, WS_LANCZOS, sizeof(float4) * (size_t)(Kmax + 1) * ncl + 64);
  // ---- the source coefficients of every step from c_k = d_k beta_k[g](mu) of every cluster ----
  auto build_cft = [&](const double* mus) {
    double* coefd = (double*)scratch(ctx, WS_COEF, sizeof(double) * (size_t)pmax * ncl);
    for (int ci = 0; ci < ncl; ++ci) {
      const int c = idx[ci];
      coefficients(ctx, TBK_FN_FREE, pc[ci], emin[c], emax[c], mus[c], kT[c], damping,
                   coefd + (size_t)ci * pmax);
    }
    std::vector<double> ch((size_t)pmax * ncl);
    TBK_CUDA(cudaMemcpyAsync(ch.data(), coefd, sizeof(double) * ch.size(), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    // per step k and cluster: (probe, y_k, y_{k-1}, y_{k+1}) coefficients of g_k (zero once k > K_c)
    std::vector<float4> cft((size_t)(Kmax + 1) * ncl, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int ci = 0; ci < ncl; ++ci) {
      const int p = pc[ci], K = p / 2;
      const double* c = ch.data() + (size_t)ci * pmax;
      std::vector<double> w(K + 2, 0.0), v(K + 2, 0.0);
      for (int k = 1; k <= K; ++k) {
        if (2 * k < p) w[k] = 2.0 * c[2 * k];
        if (k >= 2 && 2 * k - 1 < p) v[k] = 2.0 * c[2 * k - 1];
      }
      v[1] = p > 1 ? c[1] : 0.0;
      for (int k = 2; 2 * k - 1 < p; ++k) v[1] -= c[2 * k - 1];
      for (int k = 1; k <= K; ++k)
        cft[(size_t)k * ncl + ci] = make_float4(k == 1 ? (float)(v[1] / s) : 0.f, (float)(2.0 * w[k] / s),
                                                k == 1 ? 0.f : (float)(v[k] / s), (float)(v[k + 1] / s));
    }
    TBK_CUDA(cudaMemcpyAsync(d_cft, cft.data(), sizeof(float4) * cft.size(), cudaMemcpyHostToDevice, ctx->stream));
    sync(ctx);  // cft is a host vector
  };
  AdjBatch bt;
  bt.br = br;
  bt.cft = d_cft;
  bt.d_K = d_ks;
  for (int ci = 0; ci < ncl; ++ci) {
    bt.K.push_back(ks[ci]);
    bt.n_at.push_back(n_at[ci]);
  }
  double* Gacc = (double*)scratch(ctx, WS_GACC, sizeof(double) * (size_t)bo * 81 * 2);
  double* Gsym = Gacc + (size_t)bo * 81;
  TBK_CUDA(cudaMemsetAsync(Gacc, 0, sizeof(double) * (size_t)bo * 81, ctx->stream));
  if (mu) {
    build_cft(mu);
    adjoint_doubling(ctx, op, 0, s, 0, nullptr, nullptr, 0, max_panel_bytes, Gacc, err, windowed, &bt);
  } else {
    // moments from the forward sweep: per (atom, warp) partials, reduced per cluster
    const int cw = bulk_consumer_warps(op, s);
    TBK_CHECK_ARG(cw > 0, "no TMA-fed step kernel for this probe count");
    bt.pstride = ao * cw * 2;
    double* partials = (double*)scratch(ctx, WS_PARTIALS, sizeof(double) * (size_t)std::max(1, Kmax) * bt.pstride);
    double* sums = (double*)scratch(ctx, WS_SEGMENT, sizeof(double) * (2 * (size_t)std::max(1, Kmax) * ncl +
                                                                         (size_t)mo + 64));
    double* mom = moments ? moments : sums + 2 * (size_t)std::max(1, Kmax) * ncl;
    auto after_forward = [&]() {
      if (Kmax >= 1) {
        batch_reduce<<<dim3(Kmax, ncl), 256, 0, ctx->stream>>>(partials, bt.pstride, cw, d_atom0, d_nat, d_ks,
                                                                Kmax, sums);
        post_launch(ctx, "batch_reduce");
      }
      batch_finish<<<ncl, 256, 0, ctx->stream>>>(sums, std::max(1, Kmax), d_ks, d_ord, d_out, d_nat, s, 0, mom,
                                                 err + 1);
      post_launch(ctx, "batch_finish");
      // mu, Omega, E, N of every cluster
      std::vector<FermiJob> jobs(ncl);
      size_t need = 0;
      int M_max = 1;
      for (int c = 0; c < ncl; ++c) {
        FermiJob& j = jobs[c];
        j.M = quad_nodes(orders[c]);
        j.p = orders[c];
        j.emin = emin[c];
        j.emax = emax[c];
        j.n_e = n_electrons[c];
        j.kT = kT[c];
        j.mom_off = out_off_u[c];
        j.tab_off = (int64_t)need;
        j.rho_off = j.tab_off + 4 * (int64_t)j.M;
        need += 5 * (size_t)j.M + 8;
        M_max = std::max(M_max, j.M);
      }
      double* fbuf = (double*)scratch(ctx, WS_PANEL1, sizeof(double) * need);
      double* res = (double*)scratch(ctx, WS_PANEL2, sizeof(double) * 8 * (size_t)ncl + sizeof(FermiJob) * ncl + 64);
      FermiJob* d_jobs = (FermiJob*)(res + 8 * (size_t)ncl);
      TBK_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(FermiJob) * ncl, cudaMemcpyHostToDevice, ctx->stream));
      fermi_enqueue_batched(ctx, ncl, d_jobs, M_max, mom, damping, fbuf, res);
      std::vector<double> h(8 * (size_t)ncl);
      int herr[2] = {0, 0};
      TBK_CUDA(cudaMemcpyAsync(h.data(), res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
      TBK_CUDA(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, ctx->stream));
      sync(ctx);
      check_diagonal_flag(herr[0]);
      if ((herr[0] | herr[1]) & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in a recurrence kernel expired");
      TBK_CHECK_ARG(herr[0] == 0, "a block pattern is not symmetric");
      if (herr[1])
        throw Error(TBK_ERR_SPECTRUM, "a Chebyshev panel grew beyond ||r||: some cluster's spectrum is not "
                                      "inside its [emin, emax]");
      std::vector<double> mus(ncl);
      bool bad = false;
      for (int c = 0; c < ncl; ++c) {
        for (int q = 0; q < 4; ++q) observables[4 * c + q] = h[8 * c + q];
        mus[c] = h[8 * c];
        bad = bad || h[8 * c + 4] != 0.0;
      }
      if (bad) throw Error(TBK_ERR_NOCONV, "n_electrons is outside the estimated N(mu) range for some cluster");
      build_cft(mus.data());
      return std::vector<double>();
    };
    adjoint_doubling(ctx, op, 0, s, 0, after_forward, partials, 0, max_panel_bytes, Gacc, err, windowed, &bt);
  }
  // ---- G (symmetrised, per-cluster scale) and forces on the merged pattern ----
  int32_t* tr = (int32_t*)scratch(ctx, WS_TRANSPOSE, sizeof(int32_t) * (size_t)bo);
  launch_transpose_map(ctx, op.n_atoms, op.row_ptr, op.col, tr, err);
  launch_symmetrize_batched(ctx, op.n_atoms, op.row_ptr, tr, atom_cl, d_scale, Gacc, Gsym);
  double* Fm = nullptr;
  if (forces) {
    double* tq = (double*)scratch(ctx, WS_MISC, sizeof(double) * 3 * (size_t)bo + sizeof(double) * 3 * (size_t)ao);
    Fm = tq + 3 * (size_t)bo;
    launch_forces(ctx, Mdl, m_pos, op.n_atoms, op.row_ptr, op.col, tr, Gsym, tq, Fm);
  }
  for (int ci = 0; ci < ncl; ++ci) {
    const int c = idx[ci];
    if (G && G[c])
      TBK_CUDA(cudaMemcpyAsync(G[c], Gsym + (size_t)b_off[ci] * 81, sizeof(double) * 81 * (size_t)H[c].nnzb,
                               cudaMemcpyDeviceToDevice, ctx->stream));
    if (forces && forces[c])
      TBK_CUDA(cudaMemcpyAsync(forces[c], Fm + 3 * (size_t)a_off[ci], sizeof(double) * 3 * n_at[ci],
                               cudaMemcpyDeviceToDevice, ctx->stream));
  }
  int herr = 0;
  TBK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(herr);
  if (herr & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in a recurrence kernel expired");
  TBK_CHECK_ARG(herr == 0, "a block pattern is not symmetric");
}

static bool batch_merges(const tbk_bsr* H, int ncl, int s) {
  HOp op;
  op.B = 9;
  op.prec = TBK_MIXED;
  bool merged = fused_eligible(op, s, 0);
  for (int c = 0; c < ncl; ++c) merged = merged && H[c].n_orb == 9;
  return merged;
}

}  // namespace tbk

extern "C" int tbk_batched_density_and_forces(
    tbk_ctx* ctx, int32_t n_clusters, const tbk_bsr* H, const tbk_model* model,
    const double* const* pos, const double* emin, const double* emax, const uint64_t* seeds,
    int32_t n_probes, const int32_t* orders, const double* mu, const double* kT, int32_t damping,
    int32_t flags, int64_t max_panel_bytes, double* const* G, double* const* forces) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && H && emin && emax && seeds && orders && mu && kT, "NULL argument");
  TBK_CHECK_ARG(n_clusters >= 1, "n_clusters must be >= 1");
  TBK_CHECK_ARG(G || forces, "nothing to compute: G and forces are both NULL");
  TBK_CHECK_ARG((flags & ~TBK_WINDOWED) == 0, "batched adjoint runs in mixed precision; unknown flag");
  TBK_CHECK_ARG(!forces || pos, "forces need positions");
  DeviceGuard dg(ctx);
  const int s = n_probes, ncl = n_clusters;
  if (!batch_merges(H, ncl, s)) {
    // same kernels, one cluster after the other
    for (int c = 0; c < ncl; ++c) {
      const int rc = tbk_density_and_forces(ctx, &H[c], model, pos ? pos[c] : nullptr, nullptr, emin[c],
                                            emax[c], seeds[c], s, orders[c], mu[c], kT[c], damping, 0,
                                            max_panel_bytes, G ? G[c] : nullptr,
                                            forces ? forces[c] : nullptr);
      if (rc != TBK_OK) throw Error(rc, std::string("cluster ") + std::to_string(c) + ": " + tbk_last_error());
    }
    return TBK_OK;
  }
  batched_adjoint(ctx, ncl, H, model, pos, emin, emax, seeds, s, orders, mu, nullptr, kT, damping,
                  max_panel_bytes, nullptr, nullptr, G, forces, (flags & TBK_WINDOWED) != 0);
  TBK_API_END
}

extern "C" int tbk_batched_energies_and_forces(
    tbk_ctx* ctx, int32_t n_clusters, const tbk_bsr* H, const tbk_model* model,
    const double* const* pos, const double* emin, const double* emax, const uint64_t* seeds,
    int32_t n_probes, const int32_t* orders, const double* n_electrons, const double* kT,
    int32_t damping, int32_t flags, int64_t max_panel_bytes, double* moments, double* observables,
    double* const* G, double* const* forces) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && H && emin && emax && seeds && orders && n_electrons && kT && observables,
                "NULL argument");
  TBK_CHECK_ARG(n_clusters >= 1, "n_clusters must be >= 1");
  TBK_CHECK_ARG((flags & ~TBK_WINDOWED) == 0, "batched energies and forces run in mixed precision; unknown flag");
  TBK_CHECK_ARG(!forces || pos, "forces need positions");
  TBK_CHECK_ARG(n_probes >= 128 && n_probes % 128 == 0, "batches need n_probes a multiple of 128");
  for (int c = 0; c < n_clusters; ++c)
    TBK_CHECK_ARG(n_electrons[c] >= 0.0, "n_electrons must be >= 0");
  DeviceGuard dg(ctx);
  const int s = n_probes, ncl = n_clusters;
  if (!batch_merges(H, ncl, s)) {
    // the separate calls give the same results for the other shapes
    int64_t mo = 0;
    for (int c = 0; c < ncl; ++c) mo += orders[c];
    double* mom = moments ? moments : (double*)scratch(ctx, WS_SEGMENT, sizeof(double) * (size_t)mo);
    int rc = tbk_batched_moments(ctx, ncl, H, emin, emax, seeds, s, orders, 0, mom);
    if (rc != TBK_OK) throw Error(rc, tbk_last_error());
    rc = tbk_batched_fermi_level(ctx, ncl, mom, orders, emin, emax, n_electrons, kT, damping, observables);
    if (rc != TBK_OK) throw Error(rc, tbk_last_error());
    if (G || forces) {
      std::vector<double> mus(ncl);
      for (int c = 0; c < ncl; ++c) mus[c] = observables[4 * c];
      rc = tbk_batched_density_and_forces(ctx, ncl, H, model, pos, emin, emax, seeds, s, orders, mus.data(), kT,
                                          damping, 0, max_panel_bytes, G, forces);
      if (rc != TBK_OK) throw Error(rc, tbk_last_error());
    }
    return TBK_OK;
  }
  batched_adjoint(ctx, ncl, H, model, pos, emin, emax, seeds, s, orders, nullptr, n_electrons, kT, damping,
                  max_panel_bytes, moments, observables, G, forces, (flags & TBK_WINDOWED) != 0);
  TBK_API_END
}
