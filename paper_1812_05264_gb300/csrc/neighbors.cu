// a1: neighbour list by a uniform cell grid (the paper partitions the simulation volume into
// uniform cubes to build neighbour lists in linear time, Sec. II.E).  Output: CSR of all
// pairs with r^2 <= cutoff^2, self included, ascending columns.
#include <cmath>

#include "common.cuh"
#include "scan.cuh"

namespace tbk {

struct CellGrid {
  double lo[3];     // origin of the grid
  double cs[3];     // cell edge (>= cutoff)
  int nc[3];        // cells per direction
  double box[3];    // periodic lengths (0 = open)
  int periodic;
};

__global__ void bbox_partial(const double* __restrict__ pos, int n, double* __restrict__ part) {
  __shared__ double sh[6][256];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int c = 0; c < 3; ++c) {
      double v = pos[3 * i + c];
      mn[c] = fmin(mn[c], v);
      mx[c] = fmax(mx[c], v);
    }
  for (int c = 0; c < 3; ++c) {
    sh[c][threadIdx.x] = mn[c];
    sh[3 + c][threadIdx.x] = mx[c];
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int c = 0; c < 3; ++c) {
        sh[c][threadIdx.x] = fmin(sh[c][threadIdx.x], sh[c][threadIdx.x + o]);
        sh[3 + c][threadIdx.x] = fmax(sh[3 + c][threadIdx.x], sh[3 + c][threadIdx.x + o]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 6; ++c) part[6 * blockIdx.x + c] = sh[c][0];
}

__device__ __forceinline__ double wrap_coord(double x, double L) {
  return L > 0.0 ? x - L * floor(x / L) : x;
}

__device__ __forceinline__ int cell_coord(double x, const CellGrid& g, int c) {
  double u = (wrap_coord(x, g.box[c]) - g.lo[c]) / g.cs[c];
  int k = (int)floor(u);
  return k < 0 ? 0 : (k >= g.nc[c] ? g.nc[c] - 1 : k);
}

__global__ void assign_cells(const double* __restrict__ pos, int n, CellGrid g,
                             int32_t* __restrict__ atom_cell, int32_t* __restrict__ cell_count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cx = cell_coord(pos[3 * i], g, 0), cy = cell_coord(pos[3 * i + 1], g, 1),
      cz = cell_coord(pos[3 * i + 2], g, 2);
  int c = (cx * g.nc[1] + cy) * g.nc[2] + cz;
  atom_cell[i] = c;
  atomicAdd(&cell_count[c], 1);
}

__global__ void fill_cells(int n, const int32_t* __restrict__ atom_cell,
                           const int64_t* __restrict__ cell_start, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ cell_atoms) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = atom_cell[i];
  int k = atomicAdd(&cursor[c], 1);
  cell_atoms[cell_start[c] + k] = i;
}

// Squared distance with the rounding that defines the pattern: one rounding per operation,
// no contraction, ((dx*dx) + (dy*dy)) + (dz*dz), minimum image dx - L*rint(dx/L).
__device__ __forceinline__ double pair_r2(const double* __restrict__ pos, int i, int j,
                                          const CellGrid& g) {
  double r2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double d = __dsub_rn(pos[3 * j + c], pos[3 * i + c]);
    if (g.box[c] > 0.0) d = __dsub_rn(d, __dmul_rn(g.box[c], rint(__ddiv_rn(d, g.box[c]))));
    double d2 = __dmul_rn(d, d);
    r2 = c == 0 ? d2 : __dadd_rn(r2, d2);
  }
  return r2;
}

// One thread per atom: visit the 27 surrounding cells; count (col == nullptr) or write the
// row's columns in arbitrary order followed by an in-place insertion sort.
__global__ void pair_pass(const double* __restrict__ pos, int n, CellGrid g, double rc2,
                          const int32_t* __restrict__ atom_cell,
                          const int64_t* __restrict__ cell_start,
                          const int32_t* __restrict__ cell_atoms, int32_t* __restrict__ count,
                          const int64_t* __restrict__ row_start, int32_t* __restrict__ col) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = atom_cell[i];
  int cz = c % g.nc[2], cy = (c / g.nc[2]) % g.nc[1], cx = c / (g.nc[1] * g.nc[2]);
  int64_t out = col ? row_start[i] : 0;
  int cnt = 0;
  // Offsets -1..1 per direction; a periodic direction with fewer than 3 cells visits each of
  // its cells once instead (so that no cell is seen twice through the wrap).
  int lo[3], hi[3];
  for (int c3 = 0; c3 < 3; ++c3) {
    const bool few = g.box[c3] > 0.0 && g.nc[c3] < 3;
    lo[c3] = few ? 0 : -1;
    hi[c3] = few ? g.nc[c3] - 1 : 1;
  }
  for (int ox = lo[0]; ox <= hi[0]; ++ox) {
    int x = cx + ox;
    if (g.box[0] > 0.0) x = (x + g.nc[0]) % g.nc[0];
    else if (x < 0 || x >= g.nc[0]) continue;
    for (int oy = lo[1]; oy <= hi[1]; ++oy) {
      int y = cy + oy;
      if (g.box[1] > 0.0) y = (y + g.nc[1]) % g.nc[1];
      else if (y < 0 || y >= g.nc[1]) continue;
      for (int oz = lo[2]; oz <= hi[2]; ++oz) {
        int z = cz + oz;
        if (g.box[2] > 0.0) z = (z + g.nc[2]) % g.nc[2];
        else if (z < 0 || z >= g.nc[2]) continue;
        int cc = (x * g.nc[1] + y) * g.nc[2] + z;
        for (int64_t k = cell_start[cc]; k < cell_start[cc + 1]; ++k) {
          int j = cell_atoms[k];
          if (j == i || pair_r2(pos, i, j, g) <= rc2) {
            if (col) col[out + cnt] = j;
            ++cnt;
          }
        }
      }
    }
  }
  if (!col) {
    count[i] = cnt;
    return;
  }
  int32_t* r = col + out;
  for (int a = 1; a < cnt; ++a) {
    int32_t v = r[a];
    int b = a - 1;
    while (b >= 0 && r[b] > v) {
      r[b + 1] = r[b];
      --b;
    }
    r[b + 1] = v;
  }
}

__global__ void to_i32(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)in[i];
}

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_build_neighbors(tbk_ctx* ctx, const double* pos, int32_t n_atoms,
                                   const double* box, double cutoff, int32_t* row_ptr,
                                   int32_t* col, int64_t col_capacity, int64_t* nnzb) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG(n_atoms >= 0, "n_atoms < 0");
  TBK_CHECK_ARG(row_ptr != nullptr && nnzb != nullptr, "row_ptr or nnzb is NULL");
  TBK_CHECK_ARG(n_atoms == 0 || pos != nullptr, "pos is NULL");
  TBK_CHECK_ARG(cutoff > 0.0 && std::isfinite(cutoff), "cutoff must be positive");
  DeviceGuard dg(ctx);
  const int n = n_atoms;
  CellGrid g{};
  g.periodic = box != nullptr;
  if (n == 0) {
    TBK_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int32_t), ctx->stream));
    sync(ctx);
    *nnzb = 0;
    return TBK_OK;
  }
  // Bounding box (open directions) -- read back to size the grid.
  const int bb_blocks = std::min(ceil_div(n, 256), 1024);
  double* part = (double*)scratch(ctx, WS_MISC, sizeof(double) * 6 * bb_blocks);
  bbox_partial<<<bb_blocks, 256, 0, ctx->stream>>>(pos, n, part);
  post_launch(ctx, "bbox_partial");
  std::vector<double> hp(6 * bb_blocks);
  TBK_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * 6 * bb_blocks, cudaMemcpyDeviceToHost,
                           ctx->stream));
  sync(ctx);
  double lo[3], hi[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = INFINITY;
    hi[c] = -INFINITY;
    for (int b = 0; b < bb_blocks; ++b) {
      lo[c] = std::min(lo[c], hp[6 * b + c]);
      hi[c] = std::max(hi[c], hp[6 * b + 3 + c]);
    }
    TBK_CHECK_ARG(std::isfinite(lo[c]) && std::isfinite(hi[c]), "positions must be finite");
  }
  int64_t ncells = 1;
  for (int c = 0; c < 3; ++c) {
    if (box) {
      const double L = box[c];
      TBK_CHECK_ARG(L > 2.0 * cutoff, "periodic box must be longer than 2 cutoffs (unique minimum image)");
      g.box[c] = L;
      g.lo[c] = 0.0;
      g.nc[c] = (int)std::floor(L / cutoff);
      g.cs[c] = L / g.nc[c];
    } else {
      g.box[c] = 0.0;
      g.lo[c] = lo[c];
      const double ext = hi[c] - lo[c];
      g.nc[c] = std::max(1, (int)std::min(std::floor(ext / cutoff), 1.0e6));
      g.cs[c] = g.nc[c] > 1 ? ext / g.nc[c] : std::max(ext, cutoff) * 1.000001 + 1e-300;
    }
  }
  // Keep the grid at most ~8 cells per atom (coarser cells stay correct: edge >= cutoff).
  if (!box) {
    while ((int64_t)g.nc[0] * g.nc[1] * g.nc[2] > 8LL * n + 1024) {
      int c = (g.nc[0] >= g.nc[1] && g.nc[0] >= g.nc[2]) ? 0 : (g.nc[1] >= g.nc[2] ? 1 : 2);
      g.nc[c] = std::max(1, g.nc[c] / 2);
      g.cs[c] = g.nc[c] > 1 ? (hi[c] - lo[c]) / g.nc[c] : std::max(hi[c] - lo[c], cutoff) * 1.000001;
    }
  } else {
    TBK_CHECK_ARG((int64_t)g.nc[0] * g.nc[1] * g.nc[2] <= 64LL * n + 4096,
                  "periodic box is too large for the number of atoms");
  }
  ncells = (int64_t)g.nc[0] * g.nc[1] * g.nc[2];

  int32_t* atom_cell = (int32_t*)scratch(ctx, WS_CELLS, sizeof(int32_t) * (size_t)n);
  int32_t* cell_count = (int32_t*)scratch(ctx, WS_CELLS2, sizeof(int32_t) * (size_t)(ncells + n + 1) * 2);
  int32_t* cursor = cell_count + (ncells + n + 1);   // second half: cursors / row counts
  int64_t* cell_start = (int64_t*)scratch(ctx, WS_CELLS3, sizeof(int64_t) * (size_t)(ncells + 1 + n + 1));
  int64_t* row_start = cell_start + (ncells + 1);
  const size_t tmp_elems = scan_tmp_elems(std::max<int64_t>(ncells, n));
  int32_t* cell_atoms = (int32_t*)scratch(ctx, WS_MISC, sizeof(int32_t) * (size_t)n + sizeof(int64_t) * (tmp_elems + 8));
  int64_t* tmp = (int64_t*)(((uintptr_t)(cell_atoms + n) + 15) & ~(uintptr_t)15);

  TBK_CUDA(cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * (size_t)ncells, ctx->stream));
  TBK_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)ncells, ctx->stream));
  assign_cells<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(pos, n, g, atom_cell, cell_count);
  post_launch(ctx, "assign_cells");
  exclusive_scan_i32(ctx, cell_count, cell_start, ncells, tmp);
  fill_cells<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(n, atom_cell, cell_start, cursor, cell_atoms);
  post_launch(ctx, "fill_cells");

  const double rc2 = cutoff * cutoff;
  int32_t* counts = cursor;  // reuse: cursors are no longer needed
  pair_pass<<<ceil_div(n, 128), 128, 0, ctx->stream>>>(pos, n, g, rc2, atom_cell, cell_start,
                                                       cell_atoms, counts, nullptr, nullptr);
  post_launch(ctx, "pair_count");
  exclusive_scan_i32(ctx, counts, row_start, n, tmp);
  int64_t total = 0;
  TBK_CUDA(cudaMemcpyAsync(&total, row_start + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  TBK_CHECK_ARG(total < (int64_t)INT32_MAX, "more than 2^31 - 1 pairs");
  *nnzb = total;
  to_i32<<<ceil_div(n + 1, 256), 256, 0, ctx->stream>>>(row_start, row_ptr, n + 1);
  post_launch(ctx, "row_ptr_i32");
  if (col) {
    TBK_CHECK_ARG(col_capacity >= total, "col_capacity is smaller than the number of pairs");
    pair_pass<<<ceil_div(n, 128), 128, 0, ctx->stream>>>(pos, n, g, rc2, atom_cell, cell_start,
                                                         cell_atoms, nullptr, row_start, col);
    post_launch(ctx, "pair_fill");
  }
  sync(ctx);
  TBK_API_END
}

// ---- many open clusters at once ----------------------------------------------------------------
//
// The same pattern as one tbk_build_neighbors call per cluster, with every pass run once over the
// atoms of all clusters: the clusters' positions are gathered into one array, each atom carries
// its cluster, and the clusters' cell grids lie end to end (cluster c's cells from coff[c]), so a
// cell holds atoms of one cluster only.  Columns are written cluster-local.

namespace tbk {

struct BatchGrid {
  const CellGrid* grid;    // per cluster
  const int64_t* coff;     // first cell of each cluster
  const int32_t* aoff;     // first atom of each cluster (n_clusters + 1 entries)
  const int32_t* atom_cl;  // cluster of each atom
};

__global__ void atom_clusters(const int32_t* __restrict__ aoff, int32_t* __restrict__ atom_cl) {
  const int c = blockIdx.x;  // one block per cluster
  for (int i = aoff[c] + threadIdx.x; i < aoff[c + 1]; i += blockDim.x) atom_cl[i] = c;
}

__global__ void assign_cells_batched(const double* __restrict__ pos, int n, BatchGrid b,
                                     int32_t* __restrict__ atom_cell, int32_t* __restrict__ cell_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cl = b.atom_cl[i];
  const CellGrid g = b.grid[cl];
  const int cx = cell_coord(pos[3 * i], g, 0), cy = cell_coord(pos[3 * i + 1], g, 1),
            cz = cell_coord(pos[3 * i + 2], g, 2);
  const int64_t c = b.coff[cl] + ((int64_t)cx * g.nc[1] + cy) * g.nc[2] + cz;
  atom_cell[i] = (int32_t)c;
  atomicAdd(&cell_count[c], 1);
}

// One thread per atom of the batch: count (cols == nullptr) or write the row's cluster-local
// columns into cols[cluster] at row_start[i] - row_start[first atom of the cluster], then sort.
__global__ void pair_pass_batched(const double* __restrict__ pos, int n, BatchGrid b, double rc2,
                                  const int32_t* __restrict__ atom_cell,
                                  const int64_t* __restrict__ cell_start,
                                  const int32_t* __restrict__ cell_atoms, int32_t* __restrict__ count,
                                  const int64_t* __restrict__ row_start, int32_t* const* __restrict__ cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cl = b.atom_cl[i];
  const CellGrid g = b.grid[cl];
  const int64_t c0 = b.coff[cl];
  const int a0 = b.aoff[cl];
  const int64_t lc = atom_cell[i] - c0;
  const int cz = (int)(lc % g.nc[2]), cy = (int)((lc / g.nc[2]) % g.nc[1]),
            cx = (int)(lc / ((int64_t)g.nc[1] * g.nc[2]));
  int32_t* col = cols ? cols[cl] : nullptr;
  const int64_t out = col ? row_start[i] - row_start[a0] : 0;
  int cnt = 0;
  for (int x = cx - 1; x <= cx + 1; ++x) {
    if (x < 0 || x >= g.nc[0]) continue;
    for (int y = cy - 1; y <= cy + 1; ++y) {
      if (y < 0 || y >= g.nc[1]) continue;
      for (int z = cz - 1; z <= cz + 1; ++z) {
        if (z < 0 || z >= g.nc[2]) continue;
        const int64_t cc = c0 + ((int64_t)x * g.nc[1] + y) * g.nc[2] + z;
        for (int64_t k = cell_start[cc]; k < cell_start[cc + 1]; ++k) {
          const int j = cell_atoms[k];
          if (j == i || pair_r2(pos, i, j, g) <= rc2) {
            if (col) col[out + cnt] = j - a0;
            ++cnt;
          }
        }
      }
    }
  }
  if (!col) {
    count[i] = cnt;
    return;
  }
  int32_t* r = col + out;
  for (int a = 1; a < cnt; ++a) {
    const int32_t v = r[a];
    int q = a - 1;
    while (q >= 0 && r[q] > v) {
      r[q + 1] = r[q];
      --q;
    }
    r[q + 1] = v;
  }
}

// totals[c] = pairs of cluster c; row_ptr of cluster c = row_start over its rows, less its first
__global__ void cluster_totals(int n_clusters, const int32_t* __restrict__ aoff,
                               const int64_t* __restrict__ row_start, int64_t* __restrict__ totals) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_clusters) totals[c] = row_start[aoff[c + 1]] - row_start[aoff[c]];
}

__global__ void row_ptrs_batched(const int32_t* __restrict__ aoff, const int64_t* __restrict__ row_start,
                                 int32_t* const* __restrict__ rps) {
  const int c = blockIdx.x;  // one block per cluster
  const int a0 = aoff[c], nc = aoff[c + 1] - a0;
  const int64_t base = row_start[a0];
  for (int r = threadIdx.x; r <= nc; r += blockDim.x) rps[c][r] = (int32_t)(row_start[a0 + r] - base);
}

// The cell grid of an open cluster with bounding box [lo, hi] (the rules of tbk_build_neighbors).
static CellGrid open_grid(const double lo[3], const double hi[3], double cutoff, int n) {
  CellGrid g{};
  g.periodic = 0;
  for (int c = 0; c < 3; ++c) {
    g.box[c] = 0.0;
    g.lo[c] = lo[c];
    const double ext = hi[c] - lo[c];
    g.nc[c] = std::max(1, (int)std::min(std::floor(ext / cutoff), 1.0e6));
    g.cs[c] = g.nc[c] > 1 ? ext / g.nc[c] : std::max(ext, cutoff) * 1.000001 + 1e-300;
  }
  while ((int64_t)g.nc[0] * g.nc[1] * g.nc[2] > 8LL * n + 1024) {
    const int c = (g.nc[0] >= g.nc[1] && g.nc[0] >= g.nc[2]) ? 0 : (g.nc[1] >= g.nc[2] ? 1 : 2);
    g.nc[c] = std::max(1, g.nc[c] / 2);
    g.cs[c] = g.nc[c] > 1 ? (hi[c] - lo[c]) / g.nc[c] : std::max(hi[c] - lo[c], cutoff) * 1.000001;
  }
  return g;
}

}  // namespace tbk

extern "C" int tbk_batched_build_neighbors(tbk_ctx* ctx, int32_t n_clusters, const double* const* pos,
                                           const int32_t* n_atoms, double cutoff, int32_t* const* row_ptr,
                                           int32_t* const* col, const int64_t* col_capacity,
                                           int64_t* nnzb) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG(n_clusters >= 1, "n_clusters must be >= 1");
  TBK_CHECK_ARG(pos && n_atoms && row_ptr && nnzb, "NULL argument");
  TBK_CHECK_ARG(cutoff > 0.0 && std::isfinite(cutoff), "cutoff must be positive");
  TBK_CHECK_ARG(col == nullptr || col_capacity != nullptr, "col_capacity is NULL");
  const int ncl = n_clusters;
  std::vector<int32_t> aoff(ncl + 1, 0);
  for (int c = 0; c < ncl; ++c) {
    TBK_CHECK_ARG(n_atoms[c] >= 1, "every cluster needs at least one atom");
    TBK_CHECK_ARG(pos[c] != nullptr && row_ptr[c] != nullptr, "NULL position or row_ptr array");
    TBK_CHECK_ARG((int64_t)aoff[c] + n_atoms[c] < INT32_MAX, "more than 2^31 - 1 atoms in the batch");
    aoff[c + 1] = aoff[c] + n_atoms[c];
  }
  const int n = aoff[ncl];
  DeviceGuard dg(ctx);

  // bounding boxes of all clusters, read back once
  std::vector<int> bbb(ncl), pboff(ncl + 1, 0);
  for (int c = 0; c < ncl; ++c) {
    bbb[c] = std::min(ceil_div(n_atoms[c], 256), 1024);
    pboff[c + 1] = pboff[c] + bbb[c];
  }
  // WS_SEGMENT: gathered positions | bbox partials | grids | coff | aoff | totals | pointers
  const size_t o_pos = 0;
  const size_t o_part = o_pos + sizeof(double) * 3 * (size_t)n;
  const size_t o_grid = o_part + sizeof(double) * 6 * (size_t)pboff[ncl];
  const size_t o_coff = o_grid + sizeof(CellGrid) * ncl;
  const size_t o_aoff = o_coff + sizeof(int64_t) * ncl;
  const size_t o_tot = (o_aoff + sizeof(int32_t) * (ncl + 1) + 15) & ~(size_t)15;
  const size_t o_rps = o_tot + sizeof(int64_t) * ncl;
  const size_t o_cols = o_rps + sizeof(int32_t*) * ncl;
  const size_t seg_bytes = o_cols + sizeof(int32_t*) * ncl;
  char* seg = (char*)scratch(ctx, WS_SEGMENT, seg_bytes);
  double* pos_all = (double*)(seg + o_pos);
  double* part = (double*)(seg + o_part);
  for (int c = 0; c < ncl; ++c) {
    TBK_CUDA(cudaMemcpyAsync(pos_all + 3 * (size_t)aoff[c], pos[c], sizeof(double) * 3 * n_atoms[c],
                             cudaMemcpyDeviceToDevice, ctx->stream));
    bbox_partial<<<bbb[c], 256, 0, ctx->stream>>>(pos[c], n_atoms[c], part + 6 * (size_t)pboff[c]);
    post_launch(ctx, "bbox_partial");
  }
  std::vector<double> hp(6 * (size_t)pboff[ncl]);
  TBK_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  std::vector<CellGrid> grids(ncl);
  std::vector<int64_t> coff(ncl);
  int64_t ncells = 0;
  for (int c = 0; c < ncl; ++c) {
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = INFINITY;
      hi[d] = -INFINITY;
      for (int b = pboff[c]; b < pboff[c + 1]; ++b) {
        lo[d] = std::min(lo[d], hp[6 * (size_t)b + d]);
        hi[d] = std::max(hi[d], hp[6 * (size_t)b + 3 + d]);
      }
      TBK_CHECK_ARG(std::isfinite(lo[d]) && std::isfinite(hi[d]), "positions must be finite");
    }
    grids[c] = open_grid(lo, hi, cutoff, n_atoms[c]);
    coff[c] = ncells;
    ncells += (int64_t)grids[c].nc[0] * grids[c].nc[1] * grids[c].nc[2];
  }
  TBK_CHECK_ARG(ncells < INT32_MAX, "too many cells in the batch");
  CellGrid* d_grid = (CellGrid*)(seg + o_grid);
  int64_t* d_coff = (int64_t*)(seg + o_coff);
  int32_t* d_aoff = (int32_t*)(seg + o_aoff);
  int64_t* d_tot = (int64_t*)(seg + o_tot);
  int32_t** d_rps = (int32_t**)(seg + o_rps);
  int32_t** d_cols = (int32_t**)(seg + o_cols);
  TBK_CUDA(cudaMemcpyAsync(d_grid, grids.data(), sizeof(CellGrid) * ncl, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_coff, coff.data(), sizeof(int64_t) * ncl, cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_aoff, aoff.data(), sizeof(int32_t) * (ncl + 1), cudaMemcpyHostToDevice, ctx->stream));
  TBK_CUDA(cudaMemcpyAsync(d_rps, row_ptr, sizeof(int32_t*) * ncl, cudaMemcpyHostToDevice, ctx->stream));

  int32_t* atom_cell = (int32_t*)scratch(ctx, WS_CELLS, sizeof(int32_t) * 2 * (size_t)n);
  int32_t* atom_cl = atom_cell + n;
  int32_t* cell_count = (int32_t*)scratch(ctx, WS_CELLS2, sizeof(int32_t) * (size_t)(ncells + n + 1) * 2);
  int32_t* cursor = cell_count + (ncells + n + 1);   // then the row counts
  int64_t* cell_start = (int64_t*)scratch(ctx, WS_CELLS3, sizeof(int64_t) * (size_t)(ncells + 1 + n + 1));
  int64_t* row_start = cell_start + (ncells + 1);
  const size_t tmp_elems = scan_tmp_elems(std::max<int64_t>(ncells, n));
  int32_t* cell_atoms = (int32_t*)scratch(ctx, WS_MISC, sizeof(int32_t) * (size_t)n + sizeof(int64_t) * (tmp_elems + 8));
  int64_t* tmp = (int64_t*)(((uintptr_t)(cell_atoms + n) + 15) & ~(uintptr_t)15);
  const BatchGrid bg{d_grid, d_coff, d_aoff, atom_cl};

  atom_clusters<<<ncl, 256, 0, ctx->stream>>>(d_aoff, atom_cl);
  post_launch(ctx, "atom_clusters");
  TBK_CUDA(cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * (size_t)ncells, ctx->stream));
  TBK_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)ncells, ctx->stream));
  assign_cells_batched<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(pos_all, n, bg, atom_cell, cell_count);
  post_launch(ctx, "assign_cells_batched");
  exclusive_scan_i32(ctx, cell_count, cell_start, ncells, tmp);
  fill_cells<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(n, atom_cell, cell_start, cursor, cell_atoms);
  post_launch(ctx, "fill_cells");
  const double rc2 = cutoff * cutoff;
  int32_t* counts = cursor;
  pair_pass_batched<<<ceil_div(n, 128), 128, 0, ctx->stream>>>(pos_all, n, bg, rc2, atom_cell, cell_start,
                                                               cell_atoms, counts, nullptr, nullptr);
  post_launch(ctx, "pair_count_batched");
  exclusive_scan_i32(ctx, counts, row_start, n, tmp);
  cluster_totals<<<ceil_div(ncl, 128), 128, 0, ctx->stream>>>(ncl, d_aoff, row_start, d_tot);
  post_launch(ctx, "cluster_totals");
  row_ptrs_batched<<<ncl, 256, 0, ctx->stream>>>(d_aoff, row_start, d_rps);
  post_launch(ctx, "row_ptrs_batched");
  std::vector<int64_t> tot(ncl);
  TBK_CUDA(cudaMemcpyAsync(tot.data(), d_tot, sizeof(int64_t) * ncl, cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  bool fits = col != nullptr;
  for (int c = 0; c < ncl; ++c) {
    TBK_CHECK_ARG(tot[c] < (int64_t)INT32_MAX, "more than 2^31 - 1 pairs in a cluster");
    nnzb[c] = tot[c];
    if (col && (col[c] == nullptr || col_capacity[c] < tot[c])) fits = false;
  }
  if (col) {
    TBK_CHECK_ARG(fits, "a col array is NULL or smaller than its cluster's number of pairs");
    TBK_CUDA(cudaMemcpyAsync(d_cols, col, sizeof(int32_t*) * ncl, cudaMemcpyHostToDevice, ctx->stream));
    pair_pass_batched<<<ceil_div(n, 128), 128, 0, ctx->stream>>>(pos_all, n, bg, rc2, atom_cell, cell_start,
                                                                 cell_atoms, nullptr, row_start, d_cols);
    post_launch(ctx, "pair_fill_batched");
  }
  sync(ctx);
  TBK_API_END
}
