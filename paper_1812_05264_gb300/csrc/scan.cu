#include "scan.cuh"

namespace tbk {

static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_ITEMS = 4;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total) {
  // Hillis-Steele over the block's per-thread sums (256 threads).
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < SCAN_THREADS; o <<= 1) {
    int64_t a = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += a;
    __syncthreads();
  }
  int64_t incl = sh[t];
  *total = sh[SCAN_THREADS - 1];
  return incl - v;
}

__global__ void scan_tiles(const int32_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                           int64_t* __restrict__ tile_sums) {
  __shared__ int64_t sh[SCAN_THREADS];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = (base + i < n) ? (int64_t)in[base + i] : 0;
    s += v[i];
  }
  int64_t total;
  int64_t run = block_exclusive_scan(s, sh, &total);
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the tile sums in place, grand total to *grand.
__global__ void scan_sums(int64_t* __restrict__ sums, int64_t m, int64_t* __restrict__ grand) {
  __shared__ int64_t sh[SCAN_THREADS];
  const int64_t per = (m + SCAN_THREADS - 1) / SCAN_THREADS;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  int64_t s = 0;
  for (int64_t i = b0; i < b0 + per && i < m; ++i) s += sums[i];
  int64_t total;
  int64_t run = block_exclusive_scan(s, sh, &total);
  for (int64_t i = b0; i < b0 + per && i < m; ++i) {
    int64_t x = sums[i];
    sums[i] = run;
    run += x;
  }
  if (threadIdx.x == 0) *grand = total;
}

__global__ void scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ sums,
                         const int64_t* __restrict__ grand) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[i / SCAN_TILE];
  if (i == 0) out[n] = *grand;
}

size_t scan_tmp_elems(int64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 2; }

void exclusive_scan_i32(tbk_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, int64_t* tmp) {
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* grand = tmp + tiles;
  if (n > 0) {
    scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, ctx->stream>>>(in, out, n, tmp);
    post_launch(ctx, "scan_tiles");
  }
  scan_sums<<<1, SCAN_THREADS, 0, ctx->stream>>>(tmp, tiles, grand);
  post_launch(ctx, "scan_sums");
  scan_add<<<(unsigned)((n + 256) / 256), 256, 0, ctx->stream>>>(out, n, tmp, grand);
  post_launch(ctx, "scan_add");
}

}  // namespace tbk
