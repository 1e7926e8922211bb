// Internal helpers shared by the libtbk translation units: the context, device scratch,
// error handling across the C ABI, and small device utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tbk.h"

namespace tbk {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_error(const char* msg);

#define TBK_CHECK_ARG(cond, msg)                                              \
  do {                                                                        \
    if (!(cond)) throw ::tbk::Error(TBK_ERR_ARG, std::string(__func__) + ": " + (msg)); \
  } while (0)

#define TBK_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t _e = (call);                                                  \
    if (_e != cudaSuccess)                                                    \
      throw ::tbk::Error(_e == cudaErrorMemoryAllocation ? TBK_ERR_OOM : TBK_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// Named scratch slots.  Each slot is a grow-only device buffer owned by the context.
enum Slot {
  WS_PANEL0 = 0, WS_PANEL1, WS_PANEL2, WS_PANEL3, WS_HHAT, WS_PARTIALS, WS_FLAGS, WS_COEF,
  WS_TABLE, WS_NODES, WS_CELLS, WS_CELLS2, WS_CELLS3, WS_LANCZOS, WS_GACC, WS_TRANSPOSE,
  WS_CHECKPOINTS, WS_SEGMENT, WS_MISC, WS_PROBES,
  WS_LOCAL0, WS_LOCAL1, WS_LOCAL2, WS_LOCAL3, WS_LOCAL4, WS_NSLOTS
};

}  // namespace tbk

struct tbk_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t launches = 0;
  void* slot_ptr[tbk::WS_NSLOTS] = {};
  size_t slot_bytes[tbk::WS_NSLOTS] = {};
  void* pinned = nullptr;        // small pinned host buffer for scalar read-back
  size_t pinned_bytes = 0;
  int stall_next_step = 0;       // test hook: the next TMA-fed step's producer issues no copies
  int stall_next_adjoint = 0;    // test hook: the next fused adjoint step's producer issues no copies
  struct Tuned {                 // tbk_autotune's choices, per operator shape and probe count
    int64_t n_rows, nnzb;
    int s, cw, windowed;        // windowed: the outer-product schedule (0 fused, 1 windowed, 2 tensor cores)
  };
  std::vector<Tuned> tuned;
  int timed_mask = 0;            // bit f set: launches of kernel family f are bracketed by events
  std::vector<cudaEvent_t> timer_events;  // (begin, end) pairs
  std::vector<int> timer_family;          // family of each pair
  size_t timer_used = 0;                  // events in use
};

namespace tbk {

// Device scratch of at least `bytes` in slot s (contents undefined after growth).
void* scratch(tbk_ctx* ctx, Slot s, size_t bytes);
// Pinned host staging of at least `bytes`.
void* pinned(tbk_ctx* ctx, size_t bytes);
// Check the launch that was just enqueued and count it.
void post_launch(tbk_ctx* ctx, const char* what);
// Make ctx->device current for the scope.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(tbk_ctx* ctx);
  ~DeviceGuard();
};
void sync(tbk_ctx* ctx);
// The tuned choice for an operator of n_rows rows and nnzb blocks at s probes, or NULL.
const tbk_ctx::Tuned* find_tuned(const tbk_ctx* ctx, int64_t n_rows, int64_t nnzb, int s);
// Device bytes that slot s may grow to: what is free plus what s already holds, less a reserve
// of 2 GiB + 3 % of the device for everything else.
size_t panel_budget(tbk_ctx* ctx, Slot s);
// Brackets the launches of one kernel family with events on ctx->stream when that family is
// selected by tbk_kernel_timer (and the stream is not being captured into a graph).
struct KernelTimerScope {
  tbk_ctx* ctx = nullptr;
  KernelTimerScope(tbk_ctx* c, int kernel);
  ~KernelTimerScope();
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// One cluster's chemical-potential solve in a batch: M quadrature nodes, order p, moments at
// mom_off, cosine table (4M doubles) at tab_off and node weights (M doubles) at rho_off of one
// scratch buffer.
struct FermiJob {
  int M, p;
  double emin, emax, n_e, kT;
  int64_t mom_off, tab_off, rho_off;
};
void fermi_enqueue_batched(tbk_ctx* ctx, int n, const FermiJob* d_jobs, int M_max, const double* moments,
                           int damping, double* buf, double* res);

}  // namespace tbk

#define TBK_API_BEGIN try {
#define TBK_API_END                                                           \
  }                                                                           \
  catch (const ::tbk::Error& e) {                                             \
    ::tbk::set_error(e.what());                                               \
    return e.code;                                                            \
  }                                                                           \
  catch (const std::exception& e) {                                           \
    ::tbk::set_error(e.what());                                               \
    return TBK_ERR_CUDA;                                                      \
  }                                                                           \
  ::tbk::set_error("");                                                       \
  return TBK_OK;

// ---------------------------------------------------------------------------------------
// Device utilities
// ---------------------------------------------------------------------------------------

// Rademacher probe entry for (row, probe): SplitMix64 output number (row * 2^32 + probe + 1)
// of a stream seeded with `seed` (Steele, Lea & Flood, OOPSLA 2014; mix64 finaliser of
// java.util.SplittableRandom).  Returns +1 or -1.
__device__ __forceinline__ float tbk_probe_sign(uint64_t seed, uint64_t row, uint64_t probe) {
  uint64_t z = seed + ((row << 32) + probe + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (z >> 63) ? -1.0f : 1.0f;
}

// Fixed-order block reduction of one double (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ double tbk_block_sum(double v, double* smem32) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) smem32[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < nwarps ? smem32[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}
