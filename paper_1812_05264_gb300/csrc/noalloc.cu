// tbk_chebyshev_moments_noalloc: the Chebyshev moments (same kernels and results as
// tbk_chebyshev_moments) with every piece of device scratch taken from one fixed array that is
// part of the library image, so that the call itself never allocates device memory.
//
// Who needs this: callers that must not allocate while they run -- code that enqueues work
// from inside a real-time or latency-bounded loop where an allocation can block on the device,
// embedders whose device memory is budgeted up front by a framework that owns all allocations,
// and drivers that forbid allocation between set-up and shutdown.  They still provide H and the
// output buffer; only the library's own scratch moves into the static array.
#include <mutex>

#include "cheb.cuh"

namespace tbk {

// 64 MiB of scratch, reserved on every device that loads the library, for the life of the
// process.  Enough for e.g. 1,000 atoms x 9 orbitals x 256 probes in mixed precision.
constexpr size_t kStaticScratchBytes = TBK_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_tbk_static_scratch[kStaticScratchBytes];

// Device address of the array, looked up once per device with that device current (under lazy
// module loading this lookup also loads the module, which commits the array's device memory).  The
// address belongs to the device's primary context: it stays valid while that context lives, i.e.
// until the process exits or calls cudaDeviceReset.  In host code
// the symbol name is only a host-side stand-in: handing it to a kernel would fault or, where the
// GPU can reach host memory, silently use the wrong memory.  Only the address returned by
// cudaGetSymbolAddress is passed to kernels.
static void* static_scratch_address(int device) {
  static std::mutex mu;
  static void* addr[256] = {};
  TBK_CHECK_ARG(device >= 0 && device < 256, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_tbk_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error(TBK_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                    cudaGetErrorString(e));
    addr[device] = p;
  }
  return addr[device];
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Switches the context's kernel timer off for the scope: a timed launch records CUDA events, and
// the first events of a context are created on demand, which this entry point must not do.
struct TimerOff {
  tbk_ctx* ctx;
  int mask;
  explicit TimerOff(tbk_ctx* c) : ctx(c), mask(c->timed_mask) { c->timed_mask = 0; }
  ~TimerOff() { ctx->timed_mask = mask; }
};

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_chebyshev_moments_noalloc(tbk_ctx* ctx, const tbk_bsr* H, double emin,
                                             double emax, uint64_t probe_seed, int32_t n_probes,
                                             int32_t order, int32_t flags, double* moments) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG(H != nullptr, "H is NULL");
  TBK_CHECK_ARG(moments != nullptr, "moments is NULL");
  TBK_CHECK_ARG(order >= 1, "order must be >= 1");
  TBK_CHECK_ARG(n_probes >= 4 && n_probes % 4 == 0, "n_probes must be a positive multiple of 4");
  TBK_CHECK_ARG((flags & ~(TBK_FP64 | TBK_MOMENTS_DIRECT | TBK_PLAIN_KERNEL)) == 0, "unknown flag");
  TBK_CHECK_ARG(H->n_orb == 1 || H->n_orb == 9, "n_orb must be 1 or 9");
  TBK_CHECK_ARG(H->n_atoms >= 1 && H->nnzb >= H->n_atoms, "empty or inconsistent matrix");
  TBK_CHECK_ARG(H->nnzb < INT32_MAX, "nnzb must be below 2^31");
  TBK_CHECK_ARG(H->row_ptr != nullptr && H->col != nullptr && H->val != nullptr,
                "H->row_ptr, H->col or H->val is NULL");
  DeviceGuard dg(ctx);
  TimerOff no_events(ctx);
  unsigned char* base = (unsigned char*)static_scratch_address(ctx->device);
  const int prec = (flags & TBK_FP64) ? TBK_FP64 : TBK_MIXED;
  const int direct = (flags & TBK_MOMENTS_DIRECT) ? 1 : 0;
  const int s = n_probes;
  const size_t esz = prec == TBK_MIXED ? 4 : 8;
  const int64_t n_rows = (int64_t)H->n_atoms * H->n_orb;
  const size_t panel = (size_t)n_rows * s * esz;
  const int K = direct ? order - 1 : order / 2;
  HOp shape;
  shape.B = H->n_orb;
  shape.prec = prec;
  shape.n_atoms = H->n_atoms;
  shape.n_rows = n_rows;    // the grid follows any tuned choice for this shape, as the steps do
  shape.nnzb = H->nnzb;
  const int nctas = step_grid_ctas(ctx, shape, s);
  // layout: flag | sums | partials | mapped H | panel A | panel B, each 256-byte aligned
  const size_t o_flag = 0;
  const size_t o_sums = o_flag + 256;
  const size_t o_part = o_sums + align256(sizeof(double) * 2 * (size_t)std::max(1, K) + 64);
  const size_t o_hhat = o_part + align256(sizeof(double) * 2 * (size_t)std::max(1, K) * nctas);
  const size_t o_pa = o_hhat + align256(mapped_h_bytes(H, prec));
  const size_t o_pb = o_pa + (K >= 1 ? align256(panel) : 0);
  const size_t need = o_pb + (K >= 2 ? align256(panel) : 0);
  if (need > kStaticScratchBytes)
    throw Error(TBK_ERR_ARG, "tbk_chebyshev_moments_noalloc: this problem needs " +
                                 std::to_string(need) + " bytes of scratch, above the static limit of " +
                                 std::to_string(kStaticScratchBytes) +
                                 " bytes; use tbk_chebyshev_moments");
  int* flag = (int*)(base + o_flag);
  double* sums = (double*)(base + o_sums);
  double* partials = (double*)(base + o_part);
  void* A = K >= 1 ? (void*)(base + o_pa) : nullptr;
  void* Bp = K >= 2 ? (void*)(base + o_pb) : nullptr;
  // the array keeps the previous call's contents: the error flag must start at zero
  TBK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  HOp op = prepare_hop_into(ctx, H, emin, emax, prec, base + o_hhat, flag);
  void *cur = nullptr, *prev = nullptr;
  for (int j = 1; j <= K; ++j) {
    StepArgs a;
    a.seed = probe_seed;
    a.s = s;
    a.direct = direct;
    a.partials = partials + (size_t)(j - 1) * nctas * 2;
    a.err = flag;
    a.force_simple = (flags & TBK_PLAIN_KERNEL) ? 1 : 0;
    if (j == 1) {
      a.cur_is_probe = 1;
      a.alpha = 1.0;
      a.yout = A;
      cur = A;
    } else if (j == 2) {
      a.yin = A;
      a.alpha = 2.0;
      a.c_r = -1.0;
      a.yout = Bp;
      prev = A;
      cur = Bp;
    } else {
      a.yin = cur;
      a.yprev = prev;
      a.yout = prev;
      a.alpha = 2.0;
      std::swap(cur, prev);
    }
    launch_step(ctx, op, a);
  }
  launch_moment_reduction(ctx, partials, nctas, K, order, s, op.n_rows, direct, sums, moments, flag);
  int hflag = 0;
  TBK_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(hflag);
  if (hflag & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait in the recurrence kernel expired");
  if (hflag)
    throw Error(TBK_ERR_SPECTRUM, "a Chebyshev panel grew beyond ||r||: the spectrum of H is not "
                                  "inside [emin, emax]");
  TBK_API_END
}
