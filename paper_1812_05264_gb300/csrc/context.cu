// Context, scratch management and the error channel of the C ABI.
#include <algorithm>

#include "common.cuh"

namespace tbk {

static thread_local std::string g_last_error;

void set_error(const char* msg) { g_last_error = msg ? msg : ""; }

size_t panel_budget(tbk_ctx* ctx, Slot s) {
  size_t fr = 0, tot = 0;
  TBK_CUDA(cudaMemGetInfo(&fr, &tot));
  const size_t have = fr + ctx->slot_bytes[s];
  const size_t reserve = ((size_t)2 << 30) + tot / 100 * 3;
  return have > reserve ? have - reserve : 0;
}

void* scratch(tbk_ctx* ctx, Slot s, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (ctx->slot_bytes[s] >= bytes) return ctx->slot_ptr[s];
  if (ctx->slot_ptr[s]) {
    const bool large = ctx->slot_bytes[s] > ((size_t)256 << 20);
    TBK_CUDA(cudaFreeAsync(ctx->slot_ptr[s], ctx->stream));
    ctx->slot_ptr[s] = nullptr;
    ctx->slot_bytes[s] = 0;
    if (large) {
      // hand the old block back to the device before the larger one is mapped, so that the two
      // never have to fit side by side
      TBK_CUDA(cudaStreamSynchronize(ctx->stream));
      cudaMemPool_t pool;
      TBK_CUDA(cudaDeviceGetDefaultMemPool(&pool, ctx->device));
      TBK_CUDA(cudaMemPoolTrimTo(pool, 0));
    }
  }
  // headroom so that slowly growing sizes do not thrash (at most 1 GiB)
  size_t want = bytes + std::min(bytes / 8, (size_t)1 << 30);
  want = (want + 255) & ~(size_t)255;
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, want, ctx->stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error(TBK_ERR_OOM, "device scratch allocation of " + std::to_string(want) +
                                 " bytes failed: " + cudaGetErrorString(e));
  }
  ctx->slot_ptr[s] = p;
  ctx->slot_bytes[s] = want;
  return p;
}

void* pinned(tbk_ctx* ctx, size_t bytes) {
  if (ctx->pinned_bytes >= bytes) return ctx->pinned;
  if (ctx->pinned) TBK_CUDA(cudaFreeHost(ctx->pinned));
  ctx->pinned = nullptr;
  ctx->pinned_bytes = 0;
  TBK_CUDA(cudaMallocHost(&ctx->pinned, bytes));
  ctx->pinned_bytes = bytes;
  return ctx->pinned;
}

void post_launch(tbk_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    throw Error(TBK_ERR_CUDA, std::string("launch of ") + what + " failed: " + cudaGetErrorString(e));
  ctx->launches++;
}

DeviceGuard::DeviceGuard(tbk_ctx* ctx) {
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != ctx->device) TBK_CUDA(cudaSetDevice(ctx->device));
}
DeviceGuard::~DeviceGuard() {
  int cur = -1;
  if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

void sync(tbk_ctx* ctx) { TBK_CUDA(cudaStreamSynchronize(ctx->stream)); }

const tbk_ctx::Tuned* find_tuned(const tbk_ctx* ctx, int64_t n_rows, int64_t nnzb, int s) {
  for (const auto& t : ctx->tuned)
    if (t.n_rows == n_rows && t.nnzb == nnzb && t.s == s) return &t;
  return nullptr;
}

static void timer_record(tbk_ctx* ctx) {
  if (ctx->timer_used == ctx->timer_events.size()) {
    cudaEvent_t e;
    TBK_CUDA(cudaEventCreate(&e));
    ctx->timer_events.push_back(e);
  }
  TBK_CUDA(cudaEventRecord(ctx->timer_events[ctx->timer_used], ctx->stream));
  ctx->timer_used++;
}

KernelTimerScope::KernelTimerScope(tbk_ctx* c, int kernel) {
  if (kernel <= 0 || kernel > 30 || !(c->timed_mask & (1 << kernel))) return;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  TBK_CUDA(cudaStreamIsCapturing(c->stream, &st));
  if (st != cudaStreamCaptureStatusNone) return;
  timer_record(c);
  const size_t pair = (c->timer_used - 1) / 2;
  if (c->timer_family.size() <= pair) c->timer_family.resize(pair + 1);
  c->timer_family[pair] = kernel;
  ctx = c;
}

KernelTimerScope::~KernelTimerScope() {
  if (!ctx) return;
  // the end event of the pair; on failure the begin event is dropped so pairs stay aligned
  try {
    timer_record(ctx);
  } catch (...) {
    ctx->timer_used--;
  }
}

}  // namespace tbk

extern "C" {

int tbk_create(tbk_ctx** out, int device, void* stream) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(out != nullptr, "out is NULL");
  int n = 0;
  TBK_CUDA(cudaGetDeviceCount(&n));
  TBK_CHECK_ARG(device >= 0 && device < n, "no such CUDA device");
  tbk_ctx* c = new tbk_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (prev >= 0) cudaSetDevice(prev);
  *out = c;
  TBK_API_END
}

int tbk_destroy(tbk_ctx* ctx) {
  TBK_API_BEGIN
  if (!ctx) return TBK_OK;
  {
    tbk::DeviceGuard g(ctx);
    cudaStreamSynchronize(ctx->stream);
    for (int s = 0; s < tbk::WS_NSLOTS; ++s)
      if (ctx->slot_ptr[s]) cudaFree(ctx->slot_ptr[s]);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    for (cudaEvent_t e : ctx->timer_events) cudaEventDestroy(e);
  }
  delete ctx;
  TBK_API_END
}

const char* tbk_last_error(void) { return tbk::g_last_error.c_str(); }

int tbk_test_stall_next_step(tbk_ctx* ctx) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  ctx->stall_next_step = 1;
  TBK_API_END
}

int tbk_test_stall_next_adjoint(tbk_ctx* ctx) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  ctx->stall_next_adjoint = 1;
  TBK_API_END
}

int tbk_kernel_timer(tbk_ctx* ctx, int32_t mask) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG((mask & ~((2 << TBK_KERNEL_WINDOW) - 2)) == 0, "unknown kernel family");
  ctx->timed_mask = mask;
  ctx->timer_used = 0;
  TBK_API_END
}

int tbk_kernel_timer_read(tbk_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && total_ms && launches, "NULL argument");
  tbk::DeviceGuard g(ctx);
  tbk::sync(ctx);
  double t = 0.0;
  int64_t n = 0;
  for (size_t i = 0; i + 1 < ctx->timer_used; i += 2) {
    if (ctx->timer_family[i / 2] != kernel) continue;
    float ms = 0.f;
    TBK_CUDA(cudaEventElapsedTime(&ms, ctx->timer_events[i], ctx->timer_events[i + 1]));
    t += ms;
    ++n;
  }
  *total_ms = t;
  *launches = n;
  TBK_API_END
}

int64_t tbk_launch_count(tbk_ctx* ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"
