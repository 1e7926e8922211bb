// Context, scratch management and the error channel of the C ABI.
#include "common.cuh"

namespace tbk {

static thread_local std::string g_last_error;

void set_error(const char* msg) { g_last_error = msg ? msg : ""; }

void* scratch(tbk_ctx* ctx, Slot s, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (ctx->slot_bytes[s] >= bytes) return ctx->slot_ptr[s];
  if (ctx->slot_ptr[s]) {
    TBK_CUDA(cudaFreeAsync(ctx->slot_ptr[s], ctx->stream));
    ctx->slot_ptr[s] = nullptr;
    ctx->slot_bytes[s] = 0;
  }
  size_t want = bytes + bytes / 8;  // headroom so that slowly growing sizes do not thrash
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
  }
  delete ctx;
  TBK_API_END
}

const char* tbk_last_error(void) { return tbk::g_last_error.c_str(); }

int64_t tbk_launch_count(tbk_ctx* ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"
