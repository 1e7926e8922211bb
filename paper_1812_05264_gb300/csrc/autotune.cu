// Timing-based choices per operator shape and probe count, kept in the context: the probe chunk
// (128, 256 or 512 probes) of each task of the TMA-fed recurrence step, and the schedule of the
// adjoint's outer products (inside each fused backward step, summed over windows of steps by
// their own kernel, or on the tensor cores after each backward step).  Every candidate computes the same results up to FP32 summation order; the
// choice only changes how the work is cut.
#include <cmath>
#include <functional>
#include <vector>

#include "cheb.cuh"

namespace tbk {

bool fused_eligible(const HOp& op, int s, int plain);

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    TBK_CUDA(cudaEventCreate(&a));
    TBK_CUDA(cudaEventCreate(&b));
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  float ms(tbk_ctx* ctx) {
    TBK_CUDA(cudaEventSynchronize(b));
    float t = 0.f;
    TBK_CUDA(cudaEventElapsedTime(&t, a, b));
    (void)ctx;
    return t;
  }
};

static void set_choice(tbk_ctx* ctx, const HOp& op, int s, int cw, int windowed) {
  for (auto& t : ctx->tuned)
    if (t.n_rows == op.n_rows && t.nnzb == op.nnzb && t.s == s) {
      t.cw = cw;
      t.windowed = windowed;
      return;
    }
  ctx->tuned.push_back({op.n_rows, op.nnzb, s, cw, windowed});
}

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_autotune(tbk_ctx* ctx, const tbk_bsr* H, double emin, double emax, int32_t n_probes,
                            int32_t* choice) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx && H && choice, "NULL argument");
  TBK_CHECK_ARG(H->n_orb == 9, "the tuned kernels take 9x9 blocks");
  TBK_CHECK_ARG(n_probes >= 128 && n_probes % 128 == 0, "n_probes must be a multiple of 128");
  DeviceGuard dg(ctx);
  const int s = n_probes;
  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  HOp op = prepare_hop(ctx, H, emin, emax, TBK_MIXED, WS_HHAT, err);
  const int cw_max = bulk_consumer_warps(op, s);
  TBK_CHECK_ARG(cw_max > 0, "no TMA-fed step for this operator");
  const size_t panel = (size_t)op.n_rows * s * 4;
  void* A = scratch(ctx, WS_PANEL0, panel);
  void* B = scratch(ctx, WS_PANEL1, panel);
  void* Cp = scratch(ctx, WS_PANEL2, panel);
  const uint64_t seed = 0x7E57;
  launch_scaled_probe(ctx, op, A, 1.0, seed, s);
  launch_scaled_probe(ctx, op, B, 0.5, seed + 1, s);

  // 1. probe chunk of the recurrence step: y_out = 2 H^ y_in - y_prev on two probe panels
  int best_cw = cw_max;
  float best = INFINITY;
  for (int cw = cw_max; cw >= 1; cw /= 2) {
    if (s % (128 * cw)) continue;
    set_choice(ctx, op, s, cw, 0);
    StepArgs a;
    a.seed = seed;
    a.s = s;
    a.yin = A;
    a.yprev = B;
    a.yout = Cp;
    a.alpha = 2.0;
    a.err = err;
    for (int w = 0; w < 2; ++w) launch_step(ctx, op, a);
    EventPair ev;
    constexpr int reps = 5;
    TBK_CUDA(cudaEventRecord(ev.a, ctx->stream));
    for (int r = 0; r < reps; ++r) launch_step(ctx, op, a);
    TBK_CUDA(cudaEventRecord(ev.b, ctx->stream));
    const float t = ev.ms(ctx) / reps;
    if (t < best) {
      best = t;
      best_cw = cw;
    }
  }
  set_choice(ctx, op, s, best_cw, 0);

  // 2. adjoint schedule (0 fused, 1 windowed, 2 tensor cores where that kernel applies), on a
  //    short sweep (K = 20 steps) with fixed coefficients
  int windowed = 0;
  if (fused_eligible(op, s, 0)) {
    const int p = 40;
    std::vector<double> c(p);
    for (int k = 0; k < p; ++k) c[k] = 1.0 / (1.0 + k);
    double* Gacc = (double*)scratch(ctx, WS_GACC, sizeof(double) * (size_t)op.nnzb * 81);
    const int n_sched = tc_sddmm_eligible(ctx, op, s, tc_sddmm_max_row(ctx, op)) ? 3 : 2;
    float t_sched[3] = {0.f, 0.f, 0.f};
    for (int w = 0; w < n_sched; ++w) {
      for (int rep = 0; rep < 2; ++rep) {  // the first run maps the panels and warms up
        TBK_CUDA(cudaMemsetAsync(Gacc, 0, sizeof(double) * (size_t)op.nnzb * 81, ctx->stream));
        EventPair ev;
        TBK_CUDA(cudaEventRecord(ev.a, ctx->stream));
        adjoint_doubling(ctx, op, seed, s, p, [&]() { return c; }, nullptr, 0, 0, Gacc, err, w, nullptr);
        TBK_CUDA(cudaEventRecord(ev.b, ctx->stream));
        t_sched[w] = ev.ms(ctx);
      }
    }
    for (int w = 1; w < n_sched; ++w)
      if (t_sched[w] < t_sched[windowed]) windowed = w;
  }
  int herr = 0;
  TBK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  check_diagonal_flag(herr);
  if (herr & 2) throw Error(TBK_ERR_TIMEOUT, "a bounded wait expired while tuning");
  set_choice(ctx, op, s, best_cw, windowed);
  choice[0] = 128 * best_cw;
  choice[1] = windowed;
  TBK_API_END
}
