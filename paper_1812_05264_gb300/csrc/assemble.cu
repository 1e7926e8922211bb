// a2: assemble the block-sparse Hamiltonian on the device (Sec. II.A: the NRL copper model is
// built from Slater-Koster two-centre blocks; Sec. IV: simple-cubic lattice test models).
#include <cmath>

#include "common.cuh"
#include "model.cuh"
#include "sk.cuh"

namespace tbk {

__device__ __forceinline__ double min_image(double d, double L) {
  return L > 0.0 ? d - L * rint(d / L) : d;
}

__global__ void assemble_kernel(DevModel M, const double* __restrict__ pos, int n_atoms,
                                const int32_t* __restrict__ row_ptr,
                                const int32_t* __restrict__ col, double* __restrict__ H,
                                int* __restrict__ err) {
  const int a = blockIdx.x * blockDim.y + threadIdx.y;  // block row per y-thread group
  if (a >= n_atoms) return;
  const int b_ = M.n_orb, bb = b_ * b_;
  for (int k = row_ptr[a] + threadIdx.x; k < row_ptr[a + 1]; k += blockDim.x) {
    const int b = col[k];
    double* out = H + (int64_t)k * bb;
    if (b == a) {
      for (int i = 0; i < bb; ++i) out[i] = 0.0;
      if (M.kind == TBK_MODEL_SK) {
        out[0] = M.onsite[0];
        for (int i = 1; i < 4; ++i) out[i * 9 + i] = M.onsite[1];
        for (int i = 4; i < 9; ++i) out[i * 9 + i] = M.onsite[2];
      }
      if (M.onsite_site)
        for (int i = 0; i < b_; ++i) out[i * b_ + i] += M.onsite_site[(int64_t)a * b_ + i];
      continue;
    }
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = min_image(pos[3 * b + c] - pos[3 * a + c], M.box[c]);
    if (M.kind == TBK_MODEL_SK) {
      double E[81];
      sk_block<double>(d, M.V, M.r0, M.decay, E);
      for (int i = 0; i < 81; ++i) out[i] = E[i];
    } else {
      int hit = -1;
      for (int t = 0; t < M.n_disp; ++t) {
        const double* q = M.disp + 3 * t;
        if (fabs(d[0] - q[0]) <= M.tol && fabs(d[1] - q[1]) <= M.tol && fabs(d[2] - q[2]) <= M.tol) {
          hit = t;
          break;
        }
      }
      if (hit < 0) {
        atomicExch(err, 1);
        for (int i = 0; i < bb; ++i) out[i] = 0.0;
      } else {
        for (int i = 0; i < bb; ++i) out[i] = M.blocks[(int64_t)hit * bb + i];
      }
    }
  }
}

DevModel upload_model(tbk_ctx* ctx, const tbk_model* model, const double* box, Slot slot) {
  TBK_CHECK_ARG(model != nullptr, "model is NULL");
  DevModel M{};
  M.kind = model->kind;
  M.n_orb = model->n_orb;
  TBK_CHECK_ARG(M.kind == TBK_MODEL_SK || M.kind == TBK_MODEL_TABLE, "unknown model kind");
  TBK_CHECK_ARG(M.n_orb == 1 || M.n_orb == 9, "n_orb must be 1 or 9");
  TBK_CHECK_ARG(M.kind != TBK_MODEL_SK || M.n_orb == 9, "the Slater-Koster model has 9 orbitals");
  for (int i = 0; i < 10; ++i) M.V[i] = model->sk_V[i];
  M.r0 = model->sk_r0;
  M.decay = model->sk_decay;
  for (int i = 0; i < 3; ++i) M.onsite[i] = model->onsite_spd[i];
  if (M.kind == TBK_MODEL_SK) TBK_CHECK_ARG(M.r0 > 0.0, "sk_r0 must be positive");
  for (int c = 0; c < 3; ++c) M.box[c] = box ? box[c] : 0.0;
  M.onsite_site = model->onsite_site;
  M.n_disp = 0;
  if (M.kind == TBK_MODEL_TABLE) {
    TBK_CHECK_ARG(model->n_disp >= 0 && (model->n_disp == 0 || (model->disp && model->disp_blocks)),
                  "table model needs disp and disp_blocks");
    M.n_disp = model->n_disp;
    M.tol = model->disp_tol > 0.0 ? model->disp_tol : 1e-6;
    const size_t bb = (size_t)M.n_orb * M.n_orb;
    const size_t bytes = sizeof(double) * (3 * (size_t)M.n_disp + bb * M.n_disp) + 16;
    double* dev = (double*)scratch(ctx, slot, bytes);
    TBK_CUDA(cudaMemcpyAsync(dev, model->disp, sizeof(double) * 3 * M.n_disp, cudaMemcpyHostToDevice, ctx->stream));
    TBK_CUDA(cudaMemcpyAsync(dev + 3 * M.n_disp, model->disp_blocks, sizeof(double) * bb * M.n_disp,
                             cudaMemcpyHostToDevice, ctx->stream));
    M.disp = dev;
    M.blocks = dev + 3 * M.n_disp;
  }
  return M;
}

}  // namespace tbk

using namespace tbk;

extern "C" int tbk_assemble_H(tbk_ctx* ctx, const tbk_model* model, const double* pos,
                              int32_t n_atoms, const double* box, const int32_t* row_ptr,
                              const int32_t* col, int64_t nnzb, double* H) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(ctx != nullptr, "ctx is NULL");
  TBK_CHECK_ARG(n_atoms >= 0 && nnzb >= 0, "negative size");
  TBK_CHECK_ARG(n_atoms == 0 || (pos && row_ptr && col && H), "NULL array");
  DeviceGuard dg(ctx);
  DevModel M = upload_model(ctx, model, box, WS_TABLE);
  if (n_atoms == 0) return TBK_OK;
  int* err = (int*)scratch(ctx, WS_FLAGS, 64);
  TBK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  dim3 blk(8, 16);
  assemble_kernel<<<ceil_div(n_atoms, 16), blk, 0, ctx->stream>>>(M, pos, n_atoms, row_ptr, col, H, err);
  post_launch(ctx, "assemble_kernel");
  int herr = 0;
  TBK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  TBK_CHECK_ARG(herr == 0, "a neighbour displacement matches no table entry");
  TBK_API_END
}
