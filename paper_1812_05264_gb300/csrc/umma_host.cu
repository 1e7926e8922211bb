// Host side of the tensor-core building blocks: tensor maps for TMA loads, through the driver's
// cuTensorMapEncodeTiled reached with cudaGetDriverEntryPointByVersion (no link against libcuda).
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "umma.cuh"

namespace tbk {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* p = nullptr;
    err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (err == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  if (!fn) throw Error(TBK_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

void make_tmap_2d(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                  int box_cols, bool swizzle128) {
  TBK_CHECK_ARG(((uintptr_t)base & 15) == 0 && (ld * 4) % 16 == 0, "tensor map base or stride not 16-byte aligned");
  TBK_CHECK_ARG(!swizzle128 || box_cols * 4 == 128, "a 128-byte swizzle needs 128-byte box rows");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(TBK_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

}  // namespace tbk
