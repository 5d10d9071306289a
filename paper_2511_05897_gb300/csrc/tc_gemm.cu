// TMA operand tensor maps (the driver entry point is obtained through the
// runtime, so the library does not link libcuda).
#include "tc_gemm.cuh"

namespace ea {
namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    EA_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) fail(EAADC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = (EncodeFn)p;
  }
  return fn;
}

}  // namespace

TmaMap make_tma_3d(const bf16* base, long long K, long long rows, long long nb, long long row_pitch,
                   long long batch_pitch, int box_rows) {
  if (((uintptr_t)base & 15) || (row_pitch * 2) % 16 || (batch_pitch * 2) % 16)
    fail(EAADC_ERR_ARG, "TMA operand not 16-byte aligned");
  if (box_rows < 1 || box_rows > 256) fail(EAADC_ERR_ARG, "TMA box rows out of range");
  TmaMap m;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)nb};
  cuuint64_t strides[2] = {(cuuint64_t)row_pitch * 2, (cuuint64_t)(batch_pitch > 0 ? batch_pitch : row_pitch * rows) * 2};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = encoder()(&m.map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(EAADC_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

}  // namespace ea
