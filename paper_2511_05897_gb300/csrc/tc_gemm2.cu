// Host side of the persistent tcgen05 GEMM: output tensor maps and launch.
#include "tc_gemm2.cuh"

namespace ea {
namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encoder2() {
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
int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    EA_CK(cudaGetDevice(&dev));
    EA_CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}
}  // namespace

TmaMap make_tma_out4d(const void* base, int elem_bytes, long long cols, long long nzlo, long long rows, long long nzhi,
                      long long pitch_zlo, long long pitch_row, long long pitch_zhi) {
  if (((uintptr_t)base & 15) || (pitch_zlo * elem_bytes) % 16 || (pitch_row * elem_bytes) % 16 ||
      (pitch_zhi * elem_bytes) % 16)
    fail(EAADC_ERR_ARG, "TMA output not 16-byte aligned");
  TmaMap m;
  cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)nzlo, (cuuint64_t)rows, (cuuint64_t)nzhi};
  cuuint64_t strides[3] = {(cuuint64_t)(pitch_zlo * elem_bytes), (cuuint64_t)(pitch_row * elem_bytes),
                           (cuuint64_t)(pitch_zhi * elem_bytes)};
  cuuint32_t box[4] = {32, 1, 32, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = encoder2()(&m.map, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          4, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          elem_bytes == 4 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(EAADC_ERR_CUDA, "cuTensorMapEncodeTiled (output) failed: " + std::to_string((int)r));
  return m;
}

int pick_bn(int N) {
  if (N <= 256) return std::max(32, (N + 15) / 16 * 16);
  int best = 256;
  long long bestw = -1;
  for (int bn = 256; bn >= 128; bn -= 32) {
    long long w = (long long)((N + bn - 1) / bn) * bn;
    if (bestw < 0 || w < bestw) { bestw = w; best = bn; }
  }
  return best;
}

namespace {
template <int kS, int kEB>
void launch_variant(cudaStream_t s, const TmaMap& A, const TmaMap& B, const TmaMap& C, const tc2::Args& a, int grid) {
  constexpr size_t kMaxSmem = 232448;  // per-block opt-in limit
  if (tc2::smem_bytes(a.BN, kS, kEB) > kMaxSmem)
    fail(EAADC_ERR_ARG, "tc_gemm2: pipeline variant does not fit shared memory at this tile width");
  static bool attr = false;  // opt in to the largest shared-memory size once per variant
  if (!attr) {
    EA_CK(cudaFuncSetAttribute(tc2::gemm_persistent<kS, kEB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)std::min(tc2::smem_bytes(256, kS, kEB), kMaxSmem)));
    attr = true;
  }
  tc2::gemm_persistent<kS, kEB><<<grid, tc2::kThreads, tc2::smem_bytes(a.BN, kS, kEB), s>>>(A.map, B.map, C.map, a);
  EA_LAUNCH();
}
}  // namespace

void tc_gemm2(cudaStream_t s, const TmaMap& A, const TmaMap& B, const TmaMap& C, const tc2::Args& a) {
  if (a.M <= 0 || a.N <= 0 || a.nz <= 0) return;
  // BN: an MMA width (multiple of 16, <= 256); the epilogue writes 32-column
  // chunks, so a width that is not a multiple of 32 needs a single column tile
  // whose last chunk runs past N (clipped by the output map).
  if (a.BN < 32 || a.BN > 256 || a.BN % 16 || (a.BN % 32 && (a.N > a.BN || a.c_col0)))
    fail(EAADC_ERR_ARG, "tc_gemm2: bad tile width");
  if (a.nzlo < 1 || a.nz % a.nzlo) fail(EAADC_ERR_ARG, "tc_gemm2: bad batch split");
  const long long tiles = (long long)((a.M + tc2::kBM - 1) / tc2::kBM) * ((a.N + a.BN - 1) / a.BN) * a.nz;
  if (tiles > (1LL << 31) - 1) fail(EAADC_ERR_ARG, "tc_gemm2: too many tiles");
  const int grid = (int)std::min<long long>(tiles, sm_count());
  const int nk = (a.K + tc2::kBK - 1) / tc2::kBK;
  const int var = a.variant ? a.variant : (nk >= 8 ? 1 : 2);
  if (var == 1) launch_variant<4, 2>(s, A, B, C, a, grid);       // long K: bytes in flight
  else if (var == 2) launch_variant<3, 4>(s, A, B, C, a, grid);  // short K: epilogue depth
  else if (var == 3) launch_variant<4, 3>(s, A, B, C, a, grid);
  else fail(EAADC_ERR_ARG, "tc_gemm2: unknown variant");
}

}  // namespace ea
