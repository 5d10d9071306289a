// Generic BF16 x BF16 -> FP32 "NT" GEMM on tcgen05 tensor cores:
//   C[z][m][n] = sum_k A[z][m][k] * B[z][n][k]      (both operands K-major)
// Operands come in through 3D TMA tensor maps (K, rows, batch) with 128-byte
// swizzle; out-of-range rows/columns read as zero, so ragged M, N and K need no
// padding in memory.  One 128 x BN output tile per CTA, 4-stage mbarrier
// pipeline: warp 0 lane 0 issues TMA, warp 1 lane 0 issues tcgen05.mma into a
// TMEM accumulator, all four warps drain TMEM (tcgen05.ld) in the epilogue.
#pragma once
#include "internal.cuh"
#include "tc_common.cuh"

namespace ea {
namespace tc {

enum EpiMode : int {
  EPI_F32 = 0,       // C32[z*czs + m*ldc + n] = alpha*acc + beta*C32
  EPI_LADDER_Z = 1,  // bf16 store of ladder stage 1 (see GemmArgs)
  EPI_F64_ADD = 2    // C64[z*czs + m*ldc + n] += alpha*acc
};

struct GemmArgs {
  int M, N, K;
  int a_row0, b_row0;  // row offsets into the maps
  int a_k0, b_k0;      // K offsets into the maps
  int a_batched, b_batched;
  int a_z0, b_z0;      // batch-coordinate offsets
  float alpha, beta;
  float* C32;
  double* C64;
  bf16* Cbf;
  long long ldc, czs;
  int v, qc;           // EPI_LADDER_Z: Z[((col/v)*v + row)*qc + z)*v + col%v]
  int* err;            // global error word (bounded waits)
};

constexpr int kBM = 128, kBK = 64, kStages = 4;

template <int BN>
constexpr size_t gemm_smem_bytes() {
  return 1024 + (size_t)kStages * (kBM * kBK + BN * kBK) * 2 + 256;
}

template <int BN, int MODE>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  constexpr uint32_t A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2;
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + kStages * A_BYTES;
  uint64_t* full = (uint64_t*)(sB + kStages * B_BYTES);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN, z = blockIdx.z;
  const int nk = (g.K + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
  }
  if (warp == 0) tmem_alloc(tmem_slot, BN < 32 ? 32 : BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int it = 0; it < nk; ++it) {
      const int s = it % kStages;
      const uint32_t ph = (it / kStages) & 1;
      if (it >= kStages && !mbar_wait(&empty[s], ph ^ 1, abort_flag, g.err, 101)) break;
      mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
      tma_load_3d(sA + s * A_BYTES, &mapA, &full[s], g.a_k0 + it * kBK, g.a_row0 + m0, g.a_batched ? g.a_z0 + z : g.a_z0);
      tma_load_3d(sB + s * B_BYTES, &mapB, &full[s], g.b_k0 + it * kBK, g.b_row0 + n0, g.b_batched ? g.b_z0 + z : g.b_z0);
      ++issued;
    }
    if (*abort_flag) {
      // drain loads still in flight before the CTA may exit
      for (int it = issued > kStages ? issued - kStages : 0; it < issued; ++it) {
        long long t0 = clock64();
        while (!mbar_try_wait(&full[it % kStages], (it / kStages) & 1) && clock64() - t0 < (1LL << 31)) {}
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16_f32(kBM, BN);
    for (int it = 0; it < nk; ++it) {
      const int s = it % kStages;
      const uint32_t ph = (it / kStages) & 1;
      if (!mbar_wait(&full[s], ph, abort_flag, g.err, 102)) break;
      tc_fence_after();
      const uint64_t ad = smem_desc_sw128(sA + s * A_BYTES);
      const uint64_t bd = smem_desc_sw128(sB + s * B_BYTES);
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j) mma_bf16(tmem, ad + 2 * j, bd + 2 * j, idesc, (it | j) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, abort_flag, g.err, 103) && !*abort_flag);
  tc_fence_after();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      tmem_ld_wait();
      if (row >= g.M) continue;
      const int colb = n0 + c0;
      if (MODE == EPI_F32) {
        float* C = g.C32 + (long long)z * g.czs + (long long)row * g.ldc;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = colb + j;
          if (col < g.N) {
            float val = g.alpha * __uint_as_float(r[j]);
            if (g.beta != 0.0f) val += g.beta * C[col];
            C[col] = val;
          }
        }
      } else if (MODE == EPI_F64_ADD) {
        double* C = g.C64 + (long long)z * g.czs + (long long)row * g.ldc;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = colb + j;
          if (col < g.N) C[col] += (double)g.alpha * (double)__uint_as_float(r[j]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = colb + j;
          if (col < g.N) {
            const int nkk = col / g.v, d = col - nkk * g.v;
            g.Cbf[(((long long)nkk * g.v + row) * g.qc + z) * g.v + d] = __float2bfloat16_rn(__uint_as_float(r[j]));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN < 32 ? 32 : BN);
}

}  // namespace tc

// Host side: tensor maps and launches (tc_gemm.cu).
struct TmaMap {
  CUtensorMap map;
};
// Map over a bf16 array viewed as [nb][rows][K] with the given pitches (elements).
TmaMap make_tma_3d(const bf16* base, long long K, long long rows, long long nb, long long row_pitch,
                   long long batch_pitch, int box_rows);
void tc_gemm(cudaStream_t s, const TmaMap& A, const TmaMap& B, const tc::GemmArgs& args, int batch, int mode,
             int bn);

}  // namespace ea
