// Persistent warp-specialised BF16 GEMM on tcgen05 (sm_103a):
//   C[z][m][n] (+)= alpha * sum_k A[z][m][k] * B[z][n][k]
// One CTA per SM loops over 128 x BN output tiles.  Warp 0 issues TMA loads
// into a kS-stage shared-memory ring, warp 1 issues tcgen05.mma into one of two
// TMEM accumulators, warps 2-5 drain the other accumulator (tcgen05.ld, the
// next 32 columns loaded while the current ones are written out), stage
// 32 x 32 sub-tiles in kEB swizzled shared-memory buffers per warp and write
// them with TMA bulk stores (or TMA reduce-adds when accumulating into C), so
// the epilogue of one tile overlaps the main loop of the next.  Two shapes:
// long K wants more bytes in flight (4 stages, 2 staging buffers), short K
// (few k-blocks per tile, many tiles) wants a deeper epilogue (3 and 4).
// In the last k-block only the MMAs that touch real K columns are issued;
// each CTA starts its K loop at a different block (the sum is order-free).
//
// Batch index z = zhi * nzlo + zlo.  Each operand's third TMA coordinate is
// chosen by a selector (none / zlo / zhi / z) plus an offset; the output map is
// 4D (column, zlo, row, zhi).  Out-of-range rows, columns and K read as zero
// and are clipped on store, so ragged shapes need no padding in memory.
#pragma once
#include "internal.cuh"
#include "tc_common.cuh"
#include "tc_gemm.cuh"

namespace ea {
namespace tc2 {
using namespace ea::tc;

enum ZSel : int { Z_NONE = 0, Z_LO = 1, Z_HI = 2, Z_ALL = 3 };

struct Args {
  int M, N, K, BN;     // BN: tile width <= 256, multiple of 32 (or of 16 when N <= BN)
  int nzlo, nz;        // batch: z in [0, nz), zlo = z % nzlo, zhi = z / nzlo
  int a_sel, b_sel, a_z0, b_z0;
  int a_row0, b_row0, a_k0, b_k0;
  int c_row0, c_col0;  // output coordinate offsets
  float alpha;
  int reduce;          // 1: C += result (TMA reduce-add), 0: C = result
  int out_bf16;        // output element type: 0 fp32, 1 bf16
  int* err;
  int variant;         // pipeline shape: 0 by K (see tc_gemm2), 1 <4 stages, 2 staging buffers>,
                       // 2 <3, 4>, 3 <4, 3>
};

constexpr int kBM = 128, kBK = 64, kEpiWarps = 4;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kStageA = kBM * kBK * 2;

__host__ __device__ constexpr size_t smem_bytes(int BN, int stages, int ebufs) {
  return 1024 + (size_t)stages * (kStageA + (size_t)BN * kBK * 2) + (size_t)kEpiWarps * ebufs * 4096 + 256;
}

__device__ __forceinline__ int zsel(int sel, int z0, int zlo, int zhi, int z) {
  return z0 + (sel == Z_LO ? zlo : sel == Z_HI ? zhi : sel == Z_ALL ? z : 0);
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
}

__device__ __forceinline__ void tma_reduce_add_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                                  int c3) {
  asm volatile("cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }

// Registers written by an asynchronous tcgen05.ld are valid only after
// tcgen05.wait::ld; this empty asm redefines them after the wait so that no
// use can be scheduled above it.
__device__ __forceinline__ void reg_fence(uint32_t (&r)[32]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) asm volatile("" : "+r"(r[i]));
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int kS, int kEB>  // pipeline stages, epilogue staging buffers per warp
__global__ void __launch_bounds__(kThreads, 1)
    gemm_persistent(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    const __grid_constant__ CUtensorMap mapC, Args g) {
  constexpr int kStages = kS;
  extern __shared__ uint8_t smem_raw[];
  const int BN = g.BN;
  const uint32_t stageB = (uint32_t)BN * kBK * 2;
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = sA + kStages * kStageA;
  uint8_t* sE = sB + kStages * stageB;  // epilogue staging: kEpiWarps x kEB x 4096 B (1024-aligned)
  uint64_t* full = (uint64_t*)(sE + kEpiWarps * kEB * 4096);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (g.M + kBM - 1) / kBM, tn = (g.N + BN - 1) / BN;
  const int ntiles = tm * tn * g.nz;
  const int nk = (g.K + kBK - 1) / kBK;
  // Each CTA walks K from its own starting block, so that CTAs sharing an
  // operand tile do not all request the same lines from L2 at the same time.
  const int krot = (int)(((long long)blockIdx.x * nk) / gridDim.x) % nk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], kEpiWarps); }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
    prefetch_tmap(&mapC);
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------ TMA producer
      int it = 0, issued = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        const int z = t / (tm * tn), rem = t % (tm * tn);
        const int mt = rem / tn, nt = rem % tn;
        const int zlo = z % g.nzlo, zhi = z / g.nzlo;
        const int az = zsel(g.a_sel, g.a_z0, zlo, zhi, z), bz = zsel(g.b_sel, g.b_z0, zlo, zhi, z);
        for (int ki = 0; ki < nk; ++ki, ++it) {
          const int kb = ki + krot < nk ? ki + krot : ki + krot - nk;
          const int s = it % kStages;
          const uint32_t ph = (it / kStages) & 1;
          if (it >= kStages && !mbar_wait(&empty[s], ph ^ 1, abort_flag, g.err, 201)) break;
          mbar_arrive_expect_tx(&full[s], kStageA + stageB);
          tma_load_3d(sA + s * kStageA, &mapA, &full[s], g.a_k0 + kb * kBK, g.a_row0 + mt * kBM, az);
          tma_load_3d(sB + s * stageB, &mapB, &full[s], g.b_k0 + kb * kBK, g.b_row0 + nt * BN, bz);
          ++issued;
        }
      }
      if (*abort_flag) {  // drain loads still in flight
        for (int i2 = issued > kStages ? issued - kStages : 0; i2 < issued; ++i2) {
          long long t0 = clock64();
          while (!mbar_try_wait(&full[i2 % kStages], (i2 / kStages) & 1) && clock64() - t0 < (1LL << 31)) {}
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------- MMA issuer
      const uint32_t idesc = idesc_bf16_f32(kBM, BN);
      int it = 0, tcount = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tcount) {
        const int buf = tcount & 1;
        const uint32_t aph = (tcount >> 1) & 1;
        if (tcount >= 2 && !mbar_wait(&acc_empty[buf], aph ^ 1, abort_flag, g.err, 202)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * 256);
        bool ok = true;
        for (int ki = 0; ki < nk; ++ki, ++it) {
          const int kb = ki + krot < nk ? ki + krot : ki + krot - nk;
          const int s = it % kStages;
          const uint32_t ph = (it / kStages) & 1;
          if (!mbar_wait(&full[s], ph, abort_flag, g.err, 203)) { ok = false; break; }
          tc_fence_after();
          const uint64_t ad = smem_desc_sw128(sA + s * kStageA);
          const uint64_t bd = smem_desc_sw128(sB + s * stageB);
          const int nmma = (min(kBK, g.K - kb * kBK) + 15) >> 4;  // past K the tile holds zeros
#pragma unroll
          for (int j = 0; j < kBK / 16; ++j)
            if (j < nmma) mma_bf16(dt, ad + 2 * j, bd + 2 * j, idesc, (ki | j) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        mma_commit(&acc_full[buf]);
        if (!ok) break;
      }
      // arrives once every MMA issued by this thread has completed
      mma_commit(mma_done);
    }
  } else {
    // --------------------------------------------------------- epilogue
    const int ew = warp - 2;          // 0..3
    const int q = warp & 3;           // TMEM lane quarter this warp may access
    uint8_t* stg = sE + ew * kEB * 4096;
    int tcount = 0, sbuf = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tcount) {
      const int buf = tcount & 1;
      const uint32_t aph = (tcount >> 1) & 1;
      if (!mbar_wait(&acc_full[buf], aph, abort_flag, g.err, 204)) break;
      if (*abort_flag) break;
      tc_fence_after();
      const int z = t / (tm * tn), rem = t % (tm * tn);
      const int mt = rem / tn, nt = rem % tn;
      const int zlo = z % g.nzlo, zhi = z / g.nzlo;
      const int row0 = g.c_row0 + mt * kBM + q * 32;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256);
      const bool rows_in = mt * kBM + q * 32 < g.M;
      // one 32 x 32 chunk: registers -> swizzled staging buffer -> TMA store
      auto drain = [&](uint32_t(&r)[32], int c0) {
        uint8_t* st = stg + sbuf * 4096;
        // the buffer may still be read by the bulk store issued kEB chunks ago
        if (lane == 0) bulk_wait_read<kEB - 1>();
        __syncwarp();
        if (!g.out_bf16) {
          // row = lane, 128-byte rows, 16-byte chunk j at (j ^ (row & 7)) (128-byte swizzle)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float4 v4 = make_float4(g.alpha * __uint_as_float(r[4 * j]), g.alpha * __uint_as_float(r[4 * j + 1]),
                                    g.alpha * __uint_as_float(r[4 * j + 2]), g.alpha * __uint_as_float(r[4 * j + 3]));
            *reinterpret_cast<float4*>(st + lane * 128 + ((j ^ (lane & 7)) << 4)) = v4;
          }
        } else {
          // row = lane, 64-byte rows, 16-byte chunk j at (j ^ ((row >> 1) & 3)) (64-byte swizzle)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 p0 = __floats2bfloat162_rn(g.alpha * __uint_as_float(r[8 * j]), g.alpha * __uint_as_float(r[8 * j + 1]));
            __nv_bfloat162 p1 = __floats2bfloat162_rn(g.alpha * __uint_as_float(r[8 * j + 2]), g.alpha * __uint_as_float(r[8 * j + 3]));
            __nv_bfloat162 p2 = __floats2bfloat162_rn(g.alpha * __uint_as_float(r[8 * j + 4]), g.alpha * __uint_as_float(r[8 * j + 5]));
            __nv_bfloat162 p3 = __floats2bfloat162_rn(g.alpha * __uint_as_float(r[8 * j + 6]), g.alpha * __uint_as_float(r[8 * j + 7]));
            uint4 u;
            u.x = *reinterpret_cast<uint32_t*>(&p0);
            u.y = *reinterpret_cast<uint32_t*>(&p1);
            u.z = *reinterpret_cast<uint32_t*>(&p2);
            u.w = *reinterpret_cast<uint32_t*>(&p3);
            *reinterpret_cast<uint4*>(st + lane * 64 + ((j ^ ((lane >> 1) & 3)) << 4)) = u;
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          const int col = g.c_col0 + nt * BN + c0;
          if (nt * BN + c0 < g.N && rows_in) {
            if (g.reduce) tma_reduce_add_4d(&mapC, st, col, zlo, row0, zhi);
            else tma_store_4d(&mapC, st, col, zlo, row0, zhi);
          }
          bulk_commit();
        }
        sbuf = sbuf + 1 == kEB ? 0 : sbuf + 1;
      };
      uint32_t ra[32], rb[32];
      tmem_ld_32x32b_x32(taddr, ra);
      for (int c0 = 0; c0 < BN; c0 += 64) {
        tmem_ld_wait();
        reg_fence(ra);
        if (c0 + 32 < BN) tmem_ld_32x32b_x32(taddr + (uint32_t)(c0 + 32), rb);
        drain(ra, c0);
        if (c0 + 32 < BN) {
          tmem_ld_wait();
          reg_fence(rb);
          if (c0 + 64 < BN) tmem_ld_32x32b_x32(taddr + (uint32_t)(c0 + 64), ra);
          drain(rb, c0 + 32);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  __syncthreads();
  if (warp == 0) {
    // all MMAs complete before TMEM is released (bounded)
    long long t0 = clock64();
    while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < (1LL << 31)) {}
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace tc2

// Host side (tc_gemm2.cu).
TmaMap make_tma_out4d(const void* base, int elem_bytes, long long cols, long long nzlo, long long rows, long long nzhi,
                      long long pitch_zlo, long long pitch_row, long long pitch_zhi);
void tc_gemm2(cudaStream_t s, const TmaMap& A, const TmaMap& B, const TmaMap& C, const tc2::Args& a);
// Tile width with the least padding of N: N rounded up to 16 when N <= 256
// (a single column tile), else a multiple of 32 in [128, 256].
int pick_bn(int N);

}  // namespace ea
