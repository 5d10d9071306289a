// FP64 building blocks (and their FP32 forms): batched GEMM, tensor permutation, pair combinations,
// a two-operand contraction engine and a one-CTA Jacobi eigensolver.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>

namespace ea {

[[noreturn]] void fail(eaadc_status st, const std::string& msg) { throw Error{st, msg}; }

long long g_kernel_launches = 0;

// ------------------------------------------------------------------- DGEMM
namespace {
constexpr int BM = 64, BN = 64, BK = 16;

// blockIdx.z = zb * ksplit + zs: batch entry zb, K slice zs of length kchunk.
// With ksplit > 1 each slice writes alpha * (its partial product) to its own
// [M][N] panel of C (panels ksplit*nbatch apart is the caller's layout).
template <class T, bool TA, bool TB, bool BETA0>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, T alpha,
                                                    const T* __restrict__ A, long long lda,
                                                    const T* __restrict__ B, long long ldb,
                                                    T beta, T* __restrict__ C, long long ldc,
                                                    GemmBatch bt, int ksplit, int kchunk, long long spanel) {
  const int zs = blockIdx.z % ksplit;
  const int z = blockIdx.z / ksplit;
  const int z1 = z / bt.nb2, z2 = z % bt.nb2;
  A += z1 * bt.sA1 + z2 * bt.sA2;
  B += z1 * bt.sB1 + z2 * bt.sB2;
  C += z1 * bt.sC1 + z2 * bt.sC2 + (long long)zs * spanel;
  const int kbeg = zs * kchunk;
  const int kend = min(K, kbeg + kchunk);
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int i = tid + 256 * r;
      int mm, kk;
      if (TA) { mm = i % BM; kk = i / BM; } else { kk = i % BK; mm = i / BK; }
      int gm = m0 + mm, gk = k0 + kk;
      T a = T(0);
      if (gm < M && gk < kend) a = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = a;
      int nn;
      if (TB) { kk = i % BK; nn = i / BK; } else { nn = i % BN; kk = i / BN; }
      int gn = n0 + nn;
      gk = k0 + kk;
      T b = T(0);
      if (gn < N && gk < kend) b = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[kk][nn] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      T* c = C + (long long)gm * ldc + gn;
      *c = BETA0 ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
    }
  }
}

// FP32 GEMM on CUDA cores: 128 x 128 output tile per CTA, K in steps of 8,
// 256 threads each holding an 8 x 8 block of C (rows ty*4+{0..3} and
// 64+ty*4+{0..3}, columns likewise from tx), the next K step fetched into
// registers while the current one is consumed from shared memory (two
// buffers, one barrier per step).  Same batching and K-split contract as
// dgemm_kernel.
constexpr int SBM = 128, SBN = 128, SBK = 8, SLD = SBM + 4;

template <bool TA, bool TB, bool BETA0>
__global__ void __launch_bounds__(256, 2) sgemm_kernel(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                       long long lda, const float* __restrict__ B, long long ldb,
                                                       float beta, float* __restrict__ C, long long ldc, GemmBatch bt,
                                                       int ksplit, int kchunk, long long spanel) {
  const int zs = blockIdx.z % ksplit;
  const int z = blockIdx.z / ksplit;
  const int z1 = z / bt.nb2, z2 = z % bt.nb2;
  A += z1 * bt.sA1 + z2 * bt.sA2;
  B += z1 * bt.sB1 + z2 * bt.sB2;
  C += z1 * bt.sC1 + z2 * bt.sC2 + (long long)zs * spanel;
  const int kbeg = zs * kchunk;
  const int kend = min(K, kbeg + kchunk);
  __shared__ __align__(16) float As[2][SBK][SLD];
  __shared__ __align__(16) float Bs[2][SBK][SLD];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * SBM, n0 = blockIdx.x * SBN;
  float ra[4], rb[4];
  // element r of this thread's share of a 128 x 8 tile: (row, k) coordinates
  auto a_rc = [&](int r, int& mm, int& kk) {
    const int e = tid + 256 * r;
    if (TA) { mm = e % SBM; kk = e / SBM; } else { kk = e % SBK; mm = e / SBK; }
  };
  auto b_rc = [&](int r, int& nn, int& kk) {
    const int e = tid + 256 * r;
    if (TB) { kk = e % SBK; nn = e / SBK; } else { nn = e % SBN; kk = e / SBN; }
  };
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int mm, kk;
      a_rc(r, mm, kk);
      const int gm = m0 + mm, gk = k0 + kk;
      ra[r] = (gm < M && gk < kend) ? (TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk]) : 0.f;
      int nn;
      b_rc(r, nn, kk);
      const int gn = n0 + nn, gk2 = k0 + kk;
      rb[r] = (gn < N && gk2 < kend) ? (TB ? B[(long long)gn * ldb + gk2] : B[(long long)gk2 * ldb + gn]) : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int mm, kk;
      a_rc(r, mm, kk);
      As[buf][kk][mm] = ra[r];
      int nn;
      b_rc(r, nn, kk);
      Bs[buf][kk][nn] = rb[r];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  int buf = 0;
  if (kbeg < kend) {
    fetch(kbeg);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += SBK) {
    const bool more = k0 + SBK < kend;
    if (more) fetch(k0 + SBK);
#pragma unroll
    for (int kk = 0; kk < SBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (gn >= N) continue;
      float* c = C + (long long)gm * ldc + gn;
      *c = BETA0 ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
    }
  }
}

template <class T>
__global__ void splitk_reduce(const T* __restrict__ P, int ksplit, long long panel, int M, int N,
                              T beta, T* __restrict__ C, long long ldc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < panel; e += (long long)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int z = 0; z < ksplit; ++z) acc += P[(long long)z * panel + e];
    const long long m = e / N, n = e % N;
    T* c = C + m * ldc + n;
    *c = (beta == T(0)) ? acc : acc + beta * (*c);
  }
}

template <bool TA, bool TB>
void sgemm_t(cudaStream_t s, int M, int N, int K, float alpha, const float* A, long long lda, const float* B,
             long long ldb, float beta, float* C, long long ldc, const GemmBatch& bt) {
  const int nbatch = bt.nb1 * bt.nb2;
  const long long tiles = (long long)((N + SBN - 1) / SBN) * ((M + SBM - 1) / SBM) * nbatch;
  // split K when the output grid cannot fill the GPU twice and K is long
  int ksplit = 1;
  if (nbatch == 1 && tiles < 304 && K >= 512) {
    ksplit = (int)std::min<long long>(std::min<long long>((608 + tiles - 1) / tiles, K / 128), 64);
    if (ksplit < 2) ksplit = 1;
  }
  if (ksplit == 1) {
    dim3 grid((N + SBN - 1) / SBN, (M + SBM - 1) / SBM, nbatch);
    if (beta == 0.f)
      sgemm_kernel<TA, TB, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, 1, K, 0);
    else
      sgemm_kernel<TA, TB, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, 1, K, 0);
    EA_LAUNCH();
    return;
  }
  const int kchunk = ((K + ksplit - 1) / ksplit + SBK - 1) / SBK * SBK;
  ksplit = (K + kchunk - 1) / kchunk;
  const long long panel = (long long)M * N;
  DArr<float> P((size_t)(panel * ksplit), s);
  dim3 grid((N + SBN - 1) / SBN, (M + SBM - 1) / SBM, ksplit);
  sgemm_kernel<TA, TB, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, 0.f, P.p, N, bt, ksplit, kchunk,
                                                  panel);
  EA_LAUNCH();
  splitk_reduce<<<(int)std::min<long long>((panel + 255) / 256, 4096), 256, 0, s>>>(P.p, ksplit, panel, M, N, beta,
                                                                                   C, ldc);
  EA_LAUNCH();
}

// Skinny products (N <= 8 columns), bandwidth-bound: every element of A is
// read once.  TA = false (A row-major M x K): one warp per row of C, lanes
// stride over K.  TA = true (A stored K x M): one thread per column of A
// (coalesced over m), K split over blockIdx.y into partial panels.
template <class T, bool TB>
__global__ void skinny_rows(int M, int N, int K, T alpha, const T* __restrict__ A, long long lda,
                            const T* __restrict__ B, long long ldb, T beta, T* __restrict__ C, long long ldc) {
  extern __shared__ unsigned char skinny_smem[];
  T* Bs = reinterpret_cast<T*>(skinny_smem);  // [K][8], zero beyond N
  for (int e = threadIdx.x; e < K * 8; e += blockDim.x) {
    const int k = e >> 3, n = e & 7;
    Bs[e] = n < N ? (TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long wpb = blockDim.x >> 5;
  for (long long m = blockIdx.x * wpb + (threadIdx.x >> 5); m < M; m += (long long)gridDim.x * wpb) {
    T acc[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) acc[n] = T(0);
    const T* a = A + m * lda;
#pragma unroll 4
    for (int k = lane; k < K; k += 32) {
      const T x = a[k];
      const T* bk = Bs + k * 8;
#pragma unroll
      for (int n = 0; n < 8; ++n) acc[n] += x * bk[n];
    }
#pragma unroll
    for (int n = 0; n < 8; ++n)
      for (int o = 16; o; o >>= 1) acc[n] += __shfl_xor_sync(0xffffffffu, acc[n], o);
    if (lane == 0)
      for (int n = 0; n < N; ++n) {
        T* c = C + m * ldc + n;
        *c = beta == T(0) ? alpha * acc[n] : alpha * acc[n] + beta * *c;
      }
  }
}

template <class T, bool TB>
__global__ void skinny_cols(int M, int N, int K, const T* __restrict__ A, long long lda, const T* __restrict__ B,
                            long long ldb, int kchunk, T* __restrict__ P) {
  extern __shared__ unsigned char skinny_smem[];
  T* Bs = reinterpret_cast<T*>(skinny_smem);  // [kchunk][8], zero beyond N
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  for (int e = threadIdx.x; e < (k1 - k0) * 8; e += blockDim.x) {
    const int k = k0 + (e >> 3), n = e & 7;
    Bs[e] = n < N ? (TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : T(0);
  }
  __syncthreads();
  if (m >= M) return;
  T acc[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) acc[n] = T(0);
#pragma unroll 8
  for (int k = k0; k < k1; ++k) {
    const T x = A[(long long)k * lda + m];
    const T* bk = Bs + (k - k0) * 8;
#pragma unroll
    for (int n = 0; n < 8; ++n) acc[n] += x * bk[n];
  }
  T* out = P + (long long)blockIdx.y * M * N + (long long)m * N;
  for (int n = 0; n < N; ++n) out[n] = acc[n];
}

template <class T, bool TA, bool TB>
void skinny_t(cudaStream_t s, int M, int N, int K, T alpha, const T* A, long long lda, const T* B, long long ldb,
              T beta, T* C, long long ldc) {
  if (!TA) {
    const int grid = (int)std::min<long long>(((long long)M + 7) / 8, 152LL * 16);
    skinny_rows<T, TB><<<grid, 256, (size_t)K * 8 * sizeof(T), s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    EA_LAUNCH();
    return;
  }
  const int bx = (M + 255) / 256;
  int ks = (int)std::max<long long>(1, std::min<long long>((608 + bx - 1) / bx, (K + 255) / 256));
  ks = std::max(ks, (K + 511) / 512);  // staged B slice <= 512 x 8 elements (32 KB in FP64)
  const int kchunk = (K + ks - 1) / ks;
  ks = (K + kchunk - 1) / kchunk;
  const long long panel = (long long)M * N;
  DArr<T> P((size_t)(panel * ks), s);
  skinny_cols<T, TB><<<dim3(bx, ks), 256, (size_t)kchunk * 8 * sizeof(T), s>>>(M, N, K, A, lda, B, ldb, kchunk,
                                                                                  P.p);
  EA_LAUNCH();
  // C = alpha * sum of panels + beta * C (splitk_reduce adds beta * C)
  if (alpha != T(1)) fail(EAADC_ERR_ARG, "skinny gemm: alpha != 1 with a transposed A");
  splitk_reduce<<<(int)std::min<long long>((panel + 255) / 256, 4096), 256, 0, s>>>(P.p, ks, panel, M, N, beta, C, ldc);
  EA_LAUNCH();
}

template <class T, bool TA, bool TB>
void dgemm_t(cudaStream_t s, int M, int N, int K, T alpha, const T* A, long long lda,
             const T* B, long long ldb, T beta, T* C, long long ldc, const GemmBatch& bt) {
  if (bt.nb1 * bt.nb2 == 1 && N <= 8 && K >= 64 && (TA ? alpha == T(1) : (long long)K * 8 * sizeof(T) <= 48 * 1024)) {
    skinny_t<T, TA, TB>(s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    return;
  }
  if constexpr (std::is_same<T, float>::value) {
    sgemm_t<TA, TB>(s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt);
    return;
  }
  const int nbatch = bt.nb1 * bt.nb2;
  const long long tiles = (long long)((N + BN - 1) / BN) * ((M + BM - 1) / BM) * nbatch;
  // split K when the output grid cannot fill the GPU and K is long
  int ksplit = 1;
  if (nbatch == 1 && tiles < 152 && K >= 1024) {
    ksplit = (int)std::min<long long>(std::min<long long>((304 + tiles - 1) / tiles, K / 256), 64);
    if (ksplit < 2) ksplit = 1;
  }
  if (ksplit == 1) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, nbatch);
    if (beta == T(0))
      dgemm_kernel<T, TA, TB, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, 1, K, 0);
    else
      dgemm_kernel<T, TA, TB, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, 1, K, 0);
    EA_LAUNCH();
    return;
  }
  const int kchunk = ((K + ksplit - 1) / ksplit + BK - 1) / BK * BK;
  ksplit = (K + kchunk - 1) / kchunk;
  const long long panel = (long long)M * N;
  DArr<T> P((size_t)(panel * ksplit), s);
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, ksplit);
  dgemm_kernel<T, TA, TB, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, T(0), P.p, N, bt, ksplit, kchunk,
                                                     panel);
  EA_LAUNCH();
  splitk_reduce<<<(int)std::min<long long>((panel + 255) / 256, 4096), 256, 0, s>>>(P.p, ksplit, panel, M, N, beta,
                                                                                   C, ldc);
  EA_LAUNCH();
}
}  // namespace

template <class T>
void gemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, long long lda, const T* B,
          long long ldb, T beta, T* C, long long ldc, const GemmBatch& bt) {
  if (M <= 0 || N <= 0 || bt.nb1 * bt.nb2 <= 0) return;
  if (bt.nb1 * bt.nb2 > 65535) fail(EAADC_ERR_ARG, "dgemm: batch too large");
  if ((M + BM - 1) / BM > 65535) fail(EAADC_ERR_ARG, "dgemm: M too large");
  if (ta && tb) dgemm_t<T, true, true>(s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt);
  else if (ta) dgemm_t<T, true, false>(s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt);
  else if (tb) dgemm_t<T, false, true>(s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt);
  else dgemm_t<T, false, false>(s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt);
}
template void gemm<double>(cudaStream_t, bool, bool, int, int, int, double, const double*, long long, const double*,
                           long long, double, double*, long long, const GemmBatch&);
template void gemm<float>(cudaStream_t, bool, bool, int, int, int, float, const float*, long long, const float*,
                          long long, float, float*, long long, const GemmBatch&);

// ----------------------------------------------------------------- permute
namespace {
struct PermArgs {
  int nd;
  long long ddim[8];
  long long sstride[8];  // stride in src of dst axis i
};

template <class T>
__global__ void permute_kernel(const T* __restrict__ src, T* __restrict__ dst, long long total,
                               PermArgs pa, T alpha, T beta) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx, off = 0;
    for (int i = pa.nd - 1; i >= 0; --i) {
      long long c = r % pa.ddim[i];
      r /= pa.ddim[i];
      off += c * pa.sstride[i];
    }
    T val = alpha * src[off];
    dst[idx] = (beta == T(0)) ? val : val + beta * dst[idx];
  }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }
}  // namespace

template <class T>
void permuteT(cudaStream_t s, const T* src, const std::vector<int>& sdims, const std::vector<int>& perm, T* dst,
              T alpha, T beta) {
  int nd = (int)sdims.size();
  if (nd > 8 || (int)perm.size() != nd) fail(EAADC_ERR_ARG, "permute: bad rank");
  long long st[8];
  long long acc = 1;
  for (int i = nd - 1; i >= 0; --i) { st[i] = acc; acc *= sdims[i]; }
  PermArgs pa;
  pa.nd = nd;
  for (int i = 0; i < nd; ++i) { pa.ddim[i] = sdims[perm[i]]; pa.sstride[i] = st[perm[i]]; }
  if (acc == 0) return;
  permute_kernel<T><<<grid_for(acc), 256, 0, s>>>(src, dst, acc, pa, alpha, beta);
  EA_LAUNCH();
}
template void permuteT<double>(cudaStream_t, const double*, const std::vector<int>&, const std::vector<int>&,
                               double*, double, double);
template void permuteT<float>(cudaStream_t, const float*, const std::vector<int>&, const std::vector<int>&, float*,
                              float, float);

// ------------------------------------------------------------ pair combine
namespace {
template <class T>
__global__ void pair_combine_kernel(const T* __restrict__ in, long long in_stride, T* __restrict__ out,
                                    long long out_stride, int nmat, int v, T c1, T c2, T alpha, T beta) {
  // 32x32 tiles of one matrix; transposed partner read through shared memory
  __shared__ T tileT[32][33];
  const int m = blockIdx.z;
  const int b0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const T* I = in + (long long)m * in_stride;
  T* O = out + (long long)m * out_stride;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  // load in[c0+.., b0+..] so that tileT[tx][ty] holds in[c][b] with c = c0+ty, b = b0+tx
  for (int r = ty; r < 32; r += 8) {
    int c = c0 + r, b = b0 + tx;
    tileT[tx][r] = (c < v && b < v) ? I[(long long)c * v + b] : T(0);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int b = b0 + r, c = c0 + tx;
    if (b < v && c < v) {
      T val = alpha * (c1 * I[(long long)b * v + c] + c2 * tileT[r][tx]);
      T* o = O + (long long)b * v + c;
      *o = (beta == T(0)) ? val : val + beta * (*o);
    }
  }
}

template <class T>
__global__ void fill_kernel(T* p, long long n, T val) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = val;
}
template <class T>
__global__ void axpby_kernel(long long n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
}  // namespace

template <class T>
void pair_combineT(cudaStream_t s, const T* in, long long in_stride, T* out, long long out_stride, int nmat, int v,
                   T c1, T c2, T alpha, T beta) {
  if (nmat <= 0 || v <= 0) return;
  if (nmat > 65535) fail(EAADC_ERR_ARG, "pair_combine: too many matrices");
  dim3 grid((v + 31) / 32, (v + 31) / 32, nmat);
  pair_combine_kernel<T><<<grid, dim3(32, 8), 0, s>>>(in, in_stride, out, out_stride, nmat, v, c1, c2, alpha, beta);
  EA_LAUNCH();
}
template void pair_combineT<double>(cudaStream_t, const double*, long long, double*, long long, int, int, double,
                                    double, double, double);
template void pair_combineT<float>(cudaStream_t, const float*, long long, float*, long long, int, int, float, float,
                                   float, float);

template <class T>
void fillT(cudaStream_t s, T* p, size_t n, T val) {
  if (!n) return;
  fill_kernel<T><<<grid_for((long long)n), 256, 0, s>>>(p, (long long)n, val);
  EA_LAUNCH();
}
template <class T>
void axpbyT(cudaStream_t s, size_t n, T a, const T* x, T b, T* y) {
  if (!n) return;
  axpby_kernel<T><<<grid_for((long long)n), 256, 0, s>>>((long long)n, a, x, b, y);
  EA_LAUNCH();
}
template void fillT<double>(cudaStream_t, double*, size_t, double);
template void fillT<float>(cudaStream_t, float*, size_t, float);
template void axpbyT<double>(cudaStream_t, size_t, double, const double*, double, double*);
template void axpbyT<float>(cudaStream_t, size_t, float, const float*, float, float*);

// ------------------------------------------------------------------ einsum
template <class T>
void einsumT(cudaStream_t s, const char* spec, T alpha, const TensT<T>& A, const TensT<T>& B, T beta,
             const TensT<T>& C) {
  std::string sp(spec);
  size_t comma = sp.find(','), arrow = sp.find("->");
  if (comma == std::string::npos || arrow == std::string::npos) fail(EAADC_ERR_ARG, "einsum: bad spec");
  std::string la = sp.substr(0, comma), lb = sp.substr(comma + 1, arrow - comma - 1), lc = sp.substr(arrow + 2);
  if (la.size() != A.dims.size() || lb.size() != B.dims.size() || lc.size() != C.dims.size())
    fail(EAADC_ERR_ARG, std::string("einsum: rank mismatch in ") + spec);
  std::map<char, int> dim;
  auto reg = [&](const std::string& l, const std::vector<int>& d) {
    for (size_t i = 0; i < l.size(); ++i) {
      auto it = dim.find(l[i]);
      if (it != dim.end() && it->second != d[i]) fail(EAADC_ERR_ARG, std::string("einsum: dim mismatch in ") + spec);
      dim[l[i]] = d[i];
    }
  };
  reg(la, A.dims); reg(lb, B.dims); reg(lc, C.dims);
  std::string fa, fb, kc;
  for (char c : la) {
    bool inb = lb.find(c) != std::string::npos, inc = lc.find(c) != std::string::npos;
    if (inb && inc) fail(EAADC_ERR_ARG, std::string("einsum: batch label unsupported in ") + spec);
    if (!inb && !inc) fail(EAADC_ERR_ARG, std::string("einsum: summed-out label unsupported in ") + spec);
    if (inc) fa += c; else kc += c;
  }
  for (char c : lb) {
    bool ina = la.find(c) != std::string::npos, inc = lc.find(c) != std::string::npos;
    if (!ina && !inc) fail(EAADC_ERR_ARG, std::string("einsum: summed-out label unsupported in ") + spec);
    if (inc) fb += c;
  }
  auto prod = [&](const std::string& l) { long long p = 1; for (char c : l) p *= dim[c]; return p; };
  long long M = prod(fa), N = prod(fb), K = prod(kc);
  auto perm_of = [&](const std::string& from, const std::string& to) {
    std::vector<int> p;
    for (char c : to) p.push_back((int)from.find(c));
    return p;
  };
  auto is_id = [](const std::vector<int>& p) { for (size_t i = 0; i < p.size(); ++i) if (p[i] != (int)i) return false; return true; };
  // Operand A is used as stored when its labels read [fa kc] (plain) or
  // [kc fa] (transposed); B likewise with [fb kc] or [kc fb].  Otherwise it is
  // permuted to [free..., contracted...].
  DArr<T> ta, tb, tc;
  const T* pa = A.p;
  bool transA = false;
  long long ldA = K;
  if (la == fa + kc) {
  } else if (la == kc + fa) {
    transA = true;
    ldA = M;
  } else {
    ta.alloc(A.size(), s);
    permuteT<T>(s, A.p, A.dims, perm_of(la, fa + kc), ta.p, T(1), T(0));
    pa = ta.p;
  }
  const T* pb = B.p;
  bool transB = true;  // B used as N x K
  long long ldB = K;
  if (lb == fb + kc) {
  } else if (lb == kc + fb) {
    transB = false;
    ldB = N;
  } else {
    tb.alloc(B.size(), s);
    permuteT<T>(s, B.p, B.dims, perm_of(lb, fb + kc), tb.p, T(1), T(0));
    pb = tb.p;
  }
  std::string lt = fa + fb;
  std::vector<int> pC = perm_of(lt, lc);
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) fail(EAADC_ERR_ARG, "einsum: extent too large");
  if (is_id(pC)) {
    gemm<T>(s, transA, transB, (int)M, (int)N, (int)K, alpha, pa, ldA, pb, ldB, beta, C.p, N, GemmBatch());
  } else {
    tc.alloc((size_t)(M * N), s);
    gemm<T>(s, transA, transB, (int)M, (int)N, (int)K, T(1), pa, ldA, pb, ldB, T(0), tc.p, N, GemmBatch());
    std::vector<int> tdims;
    for (char c : lt) tdims.push_back(dim[c]);
    permuteT<T>(s, tc.p, tdims, pC, C.p, alpha, beta);
  }
}
template void einsumT<double>(cudaStream_t, const char*, double, const TensT<double>&, const TensT<double>&, double,
                              const TensT<double>&);
template void einsumT<float>(cudaStream_t, const char*, float, const TensT<float>&, const TensT<float>&, float,
                             const TensT<float>&);

// ------------------------------------------------------------------ Jacobi
namespace {
__global__ void __launch_bounds__(1024) jacobi_kernel(int m, double* __restrict__ Ag, double* __restrict__ w,
                                                      double* __restrict__ Ug, int max_sweeps) {
  extern __shared__ double sm[];
  const int n = (m + 1) & ~1;  // even number of players (dummy index m if m is odd)
  double* A = sm;              // [m][m]
  double* U = sm + (size_t)m * m;
  double* cs = U + (size_t)m * m;  // [n/2] cos
  double* sn = cs + n / 2;         // [n/2] sin
  int* pp = (int*)(sn + n / 2);    // [n/2]
  int* qq = pp + n / 2;
  __shared__ double red[32];
  __shared__ int stop;
  const int tid = threadIdx.x, nt = blockDim.x;
  // batch: one matrix per CTA
  Ag += (size_t)blockIdx.x * m * m;
  Ug += (size_t)blockIdx.x * m * m;
  w += (size_t)blockIdx.x * m;
  for (int i = tid; i < m * m; i += nt) {
    A[i] = Ag[i];
    U[i] = (i / m == i % m) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence: off-diagonal vs diagonal magnitude
    double off = 0.0, dg = 0.0;
    for (int i = tid; i < m * m; i += nt) {
      double a = A[i];
      if (i / m == i % m) dg += a * a; else off += a * a;
    }
    for (int o = 16; o; o >>= 1) { off += __shfl_xor_sync(0xffffffffu, off, o); dg += __shfl_xor_sync(0xffffffffu, dg, o); }
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < (nt + 31) / 32; ++i) t += red[i];
      red[0] = t;
    }
    __syncthreads();
    off = red[0];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = dg;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < (nt + 31) / 32; ++i) t += red[i];
      stop = (off <= 1e-30 * t) || (off < 1e-300);
    }
    __syncthreads();
    if (stop) break;
    for (int step = 0; step < n - 1; ++step) {
      for (int i = tid; i < n / 2; i += nt) {
        int a = (i == 0) ? 0 : 1 + (i - 1 + step) % (n - 1);
        int j = n - 1 - i;
        int b = 1 + (j - 1 + step) % (n - 1);
        int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < m) {
          double apq = A[p * m + q];
          if (fabs(apq) > 1e-300) {
            double th = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
            double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
      }
      __syncthreads();
      // A <- A J (columns p, q) and U <- U J
      for (int e = tid; e < (n / 2) * m; e += nt) {
        int i = e / m, r = e % m;
        int p = pp[i], q = qq[i];
        if (q >= m) continue;
        double c = cs[i], s = sn[i];
        double ap = A[r * m + p], aq = A[r * m + q];
        A[r * m + p] = c * ap - s * aq;
        A[r * m + q] = s * ap + c * aq;
        double up = U[r * m + p], uq = U[r * m + q];
        U[r * m + p] = c * up - s * uq;
        U[r * m + q] = s * up + c * uq;
      }
      __syncthreads();
      // A <- J^T A (rows p, q)
      for (int e = tid; e < (n / 2) * m; e += nt) {
        int i = e / m, r = e % m;
        int p = pp[i], q = qq[i];
        if (q >= m) continue;
        double c = cs[i], s = sn[i];
        double ap = A[p * m + r], aq = A[q * m + r];
        A[p * m + r] = c * ap - s * aq;
        A[q * m + r] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
  // sort eigenvalues ascending (selection by rank; ties broken by index)
  for (int i = tid; i < m; i += nt) {
    double di = A[i * m + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      double dj = A[j * m + j];
      rank += (dj < di) || (dj == di && j < i);
    }
    w[rank] = di;
    for (int r = 0; r < m; ++r) Ug[r * m + rank] = U[r * m + i];
  }
}
}  // namespace

void jacobi_eigh(cudaStream_t s, int m, double* A, double* w, double* U, int nbatch) {
  if (m <= 0 || nbatch <= 0) return;
  if (m > 96) fail(EAADC_ERR_ARG, "jacobi_eigh: m > 96");
  int n = (m + 1) & ~1;
  size_t smem = sizeof(double) * (2 * (size_t)m * m + n) + sizeof(int) * n;
  static bool attr = false;
  if (!attr) {
    EA_CK(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  jacobi_kernel<<<nbatch, 1024, smem, s>>>(m, A, w, U, 60);
  EA_LAUNCH();
}

}  // namespace ea
