// eaadc_ladder_noalloc: the tensor-core DF ladder with no device allocation.
//
// eaadc_ladder takes its working memory (the BF16 copy of the vectors, the
// stage-1 intermediate and, for widths that are not a multiple of 8, an FP32
// staging copy of the result) from the stream-ordered allocator on every
// call.  Some callers cannot allow that: a process whose device memory is
// already handed out to its own memory manager (a framework's caching
// allocator, a server that reserves HBM at start-up) sees such allocations
// fail or forces its manager to release memory, and a cudaFree synchronises
// the whole device, which stalls the caller's other streams.  This variant
// takes the same working memory from one fixed array in device memory
// (kScratchBytes, below), which every GPU that loads the library holds until
// the process exits.  It computes the same two stages as eaadc_ladder; the
// auxiliary index is cut into as many blocks as the array needs.
#include "internal.cuh"
#include "tc_gemm2.cuh"

#include <algorithm>
#include <mutex>
#include <string>

namespace {

using ea::bf16;
namespace tc2 = ea::tc2;

constexpr size_t kScratchBytes = EAADC_LADDER_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_ladder_scratch[kScratchBytes];

// Device address of g_ladder_scratch per device, looked up once with that
// device current (the host-side symbol is only a stand-in for it).
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

void* scratch_address(int dev) {
  if (dev < 0 || dev >= kMaxDevices) ea::fail(EAADC_ERR_ARG, "ladder_noalloc: device index beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_ladder_scratch);
    if (e != cudaSuccess || !p)
      ea::fail(EAADC_ERR_CUDA, std::string("ladder_noalloc: cudaGetSymbolAddress of the scratch array failed: ") +
                                   cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

size_t round256(size_t n) { return (n + 255) / 256 * 256; }
long long pad8(long long n) { return (n + 7) / 8 * 8; }
long long rp64(long long n) { return (n + 63) / 64 * 64; }  // BF16 row pitch: whole 128-byte lines
long long rp32(long long n) { return (n + 31) / 32 * 32; }  // FP32 row pitch: whole 128-byte lines
int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

// W[(n,k,d)][e] (row pitch wp) = bf16(x[n][v + (k,d,e)])
__global__ void noalloc_pack_w(const double* __restrict__ x, bf16* __restrict__ W, int nvec, long long dim, int v,
                               long long n2, long long wp) {
  const long long total = n2 * nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / n2, r = i % n2;
    W[(i / v) * wp + i % v] = __float2bfloat16_rn((float)x[n * dim + v + r]);
  }
}

// out[r][c] (row pitch v) = L[r][c] (row pitch lp), c < v
__global__ void noalloc_compact(const float* __restrict__ L, long long lp, float* __restrict__ out, long long rows,
                                int v) {
  const long long total = rows * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    out[i] = L[(i / v) * lp + i % v];
}

tc2::Args plain_args(int M, int N, int K, int* err) {
  tc2::Args g{};
  g.M = M; g.N = N; g.K = K;
  g.BN = ea::pick_bn(N);
  g.nzlo = 1; g.nz = 1;
  g.alpha = 1.f;
  g.err = err;
  return g;
}

void ladder_noalloc(cudaStream_t s, ea::State& st, int nvec, const double* x, float* out, unsigned char* base) {
  using namespace ea;
  const int o = st.o, v = st.v, naux = st.naux;
  const long long dp = pad8(v), wp = rp64(v), lp = rp32(v), bk = (long long)naux * dp;
  const long long bvp = st.bvv_pitch, bbp = st.bb_pitch;
  const long long nmat = (long long)nvec * o, n2 = (long long)o * v * v;
  const bool staged = v % 4 != 0;  // rows of out are not whole 16-byte units: stage the result
  // scratch layout: [W bf16 nmat*v*wp] [L fp32 nmat*v*lp, if staged] [Z bf16 nmat*v*zp]
  const size_t wbytes = round256((size_t)(nmat * v * wp) * sizeof(bf16));
  const size_t lbytes = staged ? round256((size_t)(nmat * v * lp) * sizeof(float)) : 0;
  auto zbytes = [&](long long q) { return (size_t)(nmat * v * rp64(q * dp)) * sizeof(bf16); };
  if (wbytes + lbytes + zbytes(1) > kScratchBytes)
    fail(EAADC_ERR_ARG, "ladder_noalloc: " + std::to_string(nvec) + " vectors need at least " +
                            std::to_string(wbytes + lbytes + zbytes(1)) + " bytes of scratch, the fixed limit is " +
                            std::to_string(kScratchBytes) + " (use fewer vectors per call, or eaadc_ladder)");
  const size_t zroom = kScratchBytes - wbytes - lbytes;
  int qc = (int)std::min<long long>(naux, (long long)(zroom / ((size_t)(nmat * v * dp) * sizeof(bf16))));
  while (qc > 1 && zbytes(qc) > zroom) --qc;
  const long long zp = rp64((long long)qc * dp);  // Z row pitch
  bf16* W = reinterpret_cast<bf16*>(base);
  float* L = staged ? reinterpret_cast<float*>(base + wbytes) : out;
  const long long op = staged ? lp : v;
  bf16* Z = reinterpret_cast<bf16*>(base + wbytes + lbytes);
  // Stage 1 writes only the v real columns of each dp-wide block of Z, and
  // stage 2 reads the pads: they must be zero, not what the last call left.
  if (dp != v) EA_CK(cudaMemsetAsync(Z, 0, zbytes(qc), s));

  noalloc_pack_w<<<grid_for(n2 * nvec), 256, 0, s>>>(x, W, nvec, st.dim, v, n2, wp);
  EA_LAUNCH();
  const int bn = pick_bn(v);
  TmaMap mB3 = make_tma_3d(st.Bvv_bf.p, v, v, naux, bvp, v * bvp, 128);  // stage-1 A: B^Q [Q][c][e]
  TmaMap mW = make_tma_3d(W, v, v, nmat, wp, (long long)v * wp, bn);     // stage-1 B: W [nk][d][e]
  TmaMap mBb = make_tma_3d(st.Bb_bf.p, bk, v, 1, bbp, bbp * v, bn);      // stage-2 B: [b][(Q,d)]
  TmaMap mOut = make_tma_out4d(L, 4, v, 1, nmat * v, 1, op, op, nmat * v * op);
  for (int Q0 = 0; Q0 < naux; Q0 += qc) {
    const int q = std::min(qc, naux - Q0);
    // stage 1: Z[nk][c][Q][d] = sum_e B^Q[c][e] W_nk[d][e] for Q in [Q0, Q0+q)
    tc2::Args g1 = plain_args(v, v, v, st.err.p);
    g1.nzlo = q; g1.nz = (int)(q * nmat);
    g1.a_sel = tc2::Z_LO; g1.a_z0 = Q0;
    g1.b_sel = tc2::Z_HI;
    g1.out_bf16 = 1;
    TmaMap mZo = make_tma_out4d(Z, 2, v, q, v, nmat, dp, zp, (long long)v * zp);
    tc_gemm2(s, mB3, mW, mZo, g1);
    // stage 2: L[(nk,c)][b] (+)= sum_(Q,d) Z[(nk,c)][(Q,d)] B^Q[b][d]
    TmaMap mZ = make_tma_3d(Z, (long long)q * dp, nmat * v, 1, zp, nmat * v * zp, 128);
    tc2::Args g2 = plain_args((int)(nmat * v), v, (int)(q * dp), st.err.p);
    g2.b_k0 = (int)(Q0 * dp);
    g2.reduce = Q0 > 0;
    tc_gemm2(s, mZ, mBb, mOut, g2);
  }
  if (staged) {
    noalloc_compact<<<grid_for(n2 * nvec), 256, 0, s>>>(L, lp, out, nmat * v, v);
    EA_LAUNCH();
  }
}

}  // namespace

extern "C" eaadc_status eaadc_ladder_noalloc(eaadc_ctx* ctx, int state, int nvec, const double* x_dev,
                                             float* out_dev, void* stream) {
  if (!ctx) return EAADC_ERR_ARG;
  try {
    ctx->err.clear();
    EA_CK(cudaSetDevice(ctx->device));
    if (state < 0 || state >= (int)ctx->states.size()) ea::fail(EAADC_ERR_ARG, "state index out of range");
    ea::State& st = *ctx->states[state];
    if (st.order < 3) ea::fail(EAADC_ERR_STATE, "the ladder is part of ADC(3) only");
    if (nvec <= 0 || !x_dev || !out_dev) ea::fail(EAADC_ERR_ARG, "bad vector arguments");
    if (reinterpret_cast<uintptr_t>(out_dev) % 16) ea::fail(EAADC_ERR_ARG, "out_dev must be 16-byte aligned");
    if (!st.mixed_ready || !st.err.p)
      ea::fail(EAADC_ERR_STATE,
               "the BF16 operands of this state do not exist yet: call eaadc_ladder or a reduced-precision "
               "eaadc_sigma on it once first");
    unsigned char* base = static_cast<unsigned char*>(scratch_address(ctx->device));
    ladder_noalloc((cudaStream_t)stream, st, nvec, x_dev, out_dev, base);
    return EAADC_OK;
  } catch (const ea::Error& e) {
    ctx->err = e.msg;
    return e.st;
  } catch (...) {
    ctx->err = "unknown internal error";
    return EAADC_ERR_STATE;
  }
}
