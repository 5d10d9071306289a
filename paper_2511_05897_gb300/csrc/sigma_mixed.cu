// Mixed-precision sigma: the DF particle-particle ladder and the ring terms
// run on tcgen05 tensor cores with BF16 operands and FP32 accumulation; the
// remaining terms (orbital-energy diagonal, 1p/1p block, 1p/2p1h coupling)
// stay in FP64.
//
// Ladder (Sec. II.B: four-virtual integrals are never formed; (bd|ce) enters as
// two DF contractions):
//   stage 1  Z^Q_nk[c][d] = sum_e B^Q[c][e] W_nk[d][e]          (= (B^Q W_nk^T))
//   stage 2  sigma_nk[b][c] += sum_{Q,d} B^Q[b][d] Z^Q_nk[c][d]  (= B^Q W_nk B^Q)
// processed in chunks of qc auxiliary functions so the BF16 intermediate Z
// (nk x v x qc x v) stays small (about 64 MB, resident in L2).
// Ring: sigma_A = -K A(.,.,c) - transpose_bc[J (A - 2A^T) + K A^T] with the
// stored (oo|vv) and (ov|ov) integrals as BF16 (ov x ov) GEMM operands.
#include "internal.cuh"
#include "tc_gemm.cuh"

#include <algorithm>

namespace ea {
namespace {
const double kS1 = 0.5 * (1.0 + 1.7320508075688772935);
const double kS2 = 0.5 * (1.0 - 1.7320508075688772935);
const double kI1 = 0.5 * (1.0 + 0.57735026918962576451);
const double kI2 = 0.5 * (1.0 - 0.57735026918962576451);

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }
long long pad8(long long n) { return (n + 7) / 8 * 8; }

// out[r][c] (pitch op) = in[r][c] (pitch ip), c < cols, rows r < rows
__global__ void f64_to_bf16_pitched(const double* __restrict__ in, long long ip, bf16* __restrict__ out, long long op,
                                    long long rows, long long cols) {
  long long n = rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long r = i / cols, c = i % cols;
    out[r * op + c] = __float2bfloat16_rn((float)in[r * ip + c]);
  }
}

// Bb[b][Q*v + d] (pitch bp) = B[Q][b][d]
__global__ void bmajor_bf16(const double* __restrict__ B, bf16* __restrict__ Bb, int naux, int v, long long bp) {
  long long n = (long long)naux * v * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int d = i % v;
    long long r = i / v;
    int Q = r % naux;
    int b = (int)(r / naux);
    Bb[(long long)b * bp + (long long)Q * v + d] = __float2bfloat16_rn((float)B[((long long)Q * v + b) * v + d]);
  }
}

// Wbf[(n,k,d)][e] (pitch vp) = x[n][v + (k,d,e)]
__global__ void pack_w_bf16(const double* __restrict__ x, bf16* __restrict__ W, int nvec, long long dim, int v,
                            long long n2, long long vp) {
  long long total = n2 * nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    long long n = i / n2, r = i % n2;
    long long row = i / v, e = i % v;
    W[row * vp + e] = __float2bfloat16_rn((float)x[n * dim + v + r]);
  }
}

// Ring operands from W (w-representation) with A = S^-1 W:
//   AmT[(n,x)][(l,y)] = A[n][l][y][x], AtT[(n,x)][(l,y)] = A[n][l][x][y], BmT = AmT - 2 AtT
__global__ void ring_operands(const double* __restrict__ x, bf16* __restrict__ AmT, bf16* __restrict__ BmT,
                              bf16* __restrict__ AtT, int nvec, long long dim, int o, int v, long long ovp) {
  const long long ov = (long long)o * v;
  const long long total = (long long)nvec * v * ov;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    int y = i % v;
    long long r = i / v;
    int l = r % o;
    r /= o;
    int xx = r % v;
    long long n = r / v;
    const double* W = x + n * dim + v + (long long)l * v * v;
    double wyx = W[(long long)y * v + xx], wxy = W[(long long)xx * v + y];
    double am = kI1 * wyx + kI2 * wxy;  // A[l][y][x]
    double at = kI1 * wxy + kI2 * wyx;  // A[l][x][y]
    const long long o_ = (n * v + xx) * ovp + (long long)l * v + y;
    AmT[o_] = __float2bfloat16_rn((float)am);
    AtT[o_] = __float2bfloat16_rn((float)at);
    BmT[o_] = __float2bfloat16_rn((float)(am - 2.0 * at));
  }
}

// y[n][v + (k,b,c)] += S(-T1[k][b][n][c] - T2[k][c][n][b])  +  L[(n,k)][b][c]
__global__ void combine_ring_ladder(double* __restrict__ y, const float* __restrict__ T1, const float* __restrict__ T2,
                                    const float* __restrict__ L, int nvec, long long dim, int o, int v, int ring,
                                    int ladder) {
  const long long vv = (long long)v * v, n2 = (long long)o * vv;
  const long long total = n2 * nvec;
  const long long nv = (long long)nvec * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    long long n = i / n2, r = i % n2;
    int c = r % v;
    long long q = r / v;
    int b = q % v;
    int k = (int)(q / v);
    double acc = 0.0;
    if (ring) {
      double abc = -(double)T1[((long long)k * v + b) * nv + n * v + c] - (double)T2[((long long)k * v + c) * nv + n * v + b];
      double acb = -(double)T1[((long long)k * v + c) * nv + n * v + b] - (double)T2[((long long)k * v + b) * nv + n * v + c];
      acc += kS1 * abc + kS2 * acb;
    }
    if (ladder) acc += (double)L[i];
    y[n * dim + v + r] += acc;
  }
}

__global__ void zero_int(int* p) { *p = 0; }

void prepare_mixed(cudaStream_t s, State& st) {
  if (st.mixed_ready) return;
  const int o = st.o, v = st.v, naux = st.naux;
  const long long vv = (long long)v * v, ov = (long long)o * v;
  const long long vp = pad8(v), bp = pad8((long long)naux * v), ovp = pad8(ov);
  st.Bvv_bf.alloc((size_t)(naux * v * vp), s);
  f64_to_bf16_pitched<<<gridn(naux * vv), 256, 0, s>>>(st.Bvv.p, v, st.Bvv_bf.p, vp, (long long)naux * v, v);
  EA_LAUNCH();
  st.Bb_bf.alloc((size_t)(v * bp), s);
  bmajor_bf16<<<gridn(naux * vv), 256, 0, s>>>(st.Bvv.p, st.Bb_bf.p, naux, v, bp);
  EA_LAUNCH();
  if (st.order >= 3) {
    st.Kmat_bf.alloc((size_t)(ov * ovp), s);
    st.Jmat_bf.alloc((size_t)(ov * ovp), s);
    f64_to_bf16_pitched<<<gridn(ov * ov), 256, 0, s>>>(st.Kmat.p, ov, st.Kmat_bf.p, ovp, ov, ov);
    EA_LAUNCH();
    f64_to_bf16_pitched<<<gridn(ov * ov), 256, 0, s>>>(st.Jmat.p, ov, st.Jmat_bf.p, ovp, ov, ov);
    EA_LAUNCH();
  }
  if (!st.err.p) {
    st.err.alloc(1, s);
    zero_int<<<1, 1, 0, s>>>(st.err.p);
    EA_LAUNCH();
  }
  st.mixed_ready = true;
}

tc::GemmArgs gargs(int M, int N, int K, int* err) {
  tc::GemmArgs g{};
  g.M = M; g.N = N; g.K = K;
  g.alpha = 1.f; g.beta = 0.f;
  g.err = err;
  return g;
}
}  // namespace

// sigma_nk = sum_Q B^Q W_nk B^Q for nmat pair matrices W (bf16, rows (nk,d), cols e, pitch pad8(v))
void ladder_tc(cudaStream_t s, State& st, const bf16* Wbf, int nmat, float* out) {
  const int v = st.v, naux = st.naux;
  const long long vv = (long long)v * v, vp = pad8(v), bp = pad8((long long)naux * v);
  // chunk of auxiliary functions: Z about 32M bf16 elements, qc*v a multiple of 8
  int qc = (int)std::max<long long>(1, (32LL << 20) / std::max<long long>(1, (long long)nmat * vv));
  qc = std::min(qc, naux);
  while ((qc * v) % 8) ++qc;
  DArr<bf16> Z((size_t)nmat * v * qc * v, s);
  TmaMap mB3 = make_tma_3d(st.Bvv_bf.p, v, v, naux, vp, v * vp, 128);                     // stage-1 A: [Q][c][e]
  TmaMap mW = make_tma_3d(Wbf, v, (long long)nmat * v, 1, vp, (long long)nmat * v * vp, 256);  // stage-1 B
  TmaMap mBb = make_tma_3d(st.Bb_bf.p, (long long)naux * v, v, 1, bp, bp * v, 128);        // stage-2 A
  for (int Q0 = 0; Q0 < naux; Q0 += qc) {
    const int q = std::min(qc, naux - Q0);
    // K extent of this chunk exactly q*v: columns past it read as zero, never stale or unwritten Z
    TmaMap mZ = make_tma_3d(Z.p, (long long)q * v, v, nmat, (long long)qc * v, (long long)v * qc * v, 256);
    // stage 1: batch over Q in the chunk
    tc::GemmArgs g1 = gargs(v, nmat * v, v, st.err.p);
    g1.a_batched = 1; g1.a_z0 = Q0;
    g1.Cbf = Z.p; g1.v = v; g1.qc = qc;
    tc_gemm(s, mB3, mW, g1, q, tc::EPI_LADDER_Z, 256);
    // stage 2: batch over pair matrices; K covers the q*v columns of this chunk
    tc::GemmArgs g2 = gargs(v, v, q * v, st.err.p);
    g2.a_k0 = Q0 * v;
    g2.b_batched = 1;
    g2.beta = (Q0 == 0) ? 0.f : 1.f;
    g2.C32 = out; g2.ldc = v; g2.czs = vv;
    tc_gemm(s, mBb, mZ, g2, nmat, tc::EPI_F32, 256);
  }
}

void sigma_mixed(cudaStream_t s, State& st, int nvec, const double* x, double* y) {
  prepare_mixed(s, st);
  sigma_base_fp64(s, st, nvec, x, y, false, false);
  if (st.order < 3) return;
  const int o = st.o, v = st.v;
  const long long vv = (long long)v * v, ov = (long long)o * v, n2 = ov * v, dim = st.dim;
  // ladder
  const long long vp = pad8(v), ovp = pad8(ov);
  DArr<bf16> Wbf((size_t)(ov * nvec * vp), s);
  pack_w_bf16<<<gridn(n2 * nvec), 256, 0, s>>>(x, Wbf.p, nvec, dim, v, n2, vp);
  EA_LAUNCH();
  DArr<float> L((size_t)(n2 * nvec), s);
  ladder_tc(s, st, Wbf.p, nvec * o, L.p);
  // ring
  const long long nv = (long long)nvec * v;
  DArr<bf16> AmT((size_t)(nv * ovp), s), BmT((size_t)(nv * ovp), s), AtT((size_t)(nv * ovp), s);
  ring_operands<<<gridn(nv * ov), 256, 0, s>>>(x, AmT.p, BmT.p, AtT.p, nvec, dim, o, v, ovp);
  EA_LAUNCH();
  DArr<float> T1((size_t)(ov * nv), s), T2((size_t)(ov * nv), s);
  TmaMap mK = make_tma_3d(st.Kmat_bf.p, ov, ov, 1, ovp, ov * ovp, 128);
  TmaMap mJ = make_tma_3d(st.Jmat_bf.p, ov, ov, 1, ovp, ov * ovp, 128);
  TmaMap mAm = make_tma_3d(AmT.p, ov, nv, 1, ovp, nv * ovp, 256);
  TmaMap mBm = make_tma_3d(BmT.p, ov, nv, 1, ovp, nv * ovp, 256);
  TmaMap mAt = make_tma_3d(AtT.p, ov, nv, 1, ovp, nv * ovp, 256);
  tc::GemmArgs g = gargs((int)ov, (int)nv, (int)ov, st.err.p);
  g.C32 = T1.p; g.ldc = nv;
  tc_gemm(s, mK, mAm, g, 1, tc::EPI_F32, 256);
  g.C32 = T2.p;
  tc_gemm(s, mJ, mBm, g, 1, tc::EPI_F32, 256);
  g.beta = 1.f;
  tc_gemm(s, mK, mAt, g, 1, tc::EPI_F32, 256);
  combine_ring_ladder<<<gridn(n2 * nvec), 256, 0, s>>>(y, T1.p, T2.p, L.p, nvec, dim, o, v, 1, 1);
  EA_LAUNCH();
}

// Ladder alone (FP32 output [nvec][o][v][v]) for timing the dominant kernel.
void ladder_only(cudaStream_t s, State& st, int nvec, const double* x, float* out, bool mixed) {
  const int o = st.o, v = st.v;
  const long long ov = (long long)o * v, n2 = ov * v;
  if (mixed) {
    prepare_mixed(s, st);
    const long long vp = pad8(v);
    DArr<bf16> Wbf((size_t)(ov * nvec * vp), s);
    pack_w_bf16<<<gridn(n2 * nvec), 256, 0, s>>>(x, Wbf.p, nvec, st.dim, v, n2, vp);
    EA_LAUNCH();
    ladder_tc(s, st, Wbf.p, nvec * o, out);
  } else {
    fail(EAADC_ERR_ARG, "ladder_only: FP64 ladder output is not FP32");
  }
}

void check_device_error(cudaStream_t s, State& st) {
  if (!st.err.p) return;
  int h = 0;
  EA_CK(cudaMemcpyAsync(&h, st.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  EA_CK(cudaStreamSynchronize(s));
  if (h) fail(EAADC_ERR_TIMEOUT, "a bounded device wait expired in a tensor-core kernel (code " + std::to_string(h) + ")");
}

}  // namespace ea
