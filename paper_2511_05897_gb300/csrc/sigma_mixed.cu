// Mixed-precision sigma: every o v^3-scaling contraction runs on tcgen05
// tensor cores with BF16 operands and FP32 accumulation; the orbital-energy
// diagonal, the 1p/1p block and the DF contractions that scale as
// naux * o * v^2 stay in FP64.
//
// Ladder (Sec. II.B: four-virtual integrals are never formed; (bd|ce) enters
// as two DF contractions):
//   stage 1  Z[(nk,c)][(Q,d)] = sum_e B^Q[c][e] W_nk[d][e]
//   stage 2  L[(nk,c)][b]     = sum_(Q,d) Z[(nk,c)][(Q,d)] B^Q[b][d] = (sum_Q B^Q W_nk B^Q)[b][c]
// in chunks of qc auxiliary functions (BF16 intermediate Z about 96 MB);
// stage 2 is one GEMM over all pair matrices nk, accumulated over chunks by
// TMA reduce-add.
// Ring and coupling: sigma_A = -T1[(k,b),(n,c)] - T2[(k,c),(n,b)] with
//   T1 = K AmT^T + tauC F1^T
//   T2 = J BmT^T + K AtT^T + tm2C G1^T + tauD F1^T
// (K, J: stored (oo|vv), (ov|ov) integrals; tau*: first-order amplitudes as
// (ov x ov) matrices) as two long-K GEMMs over concatenated operands, and the
// 2p1h -> 1p intermediates H1 = tauA V1^T, [H2; H3] = [tm2A; tauB] V2^T.
#include "internal.cuh"
#include "tc_gemm2.cuh"

#include <algorithm>

namespace ea {
namespace {
const double kS1 = 0.5 * (1.0 + 1.7320508075688772935);
const double kS2 = 0.5 * (1.0 - 1.7320508075688772935);
const double kI1 = 0.5 * (1.0 + 0.57735026918962576451);
const double kI2 = 0.5 * (1.0 - 0.57735026918962576451);

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }
long long pad8(long long n) { return (n + 7) / 8 * 8; }

struct OpDst {
  bf16* p;
  long long pitch;
};

// out[r][c] (pitch op) = in[r][c] (pitch ip), c < cols, rows r < rows
__global__ void f64_to_bf16_pitched(const double* __restrict__ in, long long ip, bf16* __restrict__ out, long long op,
                                    long long rows, long long cols) {
  long long n = rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long r = i / cols, c = i % cols;
    out[r * op + c] = __float2bfloat16_rn((float)in[r * ip + c]);
  }
}

// Bb[b][Q*dp + d] (pitch bp) = B[Q][b][d]; pad columns d >= v stay zero
__global__ void bmajor_bf16(const double* __restrict__ B, bf16* __restrict__ Bb, int naux, int v, long long dp,
                            long long bp) {
  long long n = (long long)naux * v * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int d = i % v;
    long long r = i / v;
    int Q = r % naux;
    int b = (int)(r / naux);
    Bb[(long long)b * bp + (long long)Q * dp + d] = __float2bfloat16_rn((float)B[((long long)Q * v + b) * v + d]);
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

// Per-vector 2p1h operands from W (w-representation), A = S^-1 W, V = S W;
// rows (n, x), columns (l, y):
//   AmT = A[l][y][x]  AtT = A[l][x][y]  BmT = AmT - 2 AtT  V1 = V[l][y][x]  V2 = V[l][x][y]
__global__ void ring_operands(const double* __restrict__ x, OpDst AmT, OpDst BmT, OpDst AtT, OpDst V1, OpDst V2,
                              int nvec, long long dim, int o, int v) {
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
    const long long row = n * v + xx, col = (long long)l * v + y;
    AmT.p[row * AmT.pitch + col] = __float2bfloat16_rn((float)am);
    AtT.p[row * AtT.pitch + col] = __float2bfloat16_rn((float)at);
    BmT.p[row * BmT.pitch + col] = __float2bfloat16_rn((float)(am - 2.0 * at));
    V1.p[row * V1.pitch + col] = __float2bfloat16_rn((float)(kS1 * wyx + kS2 * wxy));
    V2.p[row * V2.pitch + col] = __float2bfloat16_rn((float)(kS1 * wxy + kS2 * wyx));
  }
}

// F1[(n,c)][(l,d)] = F_n[l][c][d] into two destinations; G1[(n,b)][(l,d)] = G_n[b][l][d]
__global__ void fg_operands(const double* __restrict__ F, const double* __restrict__ G, OpDst F1a, OpDst F1b,
                            OpDst G1, int nvec, int o, int v) {
  const long long ov = (long long)o * v, n2 = ov * v;
  const long long total = (long long)nvec * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / n2, r = i % n2;
    {  // F_n[l][c][d]
      const int d = r % v, c = (r / v) % v, l = (int)(r / ((long long)v * v));
      const bf16 f = __float2bfloat16_rn((float)F[i]);
      const long long row = n * v + c, col = (long long)l * v + d;
      F1a.p[row * F1a.pitch + col] = f;
      F1b.p[row * F1b.pitch + col] = f;
    }
    {  // G_n[b][l][d]
      const int d = r % v, l = (r / v) % o, b = (int)(r / ov);
      G1.p[(n * v + b) * G1.pitch + (long long)l * v + d] = __float2bfloat16_rn((float)G[i]);
    }
  }
}

// FP64 per-vector H tensors from the tensor-core outputs (rows (l,d), columns (n,x)):
//   H1_n[l][d][c] = H1[(l,d)][(n,c)]
//   H2_n[b][l][d] = H23[(l,d)][(n,b)]        H3_n[l][b][d] = H23[ov + (l,d)][(n,b)]
__global__ void h_from_tc(const float* __restrict__ H1, const float* __restrict__ H23, double* __restrict__ h1,
                          double* __restrict__ h2, double* __restrict__ h3, int nvec, int o, int v, long long nv) {
  const long long ov = (long long)o * v, n2 = ov * v;
  const long long total = (long long)nvec * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / n2, r = i % n2;
    const int t = r % v, q = (r / v) % v, p = (int)(r / ((long long)v * v));
    h1[i] = (double)H1[((long long)p * v + q) * nv + n * v + t];         // l=p, d=q, c=t
    h3[i] = (double)H23[(ov + (long long)p * v + t) * nv + n * v + q];  // l=p, b=q, d=t
    const long long b = r / ov, l = (r / v) % o, d = r % v;
    h2[i] = (double)H23[(l * v + d) * nv + n * v + b];
  }
}

// y[n][v + (k,b,c)] += S(-T1[(k,b)][(n,c)] - T2[(k,c)][(n,b)]) + L[(n,k,c)][b]
// (T rows pitch nv, L rows pitch lp)
__global__ void combine_ring_ladder(double* __restrict__ y, const float* __restrict__ T1, const float* __restrict__ T2,
                                    const float* __restrict__ L, int nvec, long long dim, int o, int v, long long nv,
                                    long long lp) {
  const long long vv = (long long)v * v, n2 = (long long)o * vv;
  const long long total = n2 * nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    long long n = i / n2, r = i % n2;
    int c = r % v;
    long long q = r / v;
    int b = q % v;
    int k = (int)(q / v);
    double abc = -(double)T1[((long long)k * v + b) * nv + n * v + c] - (double)T2[((long long)k * v + c) * nv + n * v + b];
    double acb = -(double)T1[((long long)k * v + c) * nv + n * v + b] - (double)T2[((long long)k * v + b) * nv + n * v + c];
    double acc = kS1 * abc + kS2 * acb;
    acc += (double)L[((n * o + k) * v + c) * lp + b];
    y[n * dim + v + r] += acc;
  }
}

// (ov x ov) BF16 coupling operands from tau[l][k][x][y]:
//   tauA[(l,y),(k,x)] = tauC[(k,x),(l,y)] = tau[l,k,x,y]
//   tauB[(l,x),(k,y)] = tauD[(k,y),(l,x)] = tau[l,k,x,y]
//   tm2A[(l,y),(k,x)] = tm2C[(k,x),(l,y)] = tau[l,k,x,y] - 2 tau[l,k,y,x]
__global__ void tau_operands(const double* __restrict__ tau, OpDst tA, OpDst tB, OpDst tC, OpDst tD, OpDst m2A,
                             OpDst m2C, int o, int v) {
  const long long total = (long long)o * o * v * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    int y = i % v;
    long long r = i / v;
    int xx = r % v;
    r /= v;
    int k = r % o;
    int l = (int)(r / o);
    double t = tau[i];
    double tsw = tau[(((long long)l * o + k) * v + y) * v + xx];
    bf16 tb = __float2bfloat16_rn((float)t);
    bf16 mb = __float2bfloat16_rn((float)(t - 2.0 * tsw));
    const long long ly = (long long)l * v + y, kx = (long long)k * v + xx, lx = (long long)l * v + xx,
                    ky = (long long)k * v + y;
    tA.p[ly * tA.pitch + kx] = tb;
    tC.p[kx * tC.pitch + ly] = tb;
    tB.p[lx * tB.pitch + ky] = tb;
    tD.p[ky * tD.pitch + lx] = tb;
    m2A.p[ly * m2A.pitch + kx] = mb;
    m2C.p[kx * m2C.pitch + ly] = mb;
  }
}

__global__ void zero_int(int* p) { *p = 0; }

void prepare_mixed(cudaStream_t s, State& st) {
  if (st.mixed_ready) return;
  const int o = st.o, v = st.v, naux = st.naux;
  const long long vv = (long long)v * v, ov = (long long)o * v;
  const long long vp = pad8(v), bp = (long long)naux * vp, ovp = pad8(ov);
  st.Bvv_bf.alloc((size_t)(naux * v * vp), s);
  f64_to_bf16_pitched<<<gridn(naux * vv), 256, 0, s>>>(st.Bvv.p, v, st.Bvv_bf.p, vp, (long long)naux * v, v);
  EA_LAUNCH();
  st.Bb_bf.alloc((size_t)(v * bp), s);
  if (vp != v) EA_CK(cudaMemsetAsync(st.Bb_bf.p, 0, st.Bb_bf.n * sizeof(bf16), s));
  bmajor_bf16<<<gridn(naux * vv), 256, 0, s>>>(st.Bvv.p, st.Bb_bf.p, naux, v, vp, bp);
  EA_LAUNCH();
  if (st.order >= 3) {
    // A-side operands; segments are ov wide with pitch ovp (pad columns zero):
    //   T1: [K | tauC]   T2: [J | K | tm2C | tauD]   H1: tauA   H2/H3: [tm2A ; tauB] (stacked rows)
    st.Kmat_bf.alloc((size_t)(ov * 2 * ovp), s);
    st.Jmat_bf.alloc((size_t)(ov * 4 * ovp), s);
    st.tauA_bf.alloc((size_t)(ov * ovp), s);
    st.tm2A_bf.alloc((size_t)(2 * ov * ovp), s);
    EA_CK(cudaMemsetAsync(st.Kmat_bf.p, 0, st.Kmat_bf.n * sizeof(bf16), s));
    EA_CK(cudaMemsetAsync(st.Jmat_bf.p, 0, st.Jmat_bf.n * sizeof(bf16), s));
    EA_CK(cudaMemsetAsync(st.tauA_bf.p, 0, st.tauA_bf.n * sizeof(bf16), s));
    EA_CK(cudaMemsetAsync(st.tm2A_bf.p, 0, st.tm2A_bf.n * sizeof(bf16), s));
    f64_to_bf16_pitched<<<gridn(ov * ov), 256, 0, s>>>(st.Kmat.p, ov, st.Kmat_bf.p, 2 * ovp, ov, ov);
    EA_LAUNCH();
    f64_to_bf16_pitched<<<gridn(ov * ov), 256, 0, s>>>(st.Jmat.p, ov, st.Jmat_bf.p, 4 * ovp, ov, ov);
    EA_LAUNCH();
    f64_to_bf16_pitched<<<gridn(ov * ov), 256, 0, s>>>(st.Kmat.p, ov, st.Jmat_bf.p + ovp, 4 * ovp, ov, ov);
    EA_LAUNCH();
    OpDst tA{st.tauA_bf.p, ovp}, tC{st.Kmat_bf.p + ovp, 2 * ovp}, tD{st.Jmat_bf.p + 3 * ovp, 4 * ovp},
        m2C{st.Jmat_bf.p + 2 * ovp, 4 * ovp}, m2A{st.tm2A_bf.p, ovp}, tB{st.tm2A_bf.p + ov * ovp, ovp};
    tau_operands<<<gridn(ov * ov), 256, 0, s>>>(st.tau.p, tA, tB, tC, tD, m2A, m2C, o, v);
    EA_LAUNCH();
  }
  if (!st.err.p) {
    st.err.alloc(1, s);
    zero_int<<<1, 1, 0, s>>>(st.err.p);
    EA_LAUNCH();
  }
  st.mixed_ready = true;
}

tc2::Args gargs(int M, int N, int K, int* err) {
  tc2::Args g{};
  g.M = M; g.N = N; g.K = K;
  g.BN = pick_bn(N);
  g.nzlo = 1; g.nz = 1;
  g.alpha = 1.f;
  g.err = err;
  return g;
}

// compact out[r][c] (pitch v) = in[r][c] (pitch ip)
__global__ void compact_f32(const float* __restrict__ in, long long ip, float* __restrict__ out, long long rows, int v) {
  long long n = rows * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[(i / v) * ip + i % v];
}
}  // namespace

// Transposed ladder out[(nk,c)][b] (row pitch pad8(v)) = (sum_Q B^Q W_nk B^Q)[b][c]
// for nmat pair matrices W (bf16, rows (nk,d), columns e, pitch pad8(v)).
//   stage 1 (batch Q x nk): Z[nk][c][Q][d] = sum_e B^Q[c][e] W_nk[d][e]
//   stage 2 (one GEMM):     out[(nk,c)][b] (+)= sum_(Q,d) Z[(nk,c)][(Q,d)] B^Q[b][d]
// Z rows hold qc blocks of pad8(v) columns (pads zero, matching the zero pads
// of the b-major copy of B), chunk accumulation by TMA reduce-add.
void ladder_tc(cudaStream_t s, State& st, const bf16* Wbf, int nmat, float* out) {
  const int v = st.v, naux = st.naux;
  const long long dp = pad8(v), bp = (long long)naux * dp;
  // chunk of auxiliary functions: Z about 48M bf16 elements
  int qc = (int)std::max<long long>(1, (48LL << 20) / std::max<long long>(1, (long long)nmat * v * dp));
  qc = std::min(qc, naux);
  DArr<bf16> Z((size_t)nmat * v * qc * dp, s);
  if (dp != v) EA_CK(cudaMemsetAsync(Z.p, 0, Z.n * sizeof(bf16), s));
  TmaMap mB3 = make_tma_3d(st.Bvv_bf.p, v, v, naux, dp, v * dp, 128);                  // stage-1 A: [Q][c][e]
  const int bn = pick_bn(v);
  TmaMap mW = make_tma_3d(Wbf, v, v, nmat, dp, (long long)v * dp, bn);                 // stage-1 B: [nk][d][e]
  TmaMap mBb = make_tma_3d(st.Bb_bf.p, bp, v, 1, bp, bp * v, bn);                      // stage-2 B: [b][(Q,d)]
  TmaMap mOut = make_tma_out4d(out, 4, v, 1, (long long)nmat * v, 1, dp, dp, (long long)nmat * v * dp);
  for (int Q0 = 0; Q0 < naux; Q0 += qc) {
    const int q = std::min(qc, naux - Q0);
    TmaMap mZo = make_tma_out4d(Z.p, 2, v, q, v, nmat, dp, (long long)qc * dp, (long long)v * qc * dp);
    tc2::Args g1 = gargs(v, v, v, st.err.p);
    g1.nzlo = q; g1.nz = q * nmat;
    g1.a_sel = tc2::Z_LO; g1.a_z0 = Q0;
    g1.b_sel = tc2::Z_HI;
    g1.out_bf16 = 1;
    tc_gemm2(s, mB3, mW, mZo, g1);
    // K extent of this chunk exactly q*dp: columns past it read as zero
    TmaMap mZ = make_tma_3d(Z.p, (long long)q * dp, (long long)nmat * v, 1, (long long)qc * dp,
                            (long long)nmat * v * qc * dp, 128);
    tc2::Args g2 = gargs(nmat * v, v, (int)(q * dp), st.err.p);
    g2.b_k0 = (int)(Q0 * dp);
    g2.reduce = (Q0 > 0);
    tc_gemm2(s, mZ, mBb, mOut, g2);
  }
}

void sigma_mixed(cudaStream_t s, State& st, int nvec, const double* x, double* y) {
  if (st.order < 3) {  // ADC(2): first-order coupling and diagonal only, no tensor-core terms
    sigma_base_fp64(s, st, nvec, x, y, false, false);
    return;
  }
  prepare_mixed(s, st);
  const int o = st.o, v = st.v;
  const long long vv = (long long)v * v, ov = (long long)o * v, n2 = ov * v, dim = st.dim;
  const long long vp = pad8(v), ovp = pad8(ov), nv = (long long)nvec * v;
  // FP64: orbital-energy diagonal, 1p/1p block, small coupling pieces and the DF intermediates F, G
  diag_and_m11(s, st, nvec, x, y);
  DArr<double> F((size_t)(nvec * n2), s), G((size_t)(nvec * n2), s), CA((size_t)n2, s);
  for (int n = 0; n < nvec; ++n) {
    couple_1p_to_2p1h(s, st, x + n * dim, CA.p, nullptr, false, F.p + n * n2, G.p + n * n2);
    pair_combine(s, CA.p, vv, y + n * dim + v, vv, o, v, kS1, kS2, 1.0, 1.0);
  }
  // BF16 operands
  DArr<bf16> Wbf((size_t)(ov * nvec * vp), s);
  pack_w_bf16<<<gridn(n2 * nvec), 256, 0, s>>>(x, Wbf.p, nvec, dim, v, n2, vp);
  EA_LAUNCH();
  DArr<bf16> B1((size_t)(nv * 2 * ovp), s), B2((size_t)(nv * 4 * ovp), s), BV1((size_t)(nv * ovp), s),
      BV2((size_t)(nv * ovp), s);
  if (ovp != ov) {
    EA_CK(cudaMemsetAsync(B1.p, 0, B1.n * sizeof(bf16), s));
    EA_CK(cudaMemsetAsync(B2.p, 0, B2.n * sizeof(bf16), s));
  }
  // B1 = [AmT | F1], B2 = [BmT | AtT | G1 | F1]
  ring_operands<<<gridn(nv * ov), 256, 0, s>>>(x, OpDst{B1.p, 2 * ovp}, OpDst{B2.p, 4 * ovp},
                                                OpDst{B2.p + ovp, 4 * ovp}, OpDst{BV1.p, ovp}, OpDst{BV2.p, ovp},
                                                nvec, dim, o, v);
  EA_LAUNCH();
  fg_operands<<<gridn(nvec * n2), 256, 0, s>>>(F.p, G.p, OpDst{B1.p + ovp, 2 * ovp}, OpDst{B2.p + 3 * ovp, 4 * ovp},
                                               OpDst{B2.p + 2 * ovp, 4 * ovp}, nvec, o, v);
  EA_LAUNCH();
  // tensor-core GEMMs
  DArr<float> L((size_t)(ov * nvec * vp), s);
  ladder_tc(s, st, Wbf.p, nvec * o, L.p);
  const long long nvp = pad8(nv);
  DArr<float> T1((size_t)(ov * nvp), s), T2((size_t)(ov * nvp), s), H1((size_t)(ov * nvp), s),
      H23((size_t)(2 * ov * nvp), s);
  TmaMap aT1 = make_tma_3d(st.Kmat_bf.p, 2 * ovp, ov, 1, 2 * ovp, ov * 2 * ovp, 128);
  TmaMap aT2 = make_tma_3d(st.Jmat_bf.p, 4 * ovp, ov, 1, 4 * ovp, ov * 4 * ovp, 128);
  TmaMap aH1 = make_tma_3d(st.tauA_bf.p, ov, ov, 1, ovp, ov * ovp, 128);
  TmaMap aH23 = make_tma_3d(st.tm2A_bf.p, ov, 2 * ov, 1, ovp, 2 * ov * ovp, 128);
  const int bnn = pick_bn((int)nv);
  TmaMap bT1 = make_tma_3d(B1.p, 2 * ovp, nv, 1, 2 * ovp, nv * 2 * ovp, bnn);
  TmaMap bT2 = make_tma_3d(B2.p, 4 * ovp, nv, 1, 4 * ovp, nv * 4 * ovp, bnn);
  TmaMap bV1 = make_tma_3d(BV1.p, ov, nv, 1, ovp, nv * ovp, bnn);
  TmaMap bV2 = make_tma_3d(BV2.p, ov, nv, 1, ovp, nv * ovp, bnn);
  auto outmap = [&](float* p, long long rows) { return make_tma_out4d(p, 4, nv, 1, rows, 1, nvp, nvp, rows * nvp); };
  tc2::Args g = gargs((int)ov, (int)nv, (int)(2 * ovp), st.err.p);
  tc_gemm2(s, aT1, bT1, outmap(T1.p, ov), g);
  g.K = (int)(4 * ovp);
  tc_gemm2(s, aT2, bT2, outmap(T2.p, ov), g);
  g.K = (int)ov;
  tc_gemm2(s, aH1, bV1, outmap(H1.p, ov), g);
  g.M = (int)(2 * ov);
  tc_gemm2(s, aH23, bV2, outmap(H23.p, 2 * ov), g);
  combine_ring_ladder<<<gridn(n2 * nvec), 256, 0, s>>>(y, T1.p, T2.p, L.p, nvec, dim, o, v, nvp, vp);
  EA_LAUNCH();
  // 2p1h -> 1p finishing in FP64 from the tensor-core H tensors
  DArr<double> h1((size_t)(nvec * n2), s), h2((size_t)(nvec * n2), s), h3((size_t)(nvec * n2), s), V((size_t)n2, s);
  h_from_tc<<<gridn(nvec * n2), 256, 0, s>>>(H1.p, H23.p, h1.p, h2.p, h3.p, nvec, o, v, nvp);
  EA_LAUNCH();
  for (int n = 0; n < nvec; ++n) {
    pair_combine(s, x + n * dim + v, vv, V.p, vv, o, v, kS1, kS2, 1.0, 0.0);
    couple_2p1h_to_1p(s, st, V.p, y + n * dim, nullptr, h1.p + n * n2, h2.p + n * n2, h3.p + n * n2);
  }
}

// Ladder alone, transposed FP32 output [nvec][o][c][b] (= ladder[b][c]), for timing the dominant kernel.
void ladder_only(cudaStream_t s, State& st, int nvec, const double* x, float* out, bool mixed) {
  const int o = st.o, v = st.v;
  const long long ov = (long long)o * v, n2 = ov * v;
  if (!mixed) fail(EAADC_ERR_ARG, "ladder_only: tensor-core path only");
  prepare_mixed(s, st);
  const long long vp = pad8(v);
  DArr<bf16> Wbf((size_t)(ov * nvec * vp), s);
  pack_w_bf16<<<gridn(n2 * nvec), 256, 0, s>>>(x, Wbf.p, nvec, st.dim, v, n2, vp);
  EA_LAUNCH();
  if (vp == v) {
    ladder_tc(s, st, Wbf.p, nvec * o, out);
  } else {
    DArr<float> L((size_t)(ov * nvec * vp), s);
    ladder_tc(s, st, Wbf.p, nvec * o, L.p);
    compact_f32<<<gridn(n2 * nvec), 256, 0, s>>>(L.p, vp, out, ov * nvec, v);
    EA_LAUNCH();
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
