// Mixed-precision sigma: every o v^3-scaling contraction runs on tcgen05
// tensor cores with BF16 operands and FP32 accumulation; the DF coupling
// contractions that scale as naux * o * v^2 run in FP32 on CUDA cores, batched
// over the vectors; the orbital-energy diagonal and the 1p/1p block stay FP64.
//
// Ladder (Sec. II.B: four-virtual integrals are never formed; (bd|ce) enters
// as two DF contractions):
//   stage 1  Z[(nk,c)][(Q,d)] = sum_e B^Q[c][e] W_nk[d][e]
//   stage 2  L[(nk,c)][b]     = sum_(Q,d) Z[(nk,c)][(Q,d)] B^Q[b][d] = (sum_Q B^Q W_nk B^Q)[b][c]
// in chunks of qc auxiliary functions (BF16 intermediate Z of 12-96 MB, the
// chunk size and GEMM pipeline shapes picked per shape by ladder_tc's tuner);
// stage 2 is one GEMM over all pair matrices nk, accumulated over chunks by
// TMA reduce-add.
// Ring and coupling: sigma_A = -T1[(k,b),(n,c)] - T2[(k,c),(n,b)] with
//   T1 = K AmT^T + tauC F1^T
//   T2 = J BmT^T + K AtT^T + tm2C G1^T + tauD F1^T
// (K, J: stored (oo|vv), (ov|ov) integrals; tau*: first-order amplitudes as
// (ov x ov) matrices) as two long-K GEMMs over concatenated operands, and the
// 2p1h -> 1p intermediates H1 = tauA V1^T, [H2; H3] = [tm2A; tauB] V2^T.
//
// Split-BF16 mode (x3): every operand is split x = x_hi + x_lo into two BF16
// numbers and every product formed as A_hi B_hi + A_hi B_lo + A_lo B_hi
// (Henry, Tang and Heinecke, "Leveraging the bfloat16 artificial intelligence
// datatype for higher-precision computations", 2019), accumulated in FP32 by
// TMA reduce-adds: about 16 significant bits per operand at 3x the
// tensor-core work.
#include "internal.cuh"
#include "tc_gemm2.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace ea {
namespace {
const double kS1 = 0.5 * (1.0 + 1.7320508075688772935);
const double kS2 = 0.5 * (1.0 - 1.7320508075688772935);
const double kI1 = 0.5 * (1.0 + 0.57735026918962576451);
const double kI2 = 0.5 * (1.0 - 0.57735026918962576451);

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }
long long pad8(long long n) { return (n + 7) / 8 * 8; }
// Row pitches of TMA operands are whole 128-byte lines (64 BF16 or 32 FP32
// elements), so that no box row straddles two L2 lines.
long long rp64(long long n) { return (n + 63) / 64 * 64; }
long long rp32(long long n) { return (n + 31) / 32 * 32; }

// BF16 destination (row pitch in elements); lo, when set, receives the low
// part x - bf16(x) at the same position.
struct OpDst {
  bf16* p;
  long long pitch;
  bf16* lo;
};

__device__ __forceinline__ void put(const OpDst& d, long long row, long long col, double x) {
  const bf16 h = __float2bfloat16_rn((float)x);
  d.p[row * d.pitch + col] = h;
  if (d.lo) d.lo[row * d.pitch + col] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
}

// out[r][c] (pitch op) = in[r][c] (pitch ip), c < cols, rows r < rows
__global__ void f64_to_bf16_pitched(const double* __restrict__ in, long long ip, OpDst out, long long rows,
                                    long long cols) {
  long long n = rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long r = i / cols, c = i % cols;
    put(out, r, c, in[r * ip + c]);
  }
}

// Bb[b][Q*dp + d] (pitch bp) = B[Q][b][d]; pad columns d >= v stay zero
__global__ void bmajor_bf16(const double* __restrict__ B, OpDst Bb, int naux, int v, long long dp) {
  long long n = (long long)naux * v * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int d = i % v;
    long long r = i / v;
    int Q = r % naux;
    int b = (int)(r / naux);
    put(Bb, b, (long long)Q * dp + d, B[((long long)Q * v + b) * v + d]);
  }
}

// W[(n,k,d)][e] (pitch in W) = x[n][v + (k,d,e)]
__global__ void pack_w_bf16(const double* __restrict__ x, OpDst W, int nvec, long long dim, int v, long long n2) {
  long long total = n2 * nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    long long n = i / n2, r = i % n2;
    put(W, i / v, i % v, x[n * dim + v + r]);
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
    put(AmT, row, col, am);
    put(AtT, row, col, at);
    put(BmT, row, col, am - 2.0 * at);
    put(V1, row, col, kS1 * wyx + kS2 * wxy);
    put(V2, row, col, kS1 * wxy + kS2 * wyx);
  }
}

// F1[(n,c)][(l,d)] = F_n[l][c][d] into two destinations; G1[(n,b)][(l,d)] = G_n[b][l][d]
__global__ void fg_operands(const float* __restrict__ F, const float* __restrict__ G, OpDst F1a, OpDst F1b,
                            OpDst G1, int nvec, int o, int v) {
  const long long ov = (long long)o * v, n2 = ov * v;
  const long long total = (long long)nvec * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / n2, r = i % n2;
    {  // F_n[l][c][d], stored F[l][n][c][d]
      const int d = r % v, c = (r / v) % v, l = (int)(r / ((long long)v * v));
      const long long row = n * v + c, col = (long long)l * v + d;
      const float f = F[(((long long)l * nvec + n) * v + c) * v + d];
      put(F1a, row, col, (double)f);
      put(F1b, row, col, (double)f);
    }
    {  // G_n[b][l][d], stored G[b][n][l][d]
      const int d = r % v, l = (r / v) % o, b = (int)(r / ov);
      put(G1, n * v + b, (long long)l * v + d, (double)G[(((long long)b * nvec + n) * o + l) * v + d]);
    }
  }
}

// FP32 per-vector H tensors for the coupling pieces, from the tensor-core
// outputs (rows (l,d), columns (n,x)):
//   h1[n][l][c][d] = H1[(l,d)][(n,c)]   (that is H1_n[l][d][c])
//   h2[n][b][l][d] = H23[(l,d)][(n,b)]        h3[n][l][b][d] = H23[ov + (l,d)][(n,b)]
__global__ void h_from_tc(const float* __restrict__ H1, const float* __restrict__ H23, float* __restrict__ h1,
                          float* __restrict__ h2, float* __restrict__ h3, int nvec, int o, int v, long long nv) {
  const long long ov = (long long)o * v, n2 = ov * v;
  const long long total = (long long)nvec * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / n2, r = i % n2;
    const int t = r % v, q = (r / v) % v, p = (int)(r / ((long long)v * v));
    h1[i] = H1[((long long)p * v + t) * nv + n * v + q];         // h1[n][l][c][d]: l=p, c=q, d=t
    h3[i] = H23[(ov + (long long)p * v + t) * nv + n * v + q];  // h3[n][l][b][d]: l=p, b=q, d=t
    const long long b = r / ov, l = (r / v) % o, d = r % v;
    h2[i] = H23[(l * v + d) * nv + n * v + b];
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
    const double t = tau[i];
    const double m2 = t - 2.0 * tau[(((long long)l * o + k) * v + y) * v + xx];
    const long long ly = (long long)l * v + y, kx = (long long)k * v + xx, lx = (long long)l * v + xx,
                    ky = (long long)k * v + y;
    put(tA, ly, kx, t);
    put(tC, kx, ly, t);
    put(tB, lx, ky, t);
    put(tD, ky, lx, t);
    put(m2A, ly, kx, m2);
    put(m2C, kx, ly, m2);
  }
}

__global__ void zero_int(int* p) { *p = 0; }

__global__ void f64_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// y[v + (k,b,c)] += kS1 * A[k][b][c] + kS2 * A[k][c][b]   (S map of an A-representation block)
__global__ void add_S_f32(const float* __restrict__ A, double* __restrict__ y, int o, int v) {
  const long long vv = (long long)v * v, total = (long long)o * vv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / vv, r = i % vv;
    const int b = r / v, c = r % v;
    y[v + i] += kS1 * (double)A[i] + kS2 * (double)A[k * vv + (long long)c * v + b];
  }
}

// hi/lo BF16 split of an FP32 array
__global__ void split_f32(const float* __restrict__ in, bf16* __restrict__ hi, bf16* __restrict__ lo, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float x = in[i];
    const bf16 h = __float2bfloat16_rn(x);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// Yt[a][n] = x[n][a] for the 1p parts (a < v)
__global__ void gather_1p(const float* __restrict__ x, long long dim, int v, int nvec, float* __restrict__ Yt) {
  const int total = v * nvec;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
    Yt[i] = x[(long long)(i % nvec) * dim + i / nvec];
}

// y[n][a] += sy[a][n]
__global__ void add_1p_T(const float* __restrict__ sy, double* __restrict__ y, long long dim, int v, int nvec) {
  const int total = v * nvec;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
    y[(long long)(i % nvec) * dim + i / nvec] += (double)sy[i];
}

// BF16 operands of a state (and their low parts when x3): B^Q in [Q][c][e] and
// b-major [b][(Q,d)] layouts, and the concatenated (ov x ov) ring/coupling
// matrices T1: [K | tauC], T2: [J | K | tm2C | tauD], H1: tauA, H2/H3: [tm2A ; tauB].
void convert_state_operands(cudaStream_t s, State& st, bool lo) {
  const int o = st.o, v = st.v, naux = st.naux;
  const long long vv = (long long)v * v, ov = (long long)o * v;
  const long long vp = pad8(v), ovp = rp64(ov);
  auto L = [&](DArr<bf16>& a) { return lo ? a.p : nullptr; };
  auto zero = [&](DArr<bf16>& a) { EA_CK(cudaMemsetAsync(a.p, 0, a.n * sizeof(bf16), s)); };
  f64_to_bf16_pitched<<<gridn(naux * vv), 256, 0, s>>>(st.Bvv.p, v, OpDst{st.Bvv_bf.p, st.bvv_pitch, L(st.Bvv_lo)},
                                                      (long long)naux * v, v);
  EA_LAUNCH();
  if (vp != v) { zero(st.Bb_bf); if (lo) zero(st.Bb_lo); }
  bmajor_bf16<<<gridn(naux * vv), 256, 0, s>>>(st.Bvv.p, OpDst{st.Bb_bf.p, st.bb_pitch, L(st.Bb_lo)}, naux, v, vp);
  EA_LAUNCH();
  if (st.order < 3) return;
  zero(st.Kmat_bf); zero(st.Jmat_bf); zero(st.tauA_bf); zero(st.tm2A_bf);
  if (lo) { zero(st.Kmat_lo); zero(st.Jmat_lo); zero(st.tauA_lo); zero(st.tm2A_lo); }
  auto off = [&](DArr<bf16>& a, long long o2) { return lo ? a.p + o2 : nullptr; };
  f64_to_bf16_pitched<<<gridn(ov * ov), 256, 0, s>>>(st.Kmat.p, ov, OpDst{st.Kmat_bf.p, 2 * ovp, off(st.Kmat_lo, 0)},
                                                    ov, ov);
  EA_LAUNCH();
  f64_to_bf16_pitched<<<gridn(ov * ov), 256, 0, s>>>(st.Jmat.p, ov, OpDst{st.Jmat_bf.p, 4 * ovp, off(st.Jmat_lo, 0)},
                                                    ov, ov);
  EA_LAUNCH();
  f64_to_bf16_pitched<<<gridn(ov * ov), 256, 0, s>>>(
      st.Kmat.p, ov, OpDst{st.Jmat_bf.p + ovp, 4 * ovp, off(st.Jmat_lo, ovp)}, ov, ov);
  EA_LAUNCH();
  OpDst tA{st.tauA_bf.p, ovp, off(st.tauA_lo, 0)}, tC{st.Kmat_bf.p + ovp, 2 * ovp, off(st.Kmat_lo, ovp)},
      tD{st.Jmat_bf.p + 3 * ovp, 4 * ovp, off(st.Jmat_lo, 3 * ovp)},
      m2C{st.Jmat_bf.p + 2 * ovp, 4 * ovp, off(st.Jmat_lo, 2 * ovp)}, m2A{st.tm2A_bf.p, ovp, off(st.tm2A_lo, 0)},
      tB{st.tm2A_bf.p + ov * ovp, ovp, off(st.tm2A_lo, ov * ovp)};
  tau_operands<<<gridn(ov * ov), 256, 0, s>>>(st.tau.p, tA, tB, tC, tD, m2A, m2C, o, v);
  EA_LAUNCH();
}

void prepare_mixed(cudaStream_t s, State& st, bool x3) {
  const int o = st.o, v = st.v, naux = st.naux;
  const long long ov = (long long)o * v;
  const long long vp = pad8(v), ovp = rp64(ov);
  if (x3 && st.mixed_ready && !st.x3_ready) st.mixed_ready = false;  // redo with low parts
  if (st.mixed_ready) return;
  st.bvv_pitch = rp64(v);
  st.bb_pitch = rp64((long long)naux * vp);
  auto alloc_pair = [&](DArr<bf16>& hi, DArr<bf16>& lo, size_t n) {
    hi.alloc(n, s);
    if (x3) lo.alloc(n, s);
  };
  alloc_pair(st.Bvv_bf, st.Bvv_lo, (size_t)(naux * v * st.bvv_pitch));
  alloc_pair(st.Bb_bf, st.Bb_lo, (size_t)(v * st.bb_pitch));
  if (st.order >= 3) {
    alloc_pair(st.Kmat_bf, st.Kmat_lo, (size_t)(ov * 2 * ovp));
    alloc_pair(st.Jmat_bf, st.Jmat_lo, (size_t)(ov * 4 * ovp));
    alloc_pair(st.tauA_bf, st.tauA_lo, (size_t)(ov * ovp));
    alloc_pair(st.tm2A_bf, st.tm2A_lo, (size_t)(2 * ov * ovp));
  }
  convert_state_operands(s, st, x3);
  st.x3_ready = x3;
  // FP32 copies for the DF coupling pieces (CUDA-core GEMMs)
  st.Boo32.alloc(st.Boo.n, s);
  st.Bov32.alloc(st.Bov.n, s);
  st.Bvv32.alloc(st.Bvv.n, s);
  f64_to_f32<<<gridn(st.Boo.n), 256, 0, s>>>(st.Boo.p, st.Boo32.p, (long long)st.Boo.n);
  EA_LAUNCH();
  f64_to_f32<<<gridn(st.Bov.n), 256, 0, s>>>(st.Bov.p, st.Bov32.p, (long long)st.Bov.n);
  EA_LAUNCH();
  f64_to_f32<<<gridn(st.Bvv.n), 256, 0, s>>>(st.Bvv.p, st.Bvv32.p, (long long)st.Bvv.n);
  EA_LAUNCH();
  if (st.order >= 3) {
    st.tau32.alloc(st.tau.n, s);
    f64_to_f32<<<gridn(st.tau.n), 256, 0, s>>>(st.tau.p, st.tau32.p, (long long)st.tau.n);
    EA_LAUNCH();
  }
  if (!st.err.p) {
    st.err.alloc(1, s);
    zero_int<<<1, 1, 0, s>>>(st.err.p);
    EA_LAUNCH();
  }
  st.mixed_ready = true;
}

// C (=, or += when g.reduce) A B^T; with low parts, the split products
// A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated by TMA reduce-add.
void gemm_split(cudaStream_t s, const TmaMap& Ah, const TmaMap* Al, const TmaMap& Bh, const TmaMap* Bl,
                const TmaMap& C, tc2::Args g) {
  tc_gemm2(s, Ah, Bh, C, g);
  if (Al && Bl) {
    g.reduce = 1;
    tc_gemm2(s, Ah, *Bl, C, g);
    tc_gemm2(s, *Al, Bh, C, g);
  }
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

// DF coupling pieces of all nvec vectors at once (FP32, the vector index n a
// free index of one operand, so every pass over B^Q serves all vectors):
// 1p -> 2p1h: CA[n][k][b][c] = sum_Q (sum_a B^Q_ba y_a) B^Q_kc + the o^3 v^2
// term, and the inputs of the tensor-core o^2 v^3 terms F[l][n][c][d] =
// sum_Q (sum_a B^Q_la y_a) B^Q_cd, G[b][n][l][d] = sum_Q (sum_a B^Q_ba y_a) B^Q_ld.
void couple12_nv(cudaStream_t s, const CoupOps<float>& c, const float* x32, long long dim, int nvec, float* CA,
                 float* F, float* G) {
  const int o = c.o, v = c.v, naux = c.naux;
  using TT = TensT<float>;
  TT Bov{(float*)c.Bov, {naux, o, v}}, Bvv{(float*)c.Bvv, {naux, v, v}}, Boo{(float*)c.Boo, {naux, o, o}};
  DArr<float> Yt((size_t)v * nvec, s), Qy((size_t)naux * v * nvec, s), Qo((size_t)naux * o * nvec, s),
      H((size_t)o * o * o * nvec, s);
  gather_1p<<<gridn((long long)v * nvec), 256, 0, s>>>(x32, dim, v, nvec, Yt.p);
  EA_LAUNCH();
  TT Ytt{Yt.p, {v, nvec}}, Qyt{Qy.p, {naux, v, nvec}}, Qot{Qo.p, {naux, o, nvec}};
  einsumT<float>(s, "Qba,an->Qbn", 1.f, Bvv, Ytt, 0.f, Qyt);  // B^Q symmetric
  einsumT<float>(s, "Qbn,Qkc->nkbc", 1.f, Qyt, Bov, 0.f, TT{CA, {nvec, o, v, v}});
  einsumT<float>(s, "Qla,an->Qln", 1.f, Bov, Ytt, 0.f, Qot);
  einsumT<float>(s, "Qln,Qcd->lncd", 1.f, Qot, Bvv, 0.f, TT{F, {o, nvec, v, v}});
  einsumT<float>(s, "Qbn,Qld->bnld", 1.f, Qyt, Bov, 0.f, TT{G, {v, nvec, o, v}});
  einsumT<float>(s, "Qln,Qkm->lnkm", 1.f, Qot, Boo, 0.f, TT{H.p, {o, nvec, o, o}});
  einsumT<float>(s, "lnkm,lmbc->nkbc", 1.f, TT{H.p, {o, nvec, o, o}}, TT{(float*)c.tau, {o, o, v, v}}, 1.f,
                 TT{CA, {nvec, o, v, v}});
}

// 2p1h -> 1p for all vectors: sy[a][n] from V[n][k][b][c] (the S-transformed
// 2p1h parts) and the tensor-core intermediates h1[n][l][c][d], h2[n][b][l][d],
// h3[n][l][b][d].
void couple21_nv(cudaStream_t s, const CoupOps<float>& c, const float* V, int nvec, const float* h1, const float* h2,
                 const float* h3, float* sy) {
  const int o = c.o, v = c.v, naux = c.naux;
  using TT = TensT<float>;
  TT Bov{(float*)c.Bov, {naux, o, v}}, Bvv{(float*)c.Bvv, {naux, v, v}}, Boo{(float*)c.Boo, {naux, o, o}};
  TT Vt{(float*)V, {nvec, o, v, v}}, syt{sy, {v, nvec}};
  DArr<float> g((size_t)naux * v * nvec, s), tt((size_t)naux * nvec * o, s), t2q((size_t)naux * nvec * v, s),
      H4((size_t)o * o * nvec * o, s);
  TT gt{g.p, {naux, v, nvec}}, ttt{tt.p, {naux, nvec, o}}, t2qt{t2q.p, {naux, nvec, v}};
  einsumT<float>(s, "Qkc,nkbc->Qbn", 1.f, Bov, Vt, 0.f, gt);
  einsumT<float>(s, "Qba,Qbn->an", 1.f, Bvv, gt, 0.f, syt);  // B^Q symmetric
  einsumT<float>(s, "Qcd,nlcd->Qnl", -1.f, Bvv, TT{(float*)h1, {nvec, o, v, v}}, 0.f, ttt);
  einsumT<float>(s, "Qld,nbld->Qnb", 1.f, Bov, TT{(float*)h2, {nvec, v, o, v}}, 0.f, t2qt);
  einsumT<float>(s, "Qba,Qnb->an", -1.f, Bvv, t2qt, 1.f, syt);
  einsumT<float>(s, "Qbd,nlbd->Qnl", -1.f, Bvv, TT{(float*)h3, {nvec, o, v, v}}, 1.f, ttt);
  einsumT<float>(s, "lmbc,nkbc->lmnk", 1.f, TT{(float*)c.tau, {o, o, v, v}}, Vt, 0.f, TT{H4.p, {o, o, nvec, o}});
  einsumT<float>(s, "Qkm,lmnk->Qnl", 1.f, Boo, TT{H4.p, {o, o, nvec, o}}, 1.f, ttt);
  einsumT<float>(s, "Qla,Qnl->an", 1.f, Bov, ttt, 1.f, syt);
}

// W[(m,c)][d] (pitch in W) = T[m][c][d], hi/lo BF16 split when W.lo
__global__ void pack_mats_bf16(const double* __restrict__ T, OpDst W, long long total, int v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    put(W, i / v, i % v, T[i]);
}

// out[m][b][c] = L[(m,c)][b] (row pitch lp): the ladder output is transposed
__global__ void unpack_ladder(const float* __restrict__ L, long long lp, double* __restrict__ out, long long total,
                              int v) {
  const long long vv = (long long)v * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long m = i / vv, b = (i / v) % v, c = i % v;
    out[i] = (double)L[(m * v + c) * lp + b];
  }
}

// compact out[r][c] (pitch v) = in[r][c] (pitch ip)
__global__ void compact_f32(const float* __restrict__ in, long long ip, float* __restrict__ out, long long rows, int v) {
  long long n = rows * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[(i / v) * ip + i % v];
}
}  // namespace

// Transposed ladder out[(nk,c)][b] (row pitch op, FP32) = (sum_Q B^Q W_nk B^Q)[b][c]
// for nmat pair matrices W (bf16, rows (nk,d), columns e, row pitch rp64(v); Wl
// its low part in split mode).
//   stage 1 (batch Q x nk): Z[nk][c][Q][d] = sum_e B^Q[c][e] W_nk[d][e]
//   stage 2 (one GEMM):     out[(nk,c)][b] (+)= sum_(Q,d) Z[(nk,c)][(Q,d)] B^Q[b][d]
// Z rows hold qc blocks of pad8(v) columns (pads zero, matching the zero pads
// of the b-major copy of B); chunks accumulate by TMA reduce-add.  In split
// mode Z is formed in FP32 by the three split products and split again.
// ladder_run computes it in chunks of qc auxiliary functions.
struct LadderPlan {
  int qc;      // auxiliary functions per chunk
  int var1;    // tc_gemm2 pipeline variant of stage 1 (0: by K)
  int var2;    // ... of stage 2
};
static void ladder_run(cudaStream_t s, State& st, const bf16* Wbf, const bf16* Wlo, int nmat, float* out, long long op,
                       const LadderPlan& plan);

// Ladder plan (chunk size and the GEMM pipeline shape of each stage), tuned
// once per shape: the intermediate Z of one chunk should stay in L2 between
// the two stages, but larger chunks mean fewer launches and longer GEMMs;
// short-K stage 1 and long-K stage 2 want different load / epilogue depths.
// The first call for a (v, naux, nmat, split) shape times the candidate
// chunk sizes (Z of 12, 24, 48 and 96 M elements) with the default pipelines,
// then the pipeline variants of each stage at the best chunk size, with CUDA
// events on the stream (every run producing the full ladder in out), and
// keeps the fastest plan.
void ladder_tc(cudaStream_t s, State& st, const bf16* Wbf, const bf16* Wlo, int nmat, float* out, long long op,
               bool tune = true);
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, bool>, LadderPlan> g_ladder_plan;

void ladder_tc(cudaStream_t s, State& st, const bf16* Wbf, const bf16* Wlo, int nmat, float* out, long long op,
               bool tune) {
  const int v = st.v, naux = st.naux;
  const bool x3 = Wlo != nullptr;
  const long long per_q = std::max<long long>(1, (long long)nmat * v * pad8(v));
  auto qc_of = [&](long long budget) { return (int)std::min<long long>(naux, std::max<long long>(1, budget / per_q)); };
  if (!tune) {  // one-off use: the default plan (Z about 48 M elements, split mode 24 M)
    ladder_run(s, st, Wbf, Wlo, nmat, out, op, LadderPlan{qc_of(x3 ? 24LL << 20 : 48LL << 20), 0, 0});
    return;
  }
  const auto key = std::make_tuple(v, naux, nmat, x3);
  LadderPlan plan{-1, 0, 0};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_ladder_plan.find(key);
    if (it != g_ladder_plan.end()) plan = it->second;
  }
  if (plan.qc < 0) {
    std::vector<int> cand;
    for (long long b : {12LL << 20, 24LL << 20, 48LL << 20, 96LL << 20}) {
      const int q = qc_of(x3 ? b / 2 : b);
      if (std::find(cand.begin(), cand.end(), q) == cand.end()) cand.push_back(q);
    }
    plan = LadderPlan{cand.back(), 0, 0};
    if (cand.size() > 1) {
      cudaEvent_t e0, e1;
      EA_CK(cudaEventCreate(&e0));
      EA_CK(cudaEventCreate(&e1));
      auto time_plan = [&](const LadderPlan& p) {
        ladder_run(s, st, Wbf, Wlo, nmat, out, op, p);  // warm-up (and the allocation of Z)
        EA_CK(cudaEventRecord(e0, s));
        ladder_run(s, st, Wbf, Wlo, nmat, out, op, p);
        EA_CK(cudaEventRecord(e1, s));
        EA_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        EA_CK(cudaEventElapsedTime(&ms, e0, e1));
        return ms;
      };
      float best = 1e30f;
      for (int q : cand) {
        const float ms = time_plan(LadderPlan{q, 0, 0});
        if (ms < best) { best = ms; plan = LadderPlan{q, 0, 0}; }
      }
      const bool fits43 = tc2::smem_bytes(pick_bn(v), 4, 3) <= 232448;
      for (int v1 : {1, 2, 3})
        for (int v2 : {1, 2, 3}) {
          if (!fits43 && (v1 == 3 || v2 == 3)) continue;
          const LadderPlan p{plan.qc, v1, v2};
          const float ms = time_plan(p);
          if (ms < best) { best = ms; plan = p; }
        }
      EA_CK(cudaEventDestroy(e0));
      EA_CK(cudaEventDestroy(e1));
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_ladder_plan[key] = plan;
  }
  ladder_run(s, st, Wbf, Wlo, nmat, out, op, plan);
}

static void ladder_run(cudaStream_t s, State& st, const bf16* Wbf, const bf16* Wlo, int nmat, float* out, long long op,
                       const LadderPlan& plan) {
  const int v = st.v, naux = st.naux, qc = plan.qc;
  const bool x3 = Wlo != nullptr;
  const long long dp = pad8(v), wp = rp64(v), bk = (long long)naux * dp;
  const long long bvp = st.bvv_pitch, bbp = st.bb_pitch;
  const long long zp = rp64((long long)qc * dp);  // Z row pitch
  const size_t zn = (size_t)nmat * v * zp;
  DArr<bf16> Z(zn, s), Zl;
  DArr<float> Z32;
  if (x3) {
    Zl.alloc(zn, s);
    Z32.alloc(zn, s);
    if (dp != v) EA_CK(cudaMemsetAsync(Z32.p, 0, zn * sizeof(float), s));
  } else if (dp != v) {
    EA_CK(cudaMemsetAsync(Z.p, 0, zn * sizeof(bf16), s));
  }
  const int bn = pick_bn(v);
  TmaMap mB3 = make_tma_3d(st.Bvv_bf.p, v, v, naux, bvp, v * bvp, 128);  // stage-1 A: [Q][c][e]
  TmaMap mW = make_tma_3d(Wbf, v, v, nmat, wp, (long long)v * wp, bn);   // stage-1 B: [nk][d][e]
  TmaMap mBb = make_tma_3d(st.Bb_bf.p, bk, v, 1, bbp, bbp * v, bn);      // stage-2 B: [b][(Q,d)]
  TmaMap mB3l, mWl, mBbl;
  if (x3) {
    mB3l = make_tma_3d(st.Bvv_lo.p, v, v, naux, bvp, v * bvp, 128);
    mWl = make_tma_3d(Wlo, v, v, nmat, wp, (long long)v * wp, bn);
    mBbl = make_tma_3d(st.Bb_lo.p, bk, v, 1, bbp, bbp * v, bn);
  }
  TmaMap mOut = make_tma_out4d(out, 4, v, 1, (long long)nmat * v, 1, op, op, (long long)nmat * v * op);
  for (int Q0 = 0; Q0 < naux; Q0 += qc) {
    const int q = std::min(qc, naux - Q0);
    tc2::Args g1 = gargs(v, v, v, st.err.p);
    g1.nzlo = q; g1.nz = q * nmat;
    g1.a_sel = tc2::Z_LO; g1.a_z0 = Q0;
    g1.b_sel = tc2::Z_HI;
    g1.variant = plan.var1;
    if (!x3) {
      TmaMap mZo = make_tma_out4d(Z.p, 2, v, q, v, nmat, dp, zp, (long long)v * zp);
      g1.out_bf16 = 1;
      tc_gemm2(s, mB3, mW, mZo, g1);
    } else {
      TmaMap mZo = make_tma_out4d(Z32.p, 4, v, q, v, nmat, dp, zp, (long long)v * zp);
      gemm_split(s, mB3, &mB3l, mW, &mWl, mZo, g1);
      split_f32<<<gridn((long long)zn), 256, 0, s>>>(Z32.p, Z.p, Zl.p, (long long)zn);
      EA_LAUNCH();
    }
    // K extent of this chunk exactly q*dp: columns past it read as zero
    TmaMap mZ = make_tma_3d(Z.p, (long long)q * dp, (long long)nmat * v, 1, zp, (long long)nmat * v * zp, 128);
    tc2::Args g2 = gargs(nmat * v, v, (int)(q * dp), st.err.p);
    g2.b_k0 = (int)(Q0 * dp);
    g2.reduce = (Q0 > 0);
    g2.variant = plan.var2;
    if (!x3) {
      tc_gemm2(s, mZ, mBb, mOut, g2);
    } else {
      TmaMap mZl = make_tma_3d(Zl.p, (long long)q * dp, (long long)nmat * v, 1, zp, (long long)nmat * v * zp, 128);
      gemm_split(s, mZ, &mZl, mBb, &mBbl, mOut, g2);
    }
  }
}

void ladder_pairs_tc(cudaStream_t s, State& st, const double* T, int nmat, bool x3, double* out) {
  const int v = st.v;
  const long long wp = rp64(v), lp = rp32(v), total = (long long)nmat * v * v;
  prepare_mixed(s, st, x3);
  DArr<bf16> W((size_t)(nmat * v * wp), s), Wl;
  if (x3) Wl.alloc(W.n, s);
  pack_mats_bf16<<<gridn(total), 256, 0, s>>>(T, OpDst{W.p, wp, x3 ? Wl.p : nullptr}, total, v);
  EA_LAUNCH();
  DArr<float> L((size_t)(nmat * v * lp), s);
  ladder_tc(s, st, W.p, x3 ? Wl.p : nullptr, nmat, L.p, lp, false);
  unpack_ladder<<<gridn(total), 256, 0, s>>>(L.p, lp, out, total, v);
  EA_LAUNCH();
}

void sigma_mixed(cudaStream_t s, State& st, int nvec, const double* x, double* y, bool x3) {
  if (st.order < 3) {  // ADC(2): first-order coupling and diagonal only, no tensor-core terms
    sigma_base_fp64(s, st, nvec, x, y, false, false);
    return;
  }
  prepare_mixed(s, st, x3);
  const int o = st.o, v = st.v;
  const long long vv = (long long)v * v, ov = (long long)o * v, n2 = ov * v, dim = st.dim;
  const long long wp = rp64(v), lp = rp32(v), ovp = rp64(ov), nv = (long long)nvec * v;
  // FP64: orbital-energy diagonal and 1p/1p block; FP32 (CUDA cores): the DF
  // coupling pieces (first-order coupling, the o^3 v^2 term, F and G)
  diag_and_m11(s, st, nvec, x, y);
  const CoupOps<float> ops{o, v, st.naux, st.order, st.Boo32.p, st.Bov32.p, st.Bvv32.p, st.tau32.p};
  DArr<float> x32((size_t)(nvec * dim), s);
  f64_to_f32<<<gridn(nvec * dim), 256, 0, s>>>(x, x32.p, nvec * dim);
  EA_LAUNCH();
  DArr<float> F((size_t)(nvec * n2), s), G((size_t)(nvec * n2), s), CA((size_t)(nvec * n2), s);
  couple12_nv(s, ops, x32.p, dim, nvec, CA.p, F.p, G.p);
  for (int n = 0; n < nvec; ++n) {
    add_S_f32<<<gridn(n2), 256, 0, s>>>(CA.p + n * n2, y + n * dim, o, v);
    EA_LAUNCH();
  }
  // BF16 operands (and low parts in split mode)
  DArr<bf16> Wbf((size_t)(ov * nvec * wp), s), Wlo;
  if (x3) Wlo.alloc(Wbf.n, s);
  pack_w_bf16<<<gridn(n2 * nvec), 256, 0, s>>>(x, OpDst{Wbf.p, wp, x3 ? Wlo.p : nullptr}, nvec, dim, v, n2);
  EA_LAUNCH();
  DArr<bf16> B1((size_t)(nv * 2 * ovp), s), B2((size_t)(nv * 4 * ovp), s), BV1((size_t)(nv * ovp), s),
      BV2((size_t)(nv * ovp), s), B1l, B2l, BV1l, BV2l;
  if (x3) { B1l.alloc(B1.n, s); B2l.alloc(B2.n, s); BV1l.alloc(BV1.n, s); BV2l.alloc(BV2.n, s); }
  if (ovp != ov) {
    for (DArr<bf16>* a : {&B1, &B2, &B1l, &B2l})
      if (a->p) EA_CK(cudaMemsetAsync(a->p, 0, a->n * sizeof(bf16), s));
  }
  auto lo = [&](DArr<bf16>& a, long long o2) { return x3 ? a.p + o2 : nullptr; };
  // B1 = [AmT | F1], B2 = [BmT | AtT | G1 | F1]
  ring_operands<<<gridn(nv * ov), 256, 0, s>>>(
      x, OpDst{B1.p, 2 * ovp, lo(B1l, 0)}, OpDst{B2.p, 4 * ovp, lo(B2l, 0)}, OpDst{B2.p + ovp, 4 * ovp, lo(B2l, ovp)},
      OpDst{BV1.p, ovp, lo(BV1l, 0)}, OpDst{BV2.p, ovp, lo(BV2l, 0)}, nvec, dim, o, v);
  EA_LAUNCH();
  fg_operands<<<gridn(nvec * n2), 256, 0, s>>>(F.p, G.p, OpDst{B1.p + ovp, 2 * ovp, lo(B1l, ovp)},
                                               OpDst{B2.p + 3 * ovp, 4 * ovp, lo(B2l, 3 * ovp)},
                                               OpDst{B2.p + 2 * ovp, 4 * ovp, lo(B2l, 2 * ovp)}, nvec, o, v);
  EA_LAUNCH();
  // tensor-core GEMMs
  DArr<float> L((size_t)(ov * nvec * lp), s);
  ladder_tc(s, st, Wbf.p, x3 ? Wlo.p : nullptr, nvec * o, L.p, lp);
  const long long nvp = rp32(nv);
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
  TmaMap aT1l, aT2l, aH1l, aH23l, bT1l, bT2l, bV1l, bV2l;
  if (x3) {
    aT1l = make_tma_3d(st.Kmat_lo.p, 2 * ovp, ov, 1, 2 * ovp, ov * 2 * ovp, 128);
    aT2l = make_tma_3d(st.Jmat_lo.p, 4 * ovp, ov, 1, 4 * ovp, ov * 4 * ovp, 128);
    aH1l = make_tma_3d(st.tauA_lo.p, ov, ov, 1, ovp, ov * ovp, 128);
    aH23l = make_tma_3d(st.tm2A_lo.p, ov, 2 * ov, 1, ovp, 2 * ov * ovp, 128);
    bT1l = make_tma_3d(B1l.p, 2 * ovp, nv, 1, 2 * ovp, nv * 2 * ovp, bnn);
    bT2l = make_tma_3d(B2l.p, 4 * ovp, nv, 1, 4 * ovp, nv * 4 * ovp, bnn);
    bV1l = make_tma_3d(BV1l.p, ov, nv, 1, ovp, nv * ovp, bnn);
    bV2l = make_tma_3d(BV2l.p, ov, nv, 1, ovp, nv * ovp, bnn);
  }
  auto P = [&](TmaMap& m) { return x3 ? &m : nullptr; };
  auto outmap = [&](float* p, long long rows) { return make_tma_out4d(p, 4, nv, 1, rows, 1, nvp, nvp, rows * nvp); };
  tc2::Args g = gargs((int)ov, (int)nv, (int)(2 * ovp), st.err.p);
  gemm_split(s, aT1, P(aT1l), bT1, P(bT1l), outmap(T1.p, ov), g);
  g.K = (int)(4 * ovp);
  gemm_split(s, aT2, P(aT2l), bT2, P(bT2l), outmap(T2.p, ov), g);
  g.K = (int)ov;
  gemm_split(s, aH1, P(aH1l), bV1, P(bV1l), outmap(H1.p, ov), g);
  g.M = (int)(2 * ov);
  gemm_split(s, aH23, P(aH23l), bV2, P(bV2l), outmap(H23.p, 2 * ov), g);
  combine_ring_ladder<<<gridn(n2 * nvec), 256, 0, s>>>(y, T1.p, T2.p, L.p, nvec, dim, o, v, nvp, lp);
  EA_LAUNCH();
  // 2p1h -> 1p finishing (FP32, CUDA cores) from the tensor-core H tensors
  DArr<float> h1((size_t)(nvec * n2), s), h2((size_t)(nvec * n2), s), h3((size_t)(nvec * n2), s),
      V((size_t)(nvec * n2), s), sy((size_t)v * nvec, s);
  h_from_tc<<<gridn(nvec * n2), 256, 0, s>>>(H1.p, H23.p, h1.p, h2.p, h3.p, nvec, o, v, nvp);
  EA_LAUNCH();
  for (int n = 0; n < nvec; ++n)
    pair_combineT<float>(s, x32.p + n * dim + v, vv, V.p + n * n2, vv, o, v, (float)kS1, (float)kS2, 1.f, 0.f);
  couple21_nv(s, ops, V.p, nvec, h1.p, h2.p, h3.p, sy.p);
  add_1p_T<<<gridn((long long)v * nvec), 256, 0, s>>>(sy.p, y, dim, v, nvec);
  EA_LAUNCH();
}

// Ladder alone, transposed FP32 output [nvec][o][c][b] (= ladder[b][c]), for timing the dominant kernel.
void ladder_only(cudaStream_t s, State& st, int nvec, const double* x, float* out, bool mixed) {
  const int o = st.o, v = st.v;
  const long long ov = (long long)o * v, n2 = ov * v;
  if (!mixed) fail(EAADC_ERR_ARG, "ladder_only: tensor-core path only");
  prepare_mixed(s, st, st.x3_ready);
  const long long wp = rp64(v), lp = rp32(v);
  DArr<bf16> Wbf((size_t)(ov * nvec * wp), s);
  pack_w_bf16<<<gridn(n2 * nvec), 256, 0, s>>>(x, OpDst{Wbf.p, wp, nullptr}, nvec, st.dim, v, n2);
  EA_LAUNCH();
  if (v % 4 == 0) {  // rows of the caller's buffer are whole 16-byte units: write in place
    ladder_tc(s, st, Wbf.p, nullptr, nvec * o, out, v);
  } else {
    DArr<float> L((size_t)(ov * nvec * lp), s);
    ladder_tc(s, st, Wbf.p, nullptr, nvec * o, L.p, lp);
    compact_f32<<<gridn(n2 * nvec), 256, 0, s>>>(L.p, lp, out, ov * nvec, v);
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
