// Dense FP64 symmetric eigensolver for the per-state FNO and NAF bases
// (Eq. 9, 13 and 28 need the full spectra of the v x v virtual density, the
// semicanonical Fock block and the naux x naux auxiliary metric).
//
// Two-sided block Jacobi: the order-n matrix is cut into nb blocks of 32
// rows and columns (nb even; the last block padded with decoupled diagonal
// entries larger than every eigenvalue).  A sweep visits every block pair once
// in nb-1 rounds of a round-robin tournament; in a round the nb/2 disjoint
// 64 x 64 pair sub-matrices are diagonalised exactly by the in-shared-memory
// Jacobi kernel (one CTA each) and their rotations R applied as
// A <- R^T A R on the pair's rows and columns and V <- V R.  Sweeps stop when
// the off-diagonal mass falls below 1e-28 of the total.  Eigenvalues are then
// ranked on the device and the eigenvectors gathered in ascending order.
#include "internal.cuh"

#include <algorithm>
#include <cmath>

namespace ea {
namespace {

constexpr int kB = 32;       // block order
constexpr int kP = 2 * kB;   // pair sub-matrix order
constexpr int kRows = 16;    // rows (or columns) per CTA in the rotation kernels

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

// Round-robin pairing of nb players (nb even): player 0 fixed, others rotate.
__device__ __forceinline__ void pair_of(int i, int round, int nb, int& p, int& q) {
  const int a = (i == 0) ? 0 : 1 + (i - 1 + round) % (nb - 1);
  const int j = nb - 1 - i;
  const int b = 1 + (j - 1 + round) % (nb - 1);
  p = min(a, b);
  q = max(a, b);
}

__device__ __forceinline__ int pair_index(int k, int p, int q) { return k < kB ? p * kB + k : q * kB + (k - kB); }

// Ap [np][np] = A (n x n) with decoupled padding diagonal pad + i; V = I.
__global__ void pad_init(const double* __restrict__ A, int n, double* __restrict__ Ap, double* __restrict__ V, int np,
                         double pad) {
  const long long total = (long long)np * np;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / np), c = (int)(e % np);
    double a = 0.0;
    if (r < n && c < n) a = 0.5 * (A[(long long)r * n + c] + A[(long long)c * n + r]);
    else if (r == c) a = pad + r;
    Ap[e] = a;
    V[e] = (r == c) ? 1.0 : 0.0;
  }
}

// Sum of squares of A split into diagonal / off-diagonal, per-CTA partials.
__global__ void mass_partial(const double* __restrict__ A, int np, double* __restrict__ part) {
  __shared__ double so[32], sd[32];
  double off = 0.0, dg = 0.0;
  const long long total = (long long)np * np;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const double a = A[e];
    if (e / np == e % np) dg += a * a; else off += a * a;
  }
  for (int o = 16; o; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    dg += __shfl_xor_sync(0xffffffffu, dg, o);
  }
  if ((threadIdx.x & 31) == 0) { so[threadIdx.x >> 5] = off; sd[threadIdx.x >> 5] = dg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { a += so[i]; b += sd[i]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void mass_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nparts; ++i) { a += part[2 * i]; b += part[2 * i + 1]; }
    out[0] = a;
    out[1] = b;
  }
}

// S[i] = A restricted to the rows and columns of pair i (64 x 64).
__global__ void gather_pairs(const double* __restrict__ A, int np, int nb, int round, double* __restrict__ S) {
  const int i = blockIdx.y;
  int p, q;
  pair_of(i, round, nb, p, q);
  double* Si = S + (size_t)i * kP * kP;
  for (int e = threadIdx.x; e < kP * kP; e += blockDim.x) {
    const int r = e / kP, c = e % kP;
    Si[e] = A[(long long)pair_index(r, p, q) * np + pair_index(c, p, q)];
  }
}

// X[r][pair cols] <- X[r][pair cols] R_i for kRows rows per CTA (X: A or V).
__global__ void rotate_cols(double* __restrict__ X, int np, int nb, int round, const double* __restrict__ R) {
  __shared__ double Rs[kP][kP + 1];
  __shared__ double Xs[kRows][kP + 1];
  const int i = blockIdx.y, r0 = blockIdx.x * kRows;
  int p, q;
  pair_of(i, round, nb, p, q);
  const double* Ri = R + (size_t)i * kP * kP;
  for (int e = threadIdx.x; e < kP * kP; e += blockDim.x) Rs[e / kP][e % kP] = Ri[e];
  for (int e = threadIdx.x; e < kRows * kP; e += blockDim.x) {
    const int r = e / kP, k = e % kP;
    Xs[r][k] = (r0 + r < np) ? X[(long long)(r0 + r) * np + pair_index(k, p, q)] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kRows * kP; e += blockDim.x) {
    const int r = e / kP, c = e % kP;
    if (r0 + r >= np) continue;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < kP; ++k) acc += Xs[r][k] * Rs[k][c];
    X[(long long)(r0 + r) * np + pair_index(c, p, q)] = acc;
  }
}

// A[pair rows][c] <- R_i^T A[pair rows][c] for kRows columns per CTA.
__global__ void rotate_rows(double* __restrict__ A, int np, int nb, int round, const double* __restrict__ R) {
  __shared__ double Rs[kP][kP + 1];
  __shared__ double As[kP][kRows + 1];
  const int i = blockIdx.y, c0 = blockIdx.x * kRows;
  int p, q;
  pair_of(i, round, nb, p, q);
  const double* Ri = R + (size_t)i * kP * kP;
  for (int e = threadIdx.x; e < kP * kP; e += blockDim.x) Rs[e / kP][e % kP] = Ri[e];
  for (int e = threadIdx.x; e < kP * kRows; e += blockDim.x) {
    const int k = e / kRows, c = e % kRows;
    As[k][c] = (c0 + c < np) ? A[(long long)pair_index(k, p, q) * np + c0 + c] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kP * kRows; e += blockDim.x) {
    const int r = e / kRows, c = e % kRows;
    if (c0 + c >= np) continue;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < kP; ++k) acc += Rs[k][r] * As[k][c];
    A[(long long)pair_index(r, p, q) * np + c0 + c] = acc;
  }
}

// Rank the diagonal ascending (ties by index) and gather the first n
// eigenpairs: w[rank] = A[j][j], V[r][rank] = Vp[r][j] (r < n).
__global__ void rank_gather(const double* __restrict__ Ap, const double* __restrict__ Vp, int np, int n,
                            double* __restrict__ w, double* __restrict__ V) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += gridDim.x * blockDim.x) {
    const double dj = Ap[(long long)j * np + j];
    int rank = 0;
    for (int k = 0; k < np; ++k) {
      const double dk = Ap[(long long)k * np + k];
      rank += (dk < dj) || (dk == dj && k < j);
    }
    if (rank >= n) continue;
    w[rank] = dj;
    for (int r = 0; r < n; ++r) V[(long long)r * n + rank] = Vp[(long long)r * np + j];
  }
}

__global__ void frob_partial(const double* __restrict__ A, long long total, double* __restrict__ part) {
  __shared__ double sh[32];
  double t = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    t += A[e] * A[e];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) a += sh[i];
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

}  // namespace

void eigh_sym(cudaStream_t s, int n, const double* A, double* w, double* V) {
  if (n <= 0) return;
  if (n <= 96) {
    jacobi_eigh(s, n, const_cast<double*>(A), w, V, 1);
    return;
  }
  int nb = (n + kB - 1) / kB;
  nb += nb & 1;
  const int np = nb * kB, npairs = nb / 2;
  const int nparts = 128;
  DArr<double> Ap((size_t)np * np, s), Vp((size_t)np * np, s), S((size_t)npairs * kP * kP, s),
      R((size_t)npairs * kP * kP, s), wv((size_t)npairs * kP, s), part((size_t)2 * nparts, s), mass(2, s);
  // padding above every eigenvalue: |lambda| <= ||A||_F
  double h[2] = {0.0, 0.0};
  frob_partial<<<nparts, 256, 0, s>>>(A, (long long)n * n, part.p);
  EA_LAUNCH();
  mass_final<<<1, 32, 0, s>>>(part.p, nparts, mass.p);
  EA_LAUNCH();
  EA_CK(cudaMemcpyAsync(h, mass.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  EA_CK(cudaStreamSynchronize(s));
  const double pad = 2.0 * std::sqrt(h[0]) + 1.0;
  pad_init<<<gridn((long long)np * np), 256, 0, s>>>(A, n, Ap.p, Vp.p, np, pad);
  EA_LAUNCH();
  const dim3 gc((np + kRows - 1) / kRows, npairs);
  for (int sweep = 0; sweep < 40; ++sweep) {
    mass_partial<<<nparts, 256, 0, s>>>(Ap.p, np, part.p);
    EA_LAUNCH();
    mass_final<<<1, 32, 0, s>>>(part.p, nparts, mass.p);
    EA_LAUNCH();
    EA_CK(cudaMemcpyAsync(h, mass.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    EA_CK(cudaStreamSynchronize(s));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) fail(EAADC_ERR_NONFINITE, "eigh_sym: non-finite matrix");
    if (h[0] <= 1e-28 * (h[0] + h[1]) || h[0] < 1e-300) break;
    if (sweep == 39) fail(EAADC_ERR_NOCONV, "eigh_sym: block Jacobi did not converge in 40 sweeps");
    for (int round = 0; round < nb - 1; ++round) {
      gather_pairs<<<dim3(1, npairs), 256, 0, s>>>(Ap.p, np, nb, round, S.p);
      EA_LAUNCH();
      jacobi_eigh(s, kP, S.p, wv.p, R.p, npairs);
      rotate_cols<<<gc, 256, 0, s>>>(Ap.p, np, nb, round, R.p);
      EA_LAUNCH();
      rotate_rows<<<gc, 256, 0, s>>>(Ap.p, np, nb, round, R.p);
      EA_LAUNCH();
      rotate_cols<<<gc, 256, 0, s>>>(Vp.p, np, nb, round, R.p);
      EA_LAUNCH();
    }
  }
  rank_gather<<<(np + 127) / 128, 128, 0, s>>>(Ap.p, Vp.p, np, n, w, V);
  EA_LAUNCH();
}

}  // namespace ea
