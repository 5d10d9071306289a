// Block Davidson eigensolver on the device (Sec. II.A: M is diagonalised by
// Davidson's method from sigma vectors).  All vector arithmetic is FP64 and
// runs in this library's kernels; per iteration only the Ritz values, the
// residual norms and the number of accepted new directions (a few doubles)
// are read back to decide convergence.
//
// Readings (unstated in the paper): guesses are unit vectors on the nroots
// lowest diagonal entries; the correction is r / (theta - D) with
// |theta - D| floored at 1e-8; corrections are normalised, projected out of
// the subspace twice (classical Gram-Schmidt) and then orthonormalised among
// themselves by canonical orthogonalisation (eigenvectors of their Gram
// matrix, directions with eigenvalue <= 1e-18 dropped); the subspace restarts
// from the 2*nroots lowest Ritz vectors when it would exceed max_sub.
//
// Options: a reduced-precision sigma (the phase also stops at its noise
// floor) followed by FP64 iterations or by one sigma-and-Ritz step in FP64 or
// split BF16; the learned correction of precond.cu with a per-root fallback
// to the diagonal one; a trace of the first iterates (training pairs).
// Subspace updates and Gram products are bandwidth-bound kernels that read
// each basis vector once per call.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ea {
namespace {

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

// partial min over a range, excluding listed indices
__global__ void argmin_partial(const double* __restrict__ D, long long n, const int* __restrict__ excl, int nexcl,
                               double* __restrict__ pv, long long* __restrict__ pi) {
  double best = INFINITY;
  long long bi = -1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    bool skip = false;
    for (int e = 0; e < nexcl; ++e) skip |= (excl[e] == i);
    if (skip) continue;
    double d = D[i];
    if (d < best || (d == best && i < bi)) { best = d; bi = i; }
  }
  __shared__ double sv[256];
  __shared__ long long si[256];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) {
      double v2 = sv[threadIdx.x + o];
      long long i2 = si[threadIdx.x + o];
      if (i2 >= 0 && (si[threadIdx.x] < 0 || v2 < sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x]))) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { pv[blockIdx.x] = sv[0]; pi[blockIdx.x] = si[0]; }
}

__global__ void argmin_final(const double* __restrict__ pv, const long long* __restrict__ pi, int np, int* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double best = INFINITY;
  long long bi = -1;
  for (int i = 0; i < np; ++i)
    if (pi[i] >= 0 && (bi < 0 || pv[i] < best || (pv[i] == best && pi[i] < bi))) { best = pv[i]; bi = pi[i]; }
  *out = (int)bi;
}

__global__ void set_units(double* __restrict__ V, long long n, const int* __restrict__ idx, int k) {
  long long total = n * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / n);
    long long i = t % n;
    V[t] = (i == idx[r]) ? 1.0 : 0.0;
  }
}

// C[z][i][j] partial dot products are reduced here: C = sum_z P[z]
__global__ void reduce_partials(const double* __restrict__ P, int nz, int count, double* __restrict__ C, int ma,
                                int mb, long long ldc) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += P[(long long)z * count + e];
    C[(long long)(e / mb) * ldc + (e % mb)] = s;
  }
}

__global__ void symmetrize(double* __restrict__ G, int m, long long ld, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    int i = e / m, j = e % m;
    out[e] = 0.5 * (G[i * ld + j] + G[j * ld + i]);
  }
}

// R = SX - theta X, partial squared norms per (row, block)
__global__ void residual_kernel(const double* __restrict__ SX, const double* __restrict__ X,
                                const double* __restrict__ theta, double* __restrict__ R, long long n, int k,
                                double* __restrict__ part) {
  const int r = blockIdx.y;
  const double th = theta[r];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = SX[r * n + i] - th * X[r * n + i];
    R[r * n + i] = v;
    acc += v * v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[r * gridDim.x + blockIdx.x] = red[0];
}

__global__ void rownorm_partial(const double* __restrict__ X, long long n, double* __restrict__ part) {
  const int r = blockIdx.y;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = X[r * n + i];
    acc += v * v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[r * gridDim.x + blockIdx.x] = red[0];
}

__global__ void finish_norms(const double* __restrict__ part, int nb, int k, double* __restrict__ out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[r * nb + b];
  out[r] = sqrt(s);
}

// rows of X scaled by 1/norm (norm > 0)
__global__ void scale_rows(double* __restrict__ X, long long n, const double* __restrict__ nrm) {
  const int r = blockIdx.y;
  double sc = nrm[r] > 0 ? 1.0 / nrm[r] : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    X[r * n + i] *= sc;
}

// Dn[j] = R[rows[j]] / (theta[rows[j]] - D), |theta - D| floored at 1e-8
__global__ void precond_kernel(const double* __restrict__ R, const double* __restrict__ theta,
                               const double* __restrict__ D, const int* __restrict__ rows, int nn, long long n,
                               double* __restrict__ Dn) {
  const int j = blockIdx.y;
  const int r = rows[j];
  const double th = theta[r];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double den = th - D[i];
    if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
    Dn[j * n + i] = R[r * n + i] / den;
  }
}

// canonical orthogonalisation coefficients: coef[j][c] = Z[j][src(c)] / sqrt(lam[src(c)])
// for eigenvalues above thr, largest first; count written to *cnt.
__global__ void canon_coef(const double* __restrict__ Z, const double* __restrict__ lam, int nn, double thr,
                           double* __restrict__ coef, int* __restrict__ cnt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int c = 0;
  for (int e = nn - 1; e >= 0; --e) {
    if (lam[e] > thr) {
      double sc = 1.0 / sqrt(lam[e]);
      for (int j = 0; j < nn; ++j) coef[j * nn + c] = Z[j * nn + e] * sc;
      ++c;
    }
  }
  *cnt = c;
}

// Out[r][i] = alpha sum_j coef[j][r] In[j][i] + beta Out[r][i] for r in a block
// of 16 rows (blockIdx.y), j < m, grid-stride over i: one pass over In per
// block of 16 output rows.
__global__ void rowcomb_kernel(int k, long long n, int m, double alpha, const double* __restrict__ coef, int ldc,
                               const double* __restrict__ In, double beta, double* __restrict__ Out) {
  __shared__ double cs[96][16];
  const int r0 = blockIdx.y * 16;
  const int kr = min(16, k - r0);
  for (int e = threadIdx.x; e < m * 16; e += blockDim.x) {
    const int j = e / 16, r = e % 16;
    cs[j][r] = r < kr ? coef[(long long)j * ldc + r0 + r] : 0.0;
  }
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0.0;
    for (int j = 0; j < m; ++j) {
      const double x = In[(long long)j * n + i];
#pragma unroll
      for (int r = 0; r < 16; ++r) acc[r] = fma(cs[j][r], x, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r < kr) {
        double* o = Out + (long long)(r0 + r) * n + i;
        *o = beta == 0.0 ? alpha * acc[r] : alpha * acc[r] + beta * *o;
      }
    }
  }
}

// Partial inner products P[z][a][b] = sum_{t in chunk z} A[a][t] B[b][t] for a
// block of 8 rows of A (blockIdx.y) and 4 rows of B (blockIdx.z).
__global__ void gram_partial(const double* __restrict__ A, int ma, const double* __restrict__ B, int mb, long long n,
                             long long chunk, double* __restrict__ P) {
  const int a0 = blockIdx.y * 8, b0 = blockIdx.z * 4;
  const int na = min(8, ma - a0), nb = min(4, mb - b0);
  const long long t0 = (long long)blockIdx.x * chunk, t1 = min(n, t0 + chunk);
  double acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    double bv[4], av[8];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = b < nb ? B[(long long)(b0 + b) * n + t] : 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) av[a] = a < na ? A[(long long)(a0 + a) * n + t] : 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
  __shared__ double red[8][32];  // [warp][a*4+b]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double v = acc[a][b];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][a * 4 + b] = v;
    }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int a = threadIdx.x / 4, b = threadIdx.x % 4;
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    if (a < na && b < nb) P[((long long)blockIdx.x * ma + a0 + a) * mb + b0 + b] = v;
  }
}

}  // namespace

// Out[r][i] = alpha sum_j coef[j*ldc + r] In[j][i] + beta Out[r][i], r < k,
// j < m (m <= 96), rows of length n: the subspace updates of the solver.
static void rowcomb(cudaStream_t s, int k, long long n, int m, double alpha, const double* coef, int ldc,
                    const double* In, double beta, double* Out) {
  if (k <= 0 || n <= 0) return;
  if (m > 96) fail(EAADC_ERR_ARG, "rowcomb: more than 96 input rows");
  const int gx = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
  rowcomb_kernel<<<dim3(gx, (k + 15) / 16), 256, 0, s>>>(k, n, m, alpha, coef, ldc, In, beta, Out);
  EA_LAUNCH();
}

// C[i][j] = sum_t A[i][t] B[j][t] for i < ma, j < mb (split over t)
static void gram(cudaStream_t s, const double* A, int ma, const double* B, int mb, long long n, double* C,
                 long long ldc) {
  if (ma <= 0 || mb <= 0) return;
  int nz = (int)std::min<long long>(std::max<long long>(1, n / 8192), 128);
  const long long chunk = (n + nz - 1) / nz;
  nz = (int)((n + chunk - 1) / chunk);
  DArr<double> P((size_t)nz * ma * mb, s);
  gram_partial<<<dim3(nz, (ma + 7) / 8, (mb + 3) / 4), 256, 0, s>>>(A, ma, B, mb, n, chunk, P.p);
  EA_LAUNCH();
  const int count = ma * mb;
  reduce_partials<<<(count + 255) / 256, 256, 0, s>>>(P.p, nz, count, C, ma, mb, ldc);
  EA_LAUNCH();
}

static void row_norms(cudaStream_t s, const double* X, int k, long long n, double* out) {
  int nb = std::min(256, (int)std::max<long long>(1, (n + 255) / 256));
  DArr<double> part((size_t)k * nb, s);
  rownorm_partial<<<dim3(nb, k), 256, 0, s>>>(X, n, part.p);
  EA_LAUNCH();
  finish_norms<<<1, 64, 0, s>>>(part.p, nb, k, out);
  EA_LAUNCH();
}

static void apply_sigma(cudaStream_t s, State& st, int prec, int nvec, const double* x, double* y) {
  if (prec == EAADC_FP64) sigma_fp64(s, st, nvec, x, y);
  else sigma_mixed(s, st, nvec, x, y, prec == EAADC_MIXED_BF16X3);
}

__global__ void gather_scalars(const double* __restrict__ src, const int* __restrict__ idx, int n,
                               double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void gather_rows(const double* __restrict__ src, const int* __restrict__ idx, int nr, long long n,
                            double* __restrict__ dst) {
  const long long total = (long long)nr * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    dst[e] = src[(long long)idx[e / n] * n + e % n];
}

// Dn[j] = rr (1/(theta - D) + m) for the selected rows j (a non-finite m keeps
// the diagonal term)
__global__ void learned_combine(const float* __restrict__ base, const float* __restrict__ rr,
                                const float* __restrict__ m, const int* __restrict__ jrows, int nl, long long n,
                                double* __restrict__ Dn) {
  const long long total = (long long)nl * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / n);
    const long long i = e % n;
    const float mi = m[e];
    Dn[(long long)jrows[q] * n + i] = (double)base[e] + (isfinite(mi) ? (double)rr[e] * (double)mi : 0.0);
  }
}

static void learned_correction(cudaStream_t s, State& st, const Mlp& mlp, const double* R, const double* theta,
                               const double* rnorm, const std::vector<int>& un, const std::vector<int>& lr, long long n,
                               double* Dn, DArr<float>& feat, DArr<float>& rr, DArr<float>& base, DArr<float>& m,
                               DArr<double>& thd, DArr<double>& rnd) {
  const int nl = (int)lr.size();
  std::vector<int> roots(nl);
  for (int q = 0; q < nl; ++q) roots[q] = un[lr[q]];
  DArr<int> ridx((size_t)nl, s), jidx((size_t)nl, s);
  EA_CK(cudaMemcpyAsync(ridx.p, roots.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s));
  EA_CK(cudaMemcpyAsync(jidx.p, lr.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s));
  const size_t rows = (size_t)nl * n;
  if (feat.n < rows * kMlpF) {
    feat.alloc(rows * kMlpF, s);
    rr.alloc(rows, s);
    base.alloc(rows, s);
    m.alloc(rows, s);
  }
  DArr<double> Rsel(rows, s);
  gather_rows<<<gridn((long long)rows), 256, 0, s>>>(R, ridx.p, nl, n, Rsel.p);
  EA_LAUNCH();
  gather_scalars<<<1, 128, 0, s>>>(theta, ridx.p, nl, thd.p);
  EA_LAUNCH();
  gather_scalars<<<1, 128, 0, s>>>(rnorm, ridx.p, nl, rnd.p);
  EA_LAUNCH();
  precond_features(s, st, nl, Rsel.p, thd.p, rnd.p, feat.p, rr.p, base.p);
  mlp_forward(s, mlp, (long long)rows, feat.p, m.p);
  learned_combine<<<gridn((long long)rows), 256, 0, s>>>(base.p, rr.p, m.p, jidx.p, nl, n, Dn);
  EA_LAUNCH();
}

// One Davidson phase at precision `prec` starting from `k0` orthonormal rows in V.
// Returns true if converged.
static bool davidson_phase(cudaStream_t s, State& st, int k, int prec, const eaadc_davidson_opts& opt, DArr<double>& V,
                           DArr<double>& S, int mmax, int k0, std::vector<double>& theta, std::vector<double>& rn,
                           int& iters, DArr<double>& Xr, bool stop_at_floor, const Mlp* mlp) {
  const long long n = st.dim;
  int m = k0;
  apply_sigma(s, st, prec, m, V.p, S.p);
  DArr<double> G((size_t)mmax * mmax, s), Gs((size_t)mmax * mmax, s), w((size_t)mmax, s), U((size_t)mmax * mmax, s);
  DArr<double> SX((size_t)k * n, s), R((size_t)k * n, s), Dn((size_t)k * n, s), Dtmp((size_t)k * n, s);
  DArr<double> rnd((size_t)k, s), C((size_t)mmax * k, s), Gd((size_t)k * k, s), Zd((size_t)k * k, s),
      ld((size_t)k, s), coef((size_t)k * k, s), nrm((size_t)k, s);
  DArr<int> rows((size_t)k, s), cnt(1, s);
  int nb = std::min(256, (int)std::max<long long>(1, (n + 255) / 256));
  DArr<double> part((size_t)k * nb, s);
  std::vector<double> th_old(k, INFINITY);
  std::vector<double> hist;  // largest residual norm per iteration
  // learned correction: per root, whether its last step used it and whether it fell back
  const bool learned = opt.precond == 1 && mlp && mlp->ready;
  std::vector<char> used(k, 0), fell(k, 0);
  std::vector<double> rn_prev(k, INFINITY);
  DArr<float> feat, lrr, lbase, lm;
  DArr<double> thd((size_t)k, s), rnd2((size_t)k, s);
  theta.assign(k, 0.0);
  rn.assign(k, 0.0);
  bool conv = false;
  int mg = 0;  // rows/columns of G already formed
  for (int it = 1; it <= opt.maxit; ++it) {
    iters++;
    // subspace matrix G = V S^T, only the rows and columns of new vectors
    if (mg < m) {
      gram(s, V.p + (long long)mg * n, m - mg, S.p, m, n, G.p + (long long)mg * mmax, mmax);
      if (mg > 0) gram(s, V.p, mg, S.p + (long long)mg * n, m - mg, n, G.p + mg, mmax);
      mg = m;
    }
    symmetrize<<<(m * m + 255) / 256, 256, 0, s>>>(G.p, m, mmax, Gs.p);
    EA_LAUNCH();
    jacobi_eigh(s, m, Gs.p, w.p, U.p);
    // Ritz vectors and their sigma: X = U[:, :k]^T V
    rowcomb(s, k, n, m, 1.0, U.p, m, V.p, 0.0, Xr.p);
    rowcomb(s, k, n, m, 1.0, U.p, m, S.p, 0.0, SX.p);
    residual_kernel<<<dim3(nb, k), 256, 0, s>>>(SX.p, Xr.p, w.p, R.p, n, k, part.p);
    EA_LAUNCH();
    finish_norms<<<1, 64, 0, s>>>(part.p, nb, k, rnd.p);
    EA_LAUNCH();
    EA_CK(cudaMemcpyAsync(theta.data(), w.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    EA_CK(cudaMemcpyAsync(rn.data(), rnd.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    EA_CK(cudaStreamSynchronize(s));
    if (prec != EAADC_FP64) check_device_error(s, st);
    for (int r = 0; r < k; ++r)
      if (!std::isfinite(theta[r]) || !std::isfinite(rn[r])) fail(EAADC_ERR_NONFINITE, "davidson: non-finite Ritz value or residual");
    bool all = true;
    std::vector<int> un;
    for (int r = 0; r < k; ++r) {
      bool c = rn[r] <= opt.tol && std::fabs(theta[r] - th_old[r]) <= opt.etol;
      all &= c;
      if (rn[r] > opt.tol) un.push_back(r);
    }
    th_old = theta;
    if (opt.trace > 0 && st.trN < opt.trace) {
      if (st.trN == 0 || st.trK != k) {
        st.trK = k;
        st.trN = 0;
        st.trX.alloc((size_t)opt.trace * k * n, s);
        st.trR.alloc((size_t)opt.trace * k * n, s);
        st.trTheta.clear();
      }
      EA_CK(cudaMemcpyAsync(st.trX.p + (long long)st.trN * k * n, Xr.p, sizeof(double) * k * n,
                            cudaMemcpyDeviceToDevice, s));
      EA_CK(cudaMemcpyAsync(st.trR.p + (long long)st.trN * k * n, R.p, sizeof(double) * k * n,
                            cudaMemcpyDeviceToDevice, s));
      st.trTheta.insert(st.trTheta.end(), theta.begin(), theta.end());
      ++st.trN;
    }
    if (all) { conv = true; break; }
    // reduced precision: stop at the noise floor of the mixed sigma (the
    // largest residual shrank by less than 2x over the last 8 iterations)
    double worst = 0.0;
    for (int r = 0; r < k; ++r) worst = std::max(worst, rn[r]);
    hist.push_back(worst);
    if (stop_at_floor && hist.size() > 8 && worst < 1e-3 && worst > 0.5 * hist[hist.size() - 9]) break;
    if (un.empty()) continue;  // residuals small, Ritz values still moving: iterate on same space
    int nn = (int)un.size();
    EA_CK(cudaMemcpyAsync(rows.p, un.data(), sizeof(int) * nn, cudaMemcpyHostToDevice, s));
    precond_kernel<<<dim3(nb, nn), 256, 0, s>>>(R.p, w.p, st.diag.p, rows.p, nn, n, Dn.p);
    EA_LAUNCH();
    if (learned) {
      // a root whose residual grew after a learned step falls back to the diagonal correction
      std::vector<int> lr;
      for (int j = 0; j < nn; ++j) {
        const int r = un[j];
        if (used[r] && rn[r] >= rn_prev[r]) fell[r] = 1;
        used[r] = !fell[r];
        if (used[r]) lr.push_back(j);
      }
      for (int r = 0; r < k; ++r) rn_prev[r] = rn[r];
      if (!lr.empty()) learned_correction(s, st, *mlp, R.p, w.p, rnd.p, un, lr, n, Dn.p, feat, lrr, lbase, lm, thd, rnd2);
    }
    row_norms(s, Dn.p, nn, n, nrm.p);
    scale_rows<<<dim3(nb, nn), 256, 0, s>>>(Dn.p, n, nrm.p);
    EA_LAUNCH();
    for (int pass = 0; pass < 2; ++pass) {
      gram(s, V.p, m, Dn.p, nn, n, C.p, nn);
      rowcomb(s, nn, n, m, -1.0, C.p, nn, V.p, 1.0, Dn.p);
    }
    gram(s, Dn.p, nn, Dn.p, nn, n, Gd.p, nn);
    symmetrize<<<1, 256, 0, s>>>(Gd.p, nn, nn, Zd.p);
    EA_LAUNCH();
    DArr<double> Zv((size_t)nn * nn, s);
    jacobi_eigh(s, nn, Zd.p, ld.p, Zv.p);
    canon_coef<<<1, 1, 0, s>>>(Zv.p, ld.p, nn, 1e-18, coef.p, cnt.p);
    EA_LAUNCH();
    int nacc = 0;
    EA_CK(cudaMemcpyAsync(&nacc, cnt.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    EA_CK(cudaStreamSynchronize(s));
    if (nacc == 0) break;
    if (m + nacc > mmax) {
      int keep = std::min(std::max(2 * k, k), m);
      keep = std::min(keep, mmax - nacc);
      DArr<double> T((size_t)keep * n, s);
      rowcomb(s, keep, n, m, 1.0, U.p, m, V.p, 0.0, T.p);
      EA_CK(cudaMemcpyAsync(V.p, T.p, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, s));
      rowcomb(s, keep, n, m, 1.0, U.p, m, S.p, 0.0, T.p);
      EA_CK(cudaMemcpyAsync(S.p, T.p, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, s));
      m = keep;
      mg = 0;
    }
    // new orthonormal directions: coef^T Dn
    rowcomb(s, nacc, n, nn, 1.0, coef.p, nn, Dn.p, 0.0, V.p + (long long)m * n);
    apply_sigma(s, st, prec, nacc, V.p + (long long)m * n, S.p + (long long)m * n);
    m += nacc;
  }
  return conv;
}

// Final sigma-and-Ritz step on the k Ritz vectors in st.evecs: sigma at
// precision prec (FP64, or the split-BF16 one), Rayleigh-Ritz in their span,
// residual norms of that sigma.  The Ritz values are then exact to second
// order in the error of the vectors, up to the error of that sigma.
static void final_ritz(cudaStream_t s, State& st, int k, int prec, std::vector<double>& theta, std::vector<double>& rn) {
  const long long n = st.dim;
  DArr<double> SX((size_t)k * n, s), G((size_t)k * k, s), Gs((size_t)k * k, s), w((size_t)k, s), U((size_t)k * k, s),
      X2((size_t)k * n, s), S2((size_t)k * n, s), R((size_t)k * n, s), rnd((size_t)k, s);
  apply_sigma(s, st, prec, k, st.evecs.p, SX.p);
  gram(s, st.evecs.p, k, SX.p, k, n, G.p, k);
  symmetrize<<<1, 256, 0, s>>>(G.p, k, k, Gs.p);
  EA_LAUNCH();
  jacobi_eigh(s, k, Gs.p, w.p, U.p);
  rowcomb(s, k, n, k, 1.0, U.p, k, st.evecs.p, 0.0, X2.p);
  rowcomb(s, k, n, k, 1.0, U.p, k, SX.p, 0.0, S2.p);
  const int nb = std::min(256, (int)std::max<long long>(1, (n + 255) / 256));
  DArr<double> part((size_t)k * nb, s);
  residual_kernel<<<dim3(nb, k), 256, 0, s>>>(S2.p, X2.p, w.p, R.p, n, k, part.p);
  EA_LAUNCH();
  finish_norms<<<1, 64, 0, s>>>(part.p, nb, k, rnd.p);
  EA_LAUNCH();
  EA_CK(cudaMemcpyAsync(st.evecs.p, X2.p, sizeof(double) * k * n, cudaMemcpyDeviceToDevice, s));
  theta.assign(k, 0.0);
  rn.assign(k, 0.0);
  EA_CK(cudaMemcpyAsync(theta.data(), w.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  EA_CK(cudaMemcpyAsync(rn.data(), rnd.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  EA_CK(cudaStreamSynchronize(s));
}

bool davidson_state(cudaStream_t s, State& st, int nroots, const eaadc_davidson_opts& opt, double* omega,
                    double* resnorm, int* iters, const Mlp* mlp) {
  if (opt.precond == 1 && !(mlp && mlp->ready))
    fail(EAADC_ERR_STATE, "learned correction requested but no weights loaded (eaadc_precond_load)");
  st.trN = 0;
  const long long n = st.dim;
  int k = (int)std::min<long long>(nroots, n);
  int mmax = (int)std::min<long long>(std::min(opt.max_sub, 96), n);
  if (mmax < 2 * k) mmax = (int)std::min<long long>(2 * k, n);
  if (mmax > 96) fail(EAADC_ERR_ARG, "davidson: subspace would exceed 96 vectors");
  DArr<double> V((size_t)mmax * n, s), S((size_t)mmax * n, s);
  st.evecs.alloc((size_t)k * n, s);
  st.nvecs = k;
  // guesses on the k lowest diagonal entries
  DArr<int> idx((size_t)k, s);
  int npart = std::min(256, (int)std::max<long long>(1, (n + 255) / 256));
  DArr<double> pv((size_t)npart, s);
  DArr<long long> pi((size_t)npart, s);
  for (int r = 0; r < k; ++r) {
    argmin_partial<<<npart, 256, 0, s>>>(st.diag.p, n, idx.p, r, pv.p, pi.p);
    EA_LAUNCH();
    argmin_final<<<1, 1, 0, s>>>(pv.p, pi.p, npart, idx.p + r);
    EA_LAUNCH();
  }
  set_units<<<gridn(n * k), 256, 0, s>>>(V.p, n, idx.p, k);
  EA_LAUNCH();
  std::vector<double> theta, rn;
  int it = 0;
  const bool refine = opt.prec != EAADC_FP64 && opt.refine;
  bool conv = davidson_phase(s, st, k, opt.prec, opt, V, S, mmax, k, theta, rn, it, st.evecs, refine, mlp);
  if (refine && (opt.refine == 2 || opt.refine == 3)) {
    final_ritz(s, st, k, opt.refine == 2 ? EAADC_FP64 : EAADC_MIXED_BF16X3, theta, rn);
    conv = true;
  } else if (refine) {
    // FP64 refinement from the mixed-precision Ritz vectors
    EA_CK(cudaMemcpyAsync(V.p, st.evecs.p, sizeof(double) * k * n, cudaMemcpyDeviceToDevice, s));
    conv = davidson_phase(s, st, k, EAADC_FP64, opt, V, S, mmax, k, theta, rn, it, st.evecs, false, mlp);
  }
  for (int r = 0; r < k; ++r) {
    omega[r] = theta[r];
    if (resnorm) resnorm[r] = rn[r];
  }
  for (int r = k; r < nroots; ++r) {
    omega[r] = NAN;
    if (resnorm) resnorm[r] = NAN;
  }
  st.omega.assign(theta.begin(), theta.begin() + k);
  if (iters) *iters = it;
  return conv;
}

void davidson(eaadc_ctx* ctx, int nroots, const eaadc_davidson_opts& opt, double* omega, double* resnorm, int* iters,
              bool* converged) {
  *converged = true;
  for (size_t si = 0; si < ctx->states.size(); ++si) {
    State& st = *ctx->states[si];
    const bool conv = davidson_state(ctx->stream, st, nroots, opt, omega + si * nroots,
                                     resnorm ? resnorm + si * nroots : nullptr, iters ? iters + si : nullptr, &ctx->mlp);
    if (st.ref1p.p) pick_target(ctx->stream, st);
    *converged &= conv;
  }
}

}  // namespace ea
