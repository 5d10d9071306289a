// Learned Davidson correction (a per-element MLP) and its training.
//
// For a root with Ritz value theta and residual r, element I of the
// correction is rr_I (1/(theta - D_I) + m_I), rr = r/||r||, with the diagonal
// guard |theta - D_I| >= 1e-8, and m_I = MLP(f_I): three tanh layers of width
// 256 and a linear output on 16 per-element features
//   f0 rr_I sqrt(dim)      f1 asinh(D_I - theta)   f2 clip(1/(theta-D_I), +-100)/100
//   f3 eps_k (2p1h)        f4 asinh(eps_b) (1p: asinh(eps_a))  f5 asinh(eps_c) (2p1h)
//   f6 theta               f7 log10 ||r||          f8 [1p]   f9 [2p1h with b = c]
//   f10 (bb|cc) for 2p1h (the ladder diagonal, absent from D)
// (zero padding to 16).  The layers are FP32 GEMMs on CUDA cores; training
// minimises the mean over vectors of 1 - cos^2(delta, t) against the projected
// exact correction t = (I - y y^T)(y* - y), by backpropagation and Adam.
#include "internal.cuh"

#include <algorithm>
#include <cmath>

namespace ea {
namespace {

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

constexpr long long oW1 = 0, ob1 = oW1 + kMlpW * kMlpF, oW2 = ob1 + kMlpW, ob2 = oW2 + kMlpW * kMlpW,
                    oW3 = ob2 + kMlpW, ob3 = oW3 + kMlpW * kMlpW, ow4 = ob3 + kMlpW, ob4 = ow4 + kMlpW;
static_assert(ob4 + 1 == kMlpParams, "MLP parameter layout");

__device__ __forceinline__ double guard(double den) {
  return fabs(den) < 1e-8 ? (den < 0 ? -1e-8 : 1e-8) : den;
}

__global__ void features_kernel(const double* __restrict__ R, long long dim, int o, int v,
                                const double* __restrict__ D, const double* __restrict__ eo,
                                const double* __restrict__ ev, const double* __restrict__ theta,
                                const double* __restrict__ rnorm, const double* __restrict__ lad, int nvec,
                                float* __restrict__ feat, float* __restrict__ rr, float* __restrict__ base) {
  const long long total = dim * nvec;
  const double sq = sqrt((double)dim);
  const long long vv = (long long)v * v;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e / dim);
    const long long i = e % dim;
    const double th = theta[n], rn = rnorm[n];
    const double x = R[e] / rn;
    const double den = guard(th - D[i]);
    double ek = 0.0, eb, ec = 0.0, one = 0.0, dg = 0.0, ld = 0.0;
    if (i < v) {
      eb = asinh(ev[i]);
      one = 1.0;
    } else {
      const long long j = i - v;
      const int k = (int)(j / vv), b = (int)((j / v) % v), c = (int)(j % v);
      ek = eo[k];
      eb = asinh(ev[b]);
      ec = asinh(ev[c]);
      dg = (b == c) ? 1.0 : 0.0;
      ld = lad[(long long)b * v + c];
    }
    float* f = feat + e * kMlpF;
    f[0] = (float)(x * sq);
    f[1] = (float)asinh(D[i] - th);
    f[2] = (float)(fmin(fmax(1.0 / den, -100.0), 100.0) / 100.0);
    f[3] = (float)ek;
    f[4] = (float)eb;
    f[5] = (float)ec;
    f[6] = (float)th;
    f[7] = (float)log10(rn);
    f[8] = (float)one;
    f[9] = (float)dg;
    f[10] = (float)ld;
#pragma unroll
    for (int q = 11; q < kMlpF; ++q) f[q] = 0.f;
    rr[e] = (float)x;
    base[e] = (float)(x / den);
  }
}

// per vector: sum r^2, sum y.y*, sum y.y (one CTA each)
__global__ void vec_sums(const double* __restrict__ R, const double* __restrict__ Y, const double* __restrict__ Ys,
                         long long dim, double* __restrict__ out) {
  __shared__ double sh[3][32];
  const long long off = (long long)blockIdx.x * dim;
  double a = 0.0, b = 0.0, c = 0.0;
  for (long long i = threadIdx.x; i < dim; i += blockDim.x) {
    const double r = R[off + i];
    a += r * r;
    if (Y) {
      const double y = Y[off + i];
      c += y * y;
      if (Ys) b += y * Ys[off + i];
    }
  }
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = a; sh[1][threadIdx.x >> 5] = b; sh[2][threadIdx.x >> 5] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { s0 += sh[0][i]; s1 += sh[1][i]; s2 += sh[2][i]; }
    out[3 * blockIdx.x] = sqrt(s0);
    out[3 * blockIdx.x + 1] = s1;
    out[3 * blockIdx.x + 2] = s2;
  }
}

// t = (y* s - y) - y (y . (y* s - y)), s = sign(y . y*)
__global__ void target_kernel(const double* __restrict__ Y, const double* __restrict__ Ys, const double* __restrict__ sums,
                              long long dim, int nvec, float* __restrict__ T) {
  const long long total = dim * nvec;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e / dim);
    const double yys = sums[3 * n + 1], yy = sums[3 * n + 2];
    const double sg = yys < 0 ? -1.0 : 1.0;
    const double proj = sg * yys - yy;  // y . (s y* - y)
    const double y = Y[e];
    T[e] = (float)(sg * Ys[e] - y - y * proj);
  }
}

__global__ void rnorm_only(const double* __restrict__ sums, double* __restrict__ rn, int nvec) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nvec) rn[n] = sums[3 * n];
}

// H = tanh(H + b) in place, rows of kMlpW
__global__ void bias_tanh(float* __restrict__ H, const float* __restrict__ b, long long n) {
  const long long total = n * kMlpW;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    H[e] = tanhf(H[e] + b[e % kMlpW]);
}

// m[i] = H[i] . w + b (one warp per row)
__global__ void row_dot(const float* __restrict__ H, const float* __restrict__ w, const float* __restrict__ b, long long n,
                        float* __restrict__ m) {
  const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float t = 0.f;
  for (int j = lane; j < kMlpW; j += 32) t += H[row * kMlpW + j] * w[j];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) m[row] = t + b[0];
}

// per segment: c = sum d t, dd = sum d d, tt = sum t t with d = base + rr m (one CTA per segment)
__global__ void seg_sums(const int* __restrict__ segs, const float* __restrict__ base, const float* __restrict__ rr,
                         const float* __restrict__ m, const float* __restrict__ T, double* __restrict__ out) {
  __shared__ double sh[3][32];
  const int a = segs[blockIdx.x], b = segs[blockIdx.x + 1];
  double c = 0.0, dd = 0.0, tt = 0.0;
  for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
    const double d = (double)base[i] + (double)rr[i] * (double)m[i], t = T[i];
    c += d * t;
    dd += d * d;
    tt += t * t;
  }
  for (int o = 16; o; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
    tt += __shfl_xor_sync(0xffffffffu, tt, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = c; sh[1][threadIdx.x >> 5] = dd; sh[2][threadIdx.x >> 5] = tt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { s0 += sh[0][i]; s1 += sh[1][i]; s2 += sh[2][i]; }
    out[3 * blockIdx.x] = s0;
    out[3 * blockIdx.x + 1] = s1;
    out[3 * blockIdx.x + 2] = s2;
  }
}

// dL/dm_i for the mean over segments of 1 - c^2/(dd tt) (one CTA per segment)
__global__ void seg_grad(const int* __restrict__ segs, const double* __restrict__ sums, int nseg,
                         const float* __restrict__ base, const float* __restrict__ rr, const float* __restrict__ m,
                         const float* __restrict__ T, float* __restrict__ gm) {
  const int a = segs[blockIdx.x], b = segs[blockIdx.x + 1];
  const double c = sums[3 * blockIdx.x], dd = sums[3 * blockIdx.x + 1], tt = sums[3 * blockIdx.x + 2];
  const double k1 = -2.0 * c / (dd * tt) / nseg, k2 = 2.0 * c * c / (dd * dd * tt) / nseg;
  for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
    const double d = (double)base[i] + (double)rr[i] * (double)m[i];
    gm[i] = (float)((k1 * T[i] + k2 * d) * rr[i]);
  }
}

// G = outer(gm, w4) * (1 - H^2)
__global__ void out_backprop(const float* __restrict__ gm, const float* __restrict__ w4, const float* __restrict__ H,
                             long long n, float* __restrict__ G) {
  const long long total = n * kMlpW;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const float h = H[e];
    G[e] = gm[e / kMlpW] * w4[e % kMlpW] * (1.f - h * h);
  }
}

// G *= (1 - H^2)
__global__ void tanh_backprop(float* __restrict__ G, const float* __restrict__ H, long long n) {
  const long long total = n * kMlpW;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const float h = H[e];
    G[e] *= (1.f - h * h);
  }
}

// column sums of G [n][kMlpW] (and of a vector when G is nullptr: out[0] = sum v)
__global__ void col_sums(const float* __restrict__ G, long long n, float* __restrict__ out) {
  const int c = blockIdx.x;
  __shared__ float sh[32];
  float t = 0.f;
  for (long long r = threadIdx.x; r < n; r += blockDim.x) t += G[r * kMlpW + c];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) a += sh[i];
    out[c] = a;
  }
}

__global__ void vec_sum(const float* __restrict__ x, long long n, float* __restrict__ out) {
  __shared__ float sh[32];
  float t = 0.f;
  for (long long r = threadIdx.x; r < n; r += blockDim.x) t += x[r];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) a += sh[i];
    out[0] = a;
  }
}

// Adam (Kingma and Ba, 2015), bias-corrected, step >= 1
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  }
}

struct Acts {
  DArr<float> h1, h2, h3, m;
};

void forward_acts(cudaStream_t s, const Mlp& net, long long n, const float* feat, Acts& a) {
  const float* w = net.w.p;
  a.h1.alloc((size_t)(n * kMlpW), s);
  a.h2.alloc((size_t)(n * kMlpW), s);
  a.h3.alloc((size_t)(n * kMlpW), s);
  a.m.alloc((size_t)n, s);
  const int N = (int)n;
  gemm<float>(s, false, true, N, kMlpW, kMlpF, 1.f, feat, kMlpF, w + oW1, kMlpF, 0.f, a.h1.p, kMlpW, GemmBatch());
  bias_tanh<<<gridn(n * kMlpW), 256, 0, s>>>(a.h1.p, w + ob1, n);
  EA_LAUNCH();
  gemm<float>(s, false, true, N, kMlpW, kMlpW, 1.f, a.h1.p, kMlpW, w + oW2, kMlpW, 0.f, a.h2.p, kMlpW, GemmBatch());
  bias_tanh<<<gridn(n * kMlpW), 256, 0, s>>>(a.h2.p, w + ob2, n);
  EA_LAUNCH();
  gemm<float>(s, false, true, N, kMlpW, kMlpW, 1.f, a.h2.p, kMlpW, w + oW3, kMlpW, 0.f, a.h3.p, kMlpW, GemmBatch());
  bias_tanh<<<gridn(n * kMlpW), 256, 0, s>>>(a.h3.p, w + ob3, n);
  EA_LAUNCH();
  row_dot<<<(int)((n * 32 + 255) / 256), 256, 0, s>>>(a.h3.p, w + ow4, w + ob4, n, a.m.p);
  EA_LAUNCH();
}

}  // namespace

void mlp_forward(cudaStream_t s, const Mlp& net, long long n, const float* feat, float* m) {
  if (!net.ready) fail(EAADC_ERR_STATE, "no learned-correction weights loaded (eaadc_precond_load)");
  if (n <= 0) return;
  if (n > (1LL << 31) - 1) fail(EAADC_ERR_ARG, "mlp: too many rows");
  Acts a;
  forward_acts(s, net, n, feat, a);
  EA_CK(cudaMemcpyAsync(m, a.m.p, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
}

// dq[Q][b] = B^Q_bb
__global__ void bvv_diag(const double* __restrict__ Bvv, int naux, int v, double* __restrict__ dq) {
  const long long total = (long long)naux * v;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long Q = e / v, b = e % v;
    dq[e] = Bvv[(Q * v + b) * v + b];
  }
}

void precond_features(cudaStream_t s, State& st, int nvec, const double* R, const double* theta_dev,
                      const double* rnorm_dev, float* feat, float* rr, float* base) {
  if (!st.lad_diag.p) {  // (bb|cc) = sum_Q B^Q_bb B^Q_cc, once per state
    DArr<double> dq((size_t)st.naux * st.v, s);
    bvv_diag<<<gridn((long long)st.naux * st.v), 256, 0, s>>>(st.Bvv.p, st.naux, st.v, dq.p);
    EA_LAUNCH();
    st.lad_diag.alloc((size_t)st.v * st.v, s);
    dgemm(s, true, false, st.v, st.v, st.naux, 1.0, dq.p, st.v, dq.p, st.v, 0.0, st.lad_diag.p, st.v);
  }
  features_kernel<<<gridn(st.dim * nvec), 256, 0, s>>>(R, st.dim, st.o, st.v, st.diag.p, st.eo.p, st.ev.p, theta_dev,
                                                       rnorm_dev, st.lad_diag.p, nvec, feat, rr, base);
  EA_LAUNCH();
}

// Loss and gradient (into net.g) of a batch of nseg vectors; optional Adam step.
double mlp_loss_grad(cudaStream_t s, Mlp& net, int nseg, const int* segs_host, const float* feat, const float* rr,
                     const float* base, const float* T, float lr, bool update) {
  if (!net.ready) fail(EAADC_ERR_STATE, "no learned-correction weights loaded (eaadc_precond_load)");
  const long long n = segs_host[nseg];
  if (nseg < 1 || segs_host[0] != 0 || n < 1) fail(EAADC_ERR_ARG, "mlp: bad segments");
  for (int j = 0; j < nseg; ++j)
    if (segs_host[j + 1] <= segs_host[j]) fail(EAADC_ERR_ARG, "mlp: empty or unordered segment");
  DArr<int> segs((size_t)nseg + 1, s);
  EA_CK(cudaMemcpyAsync(segs.p, segs_host, sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice, s));
  Acts a;
  forward_acts(s, net, n, feat, a);
  DArr<double> sums((size_t)3 * nseg, s);
  seg_sums<<<nseg, 256, 0, s>>>(segs.p, base, rr, a.m.p, T, sums.p);
  EA_LAUNCH();
  std::vector<double> hs((size_t)3 * nseg);
  EA_CK(cudaMemcpyAsync(hs.data(), sums.p, sizeof(double) * 3 * nseg, cudaMemcpyDeviceToHost, s));
  DArr<float> gm((size_t)n, s), G((size_t)(n * kMlpW), s), G2((size_t)(n * kMlpW), s);
  seg_grad<<<nseg, 256, 0, s>>>(segs.p, sums.p, nseg, base, rr, a.m.p, T, gm.p);
  EA_LAUNCH();
  const float* w = net.w.p;
  float* g = net.g.p;
  const int N = (int)n;
  // output layer
  gemm<float>(s, true, false, kMlpW, 1, N, 1.f, a.h3.p, kMlpW, gm.p, 1, 0.f, g + ow4, 1, GemmBatch());
  vec_sum<<<1, 256, 0, s>>>(gm.p, n, g + ob4);
  EA_LAUNCH();
  out_backprop<<<gridn(n * kMlpW), 256, 0, s>>>(gm.p, w + ow4, a.h3.p, n, G.p);
  EA_LAUNCH();
  // layer 3
  gemm<float>(s, true, false, kMlpW, kMlpW, N, 1.f, G.p, kMlpW, a.h2.p, kMlpW, 0.f, g + oW3, kMlpW, GemmBatch());
  col_sums<<<kMlpW, 256, 0, s>>>(G.p, n, g + ob3);
  EA_LAUNCH();
  gemm<float>(s, false, false, N, kMlpW, kMlpW, 1.f, G.p, kMlpW, w + oW3, kMlpW, 0.f, G2.p, kMlpW, GemmBatch());
  tanh_backprop<<<gridn(n * kMlpW), 256, 0, s>>>(G2.p, a.h2.p, n);
  EA_LAUNCH();
  // layer 2
  gemm<float>(s, true, false, kMlpW, kMlpW, N, 1.f, G2.p, kMlpW, a.h1.p, kMlpW, 0.f, g + oW2, kMlpW, GemmBatch());
  col_sums<<<kMlpW, 256, 0, s>>>(G2.p, n, g + ob2);
  EA_LAUNCH();
  gemm<float>(s, false, false, N, kMlpW, kMlpW, 1.f, G2.p, kMlpW, w + oW2, kMlpW, 0.f, G.p, kMlpW, GemmBatch());
  tanh_backprop<<<gridn(n * kMlpW), 256, 0, s>>>(G.p, a.h1.p, n);
  EA_LAUNCH();
  // layer 1
  gemm<float>(s, true, false, kMlpW, kMlpF, N, 1.f, G.p, kMlpW, feat, kMlpF, 0.f, g + oW1, kMlpF, GemmBatch());
  col_sums<<<kMlpW, 256, 0, s>>>(G.p, n, g + ob1);
  EA_LAUNCH();
  if (update) {
    ++net.step;
    const float c1 = 1.f - std::pow(0.9f, (float)net.step), c2 = 1.f - std::pow(0.999f, (float)net.step);
    adam_kernel<<<gridn(kMlpParams), 256, 0, s>>>(net.w.p, net.g.p, net.mom.p, net.vel.p, kMlpParams, lr, c1, c2);
    EA_LAUNCH();
  }
  EA_CK(cudaStreamSynchronize(s));
  double L = 0.0;
  for (int j = 0; j < nseg; ++j) L += 1.0 - hs[3 * j] * hs[3 * j] / (hs[3 * j + 1] * hs[3 * j + 2]);
  return L / nseg;
}

void mlp_load(cudaStream_t s, Mlp& net, const float* host) {
  net.w.alloc((size_t)kMlpParams, s);
  net.g.alloc((size_t)kMlpParams, s);
  net.mom.alloc((size_t)kMlpParams, s);
  net.vel.alloc((size_t)kMlpParams, s);
  EA_CK(cudaMemcpyAsync(net.w.p, host, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s));
  EA_CK(cudaMemsetAsync(net.g.p, 0, sizeof(float) * kMlpParams, s));
  EA_CK(cudaMemsetAsync(net.mom.p, 0, sizeof(float) * kMlpParams, s));
  EA_CK(cudaMemsetAsync(net.vel.p, 0, sizeof(float) * kMlpParams, s));
  EA_CK(cudaStreamSynchronize(s));
  net.step = 0;
  net.ready = true;
}

// Training pairs of nvec Ritz vectors Y with residuals R and values theta;
// Ys (optional) the converged eigenvectors of the same roots.
void precond_pairs(cudaStream_t s, State& st, int nvec, const double* Y, const double* R,
                   const double* theta_host, const double* Ys, float* feat, float* rr, float* base, float* T) {
  const long long dim = st.dim;
  DArr<double> sums((size_t)3 * nvec, s), rn((size_t)nvec, s), th((size_t)nvec, s);
  EA_CK(cudaMemcpyAsync(th.p, theta_host, sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
  vec_sums<<<nvec, 256, 0, s>>>(R, Y, Ys, dim, sums.p);
  EA_LAUNCH();
  rnorm_only<<<(nvec + 127) / 128, 128, 0, s>>>(sums.p, rn.p, nvec);
  EA_LAUNCH();
  precond_features(s, st, nvec, R, th.p, rn.p, feat, rr, base);
  if (Ys && T) {
    target_kernel<<<gridn(dim * nvec), 256, 0, s>>>(Y, Ys, sums.p, dim, nvec, T);
    EA_LAUNCH();
  }
}

}  // namespace ea
