// State-specific frozen natural orbitals and natural auxiliary functions
// (Sec. II.C-E and the algorithm of Sec. III), all arithmetic on the device:
//   1. canonical EA-ADC(2) roots (FP64 Davidson) -> one target state per root;
//   2. D^MP2_ab = 2 sum_ijc tau_ij^ac (2 tau_ij^bc - tau_ij^cb) and, per state,
//      D^EA(k)_ab = y_a y_b + sum_kc (w_kac w_kbc + w_kca w_kcb) from the
//      zeroth-order ISR of the canonical root; D^SS = D^MP2 + D^EA (Eq. 17);
//   3. D^SS V = V eta (Eq. 9), keep eta > eta_crit (Eq. 10-11);
//   4. F~ = V~^T diag(eps) V~, F~ Z = Z e~ (Eq. 12-13), FNO basis V~ Z (Eq. 14);
//   5. DF factor in the FNO basis, W = J J^T over its vv block (Eq. 27-28),
//      keep eigenvectors with eigenvalue >= threshold, J~ = N~^T J (Eq. 29);
//   6. the state's ADC intermediates in the truncated space.
// Eq. 30 (ea_energies): w_corr = w^(3)_FNO + w^(2)_canonical - w^(2)_FNO, with
// the target root in a truncated space chosen as the one whose 1p part
// overlaps most with the canonical root's 1p part carried into that space.
#include "internal.cuh"

#include <algorithm>
#include <cmath>

namespace ea {
namespace {

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

// D[a][b] += y[a] y[b]
__global__ void outer_add(double* __restrict__ D, const double* __restrict__ y, int v) {
  const long long n = (long long)v * v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    D[i] += y[i / v] * y[i % v];
}

// out[a][j] = e[a] * V[a][j]
__global__ void scale_rows(const double* __restrict__ V, const double* __restrict__ e, double* __restrict__ out, int rows,
                           int cols) {
  const long long n = (long long)rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = e[i / cols] * V[i];
}

// out[r][j] = V[r][c0 + j] for j < m (V has n columns)
__global__ void copy_cols(const double* __restrict__ V, int rows, int n, int c0, int m, double* __restrict__ out) {
  const long long total = (long long)rows * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    out[i] = V[(i / m) * n + c0 + i % m];
}

// out[r] = sum_a X[r][a] ref[a], a < v (one CTA per row)
__global__ void dot_1p(const double* __restrict__ X, long long dim, const double* __restrict__ ref, int v,
                       double* __restrict__ out) {
  __shared__ double sh[32];
  const double* x = X + (long long)blockIdx.x * dim;
  double t = 0.0;
  for (int a = threadIdx.x; a < v; a += blockDim.x) t += x[a] * ref[a];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) a += sh[i];
    out[blockIdx.x] = a;
  }
}

void copy_d(cudaStream_t s, DArr<double>& dst, const double* src, size_t n) {
  dst.alloc(n, s);
  EA_CK(cudaMemcpyAsync(dst.p, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
}

// Host copy of a device vector (sizes and thresholds decide allocation sizes).
std::vector<double> to_host(cudaStream_t s, const double* p, size_t n) {
  std::vector<double> h(n);
  EA_CK(cudaMemcpyAsync(h.data(), p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  EA_CK(cudaStreamSynchronize(s));
  return h;
}

// Number of trailing entries of an ascending spectrum that a threshold keeps
// (negative threshold: all; strict: eta > thr; else eta >= thr).
int kept(const std::vector<double>& w, double thr, bool strict) {
  if (thr < 0) return (int)w.size();
  int c = 0;
  for (double x : w) c += strict ? (x > thr) : (x >= thr);
  return c;
}

}  // namespace

void pick_target(cudaStream_t s, State& st) {
  const int k = st.nvecs;
  if (k <= 0 || !st.ref1p.p) return;
  DArr<double> ov((size_t)k, s);
  dot_1p<<<k, 256, 0, s>>>(st.evecs.p, st.dim, st.ref1p.p, st.v, ov.p);
  EA_LAUNCH();
  std::vector<double> h = to_host(s, ov.p, (size_t)k);
  int best = 0;
  double bs = -1.0;
  for (int r = 0; r < k; ++r) {
    const double sc = std::fabs(h[r]) + 1e-12 * (k - 1 - r);  // ties go to the lower root
    if (sc > bs) { bs = sc; best = r; }
  }
  st.target = best;
}

void build_fno_states(eaadc_ctx* ctx, int nstates, const double* fno_thr, const double* naf_thr, int order, double x3,
                      const eaadc_davidson_opts& copts) {
  cudaStream_t s = ctx->stream;
  const int o = ctx->o, v = ctx->v, naux = ctx->naux;
  const long long oo = (long long)o * o, vv = (long long)v * v;
  // 1. canonical EA-ADC(2)
  State can;
  can.o = o; can.v = v; can.naux = naux; can.order = 2; can.x3 = 1.0;
  copy_d(s, can.eo, ctx->eo.p, o);
  copy_d(s, can.ev, ctx->ev.p, v);
  copy_d(s, can.Boo, ctx->Boo.p, ctx->Boo.n);
  copy_d(s, can.Bov, ctx->Bov.p, ctx->Bov.n);
  copy_d(s, can.Bvv, ctx->Bvv.p, ctx->Bvv.n);
  build_state_intermediates(ctx, can);
  if (can.dim < nstates) fail(EAADC_ERR_ARG, "more states requested than the canonical space holds");
  std::vector<double> w2c(nstates), rn2(nstates);
  int it2 = 0;
  if (!davidson_state(s, can, nstates, copts, w2c.data(), rn2.data(), &it2))
    fail(EAADC_ERR_NOCONV, "canonical EA-ADC(2) roots did not converge");
  // 2. MP2 virtual density (state independent)
  DArr<double> Dmp2((size_t)vv, s);
  {
    DArr<double> t2((size_t)(oo * vv), s);
    permute(s, can.tau.p, {o, o, v, v}, {0, 1, 3, 2}, t2.p, -1.0, 0.0);
    axpby(s, (size_t)(oo * vv), 2.0, can.tau.p, 1.0, t2.p);
    einsum(s, "ijac,ijbc->ab", 2.0, Tens{can.tau.p, {o, o, v, v}}, Tens{t2.p, {o, o, v, v}}, 0.0, Tens{Dmp2.p, {v, v}});
  }
  can.Jmat.release(); can.Kmat.release(); can.tau.release();

  std::vector<State*> built;
  try {
    for (int k = 0; k < nstates; ++k) {
      double* X = can.evecs.p + (long long)k * can.dim;
      Tens Wk{X + v, {o, v, v}};
      // D^SS = D^MP2 + D^EA(k)
      DArr<double> D((size_t)vv, s);
      EA_CK(cudaMemcpyAsync(D.p, Dmp2.p, sizeof(double) * vv, cudaMemcpyDeviceToDevice, s));
      outer_add<<<gridn(vv), 256, 0, s>>>(D.p, X, v);
      EA_LAUNCH();
      einsum(s, "kac,kbc->ab", 1.0, Wk, Wk, 1.0, Tens{D.p, {v, v}});
      einsum(s, "kca,kcb->ab", 1.0, Wk, Wk, 1.0, Tens{D.p, {v, v}});
      // 3. natural orbitals, keep eta > eta_crit
      DArr<double> eta((size_t)v, s), Vd((size_t)vv, s);
      eigh_sym(s, v, D.p, eta.p, Vd.p);
      const int vp = kept(to_host(s, eta.p, v), fno_thr[k], true);
      if (vp < 1) fail(EAADC_ERR_ARG, "FNO threshold of state " + std::to_string(k) + " keeps no virtual orbital");
      DArr<double> Vt((size_t)v * vp, s);
      copy_cols<<<gridn((long long)v * vp), 256, 0, s>>>(Vd.p, v, v, v - vp, vp, Vt.p);
      EA_LAUNCH();
      // 4. semicanonical FNOs
      DArr<double> Ve((size_t)v * vp, s), F((size_t)vp * vp, s), efno((size_t)vp, s), Zf((size_t)vp * vp, s),
          Bfno((size_t)v * vp, s);
      scale_rows<<<gridn((long long)v * vp), 256, 0, s>>>(Vt.p, ctx->ev.p, Ve.p, v, vp);
      EA_LAUNCH();
      dgemm(s, true, false, vp, vp, v, 1.0, Vt.p, vp, Ve.p, vp, 0.0, F.p, vp);
      eigh_sym(s, vp, F.p, efno.p, Zf.p);
      dgemm(s, false, false, v, vp, vp, 1.0, Vt.p, vp, Zf.p, vp, 0.0, Bfno.p, vp);
      // 5. DF factor in the FNO basis, then natural auxiliary functions
      DArr<double> Bov1((size_t)naux * o * vp, s), T((size_t)naux * v * vp, s), Bvv1((size_t)naux * vp * vp, s);
      dgemm(s, false, false, naux * o, vp, v, 1.0, ctx->Bov.p, v, Bfno.p, vp, 0.0, Bov1.p, vp);
      dgemm(s, false, false, naux * v, vp, v, 1.0, ctx->Bvv.p, v, Bfno.p, vp, 0.0, T.p, vp);
      einsum(s, "aA,QaB->QAB", 1.0, Tens{Bfno.p, {v, vp}}, Tens{T.p, {naux, v, vp}}, 0.0,
             Tens{Bvv1.p, {naux, vp, vp}});
      T.release();
      DArr<double> Wm((size_t)naux * naux, s), lam((size_t)naux, s), Nv((size_t)naux * naux, s);
      dgemm(s, false, true, naux, naux, vp * vp, 1.0, Bvv1.p, (long long)vp * vp, Bvv1.p, (long long)vp * vp, 0.0,
            Wm.p, naux);
      eigh_sym(s, naux, Wm.p, lam.p, Nv.p);
      const int np = kept(to_host(s, lam.p, naux), naf_thr[k], false);
      if (np < 1) fail(EAADC_ERR_ARG, "NAF threshold of state " + std::to_string(k) + " keeps no auxiliary function");
      DArr<double> N((size_t)naux * np, s);
      copy_cols<<<gridn((long long)naux * np), 256, 0, s>>>(Nv.p, naux, naux, naux - np, np, N.p);
      EA_LAUNCH();
      // 6. the truncated state
      State* st = new State();
      built.push_back(st);
      st->o = o; st->v = vp; st->naux = np; st->order = order; st->x3 = x3; st->build_prec = ctx->build_prec;
      st->vfull = v; st->nauxfull = naux; st->omega2_can = w2c[k];
      copy_d(s, st->eo, ctx->eo.p, o);
      st->ev = std::move(efno);
      st->Boo.alloc((size_t)np * oo, s);
      st->Bov.alloc((size_t)np * o * vp, s);
      st->Bvv.alloc((size_t)np * vp * vp, s);
      dgemm(s, true, false, np, (int)oo, naux, 1.0, N.p, np, ctx->Boo.p, oo, 0.0, st->Boo.p, oo);
      dgemm(s, true, false, np, o * vp, naux, 1.0, N.p, np, Bov1.p, (long long)o * vp, 0.0, st->Bov.p,
            (long long)o * vp);
      dgemm(s, true, false, np, vp * vp, naux, 1.0, N.p, np, Bvv1.p, (long long)vp * vp, 0.0, st->Bvv.p,
            (long long)vp * vp);
      st->ref1p.alloc((size_t)vp, s);
      dgemm(s, true, false, vp, 1, v, 1.0, Bfno.p, vp, X, 1, 0.0, st->ref1p.p, 1);
      build_state_intermediates(ctx, *st);
    }
  } catch (...) {
    for (auto* p : built) delete p;
    throw;
  }
  for (auto* p : ctx->states) delete p;
  ctx->states = built;
}

void ea_energies(eaadc_ctx* ctx, const eaadc_davidson_opts& opts, double* w_uncorr, double* w_corr, double* w2_can,
                 double* w2_fno) {
  cudaStream_t s = ctx->stream;
  for (size_t si = 0; si < ctx->states.size(); ++si) {
    State& st = *ctx->states[si];
    if (!st.ref1p.p) fail(EAADC_ERR_STATE, "state " + std::to_string(si) + " was not built by eaadc_build_states");
    if (st.target < 0 || st.omega.empty()) fail(EAADC_ERR_STATE, "run eaadc_davidson before eaadc_ea_energies");
    // EA-ADC(2) in the same truncated space
    State t;
    t.o = st.o; t.v = st.v; t.naux = st.naux; t.order = 2; t.x3 = 1.0;
    copy_d(s, t.eo, st.eo.p, st.eo.n);
    copy_d(s, t.ev, st.ev.p, st.ev.n);
    copy_d(s, t.Boo, st.Boo.p, st.Boo.n);
    copy_d(s, t.Bov, st.Bov.p, st.Bov.n);
    copy_d(s, t.Bvv, st.Bvv.p, st.Bvv.n);
    build_state_intermediates(ctx, t);
    // state si comes from the si-th canonical ADC(2) root: solve past it
    const int nr = std::max((int)st.omega.size(), (int)si + 2);
    std::vector<double> w2(nr);
    if (!davidson_state(s, t, nr, opts, w2.data(), nullptr, nullptr))
      fail(EAADC_ERR_NOCONV, "EA-ADC(2) roots of state " + std::to_string(si) + " did not converge");
    copy_d(s, t.ref1p, st.ref1p.p, st.ref1p.n);
    pick_target(s, t);
    const double w3 = st.omega[st.target], w2f = t.omega[t.target];
    if (w_uncorr) w_uncorr[si] = w3;
    if (w2_can) w2_can[si] = st.omega2_can;
    if (w2_fno) w2_fno[si] = w2f;
    if (w_corr) w_corr[si] = w3 + st.omega2_can - w2f;
  }
}

}  // namespace ea
