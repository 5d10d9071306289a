// extern "C" entry points; every call converts internal errors to a status
// and a message (see include/eaadc.h for the contract of each function).
#include "internal.cuh"

#include <cmath>
#include <cstring>
#include <new>

eaadc_ctx::~eaadc_ctx() {
  for (auto* s : states) delete s;
  states.clear();
}

namespace {
thread_local std::string g_static_err;

template <class F>
eaadc_status guarded(eaadc_ctx* ctx, F&& f) {
  try {
    if (ctx) ctx->err.clear();
    f();
    return EAADC_OK;
  } catch (const ea::Error& e) {
    if (ctx) ctx->err = e.msg; else g_static_err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed"; else g_static_err = "host allocation failed";
    return EAADC_ERR_ALLOC;
  } catch (...) {
    if (ctx) ctx->err = "unknown internal error"; else g_static_err = "unknown internal error";
    return EAADC_ERR_STATE;
  }
}

void set_device(const eaadc_ctx* ctx) { EA_CK(cudaSetDevice(ctx->device)); }

ea::State& get_state(eaadc_ctx* ctx, int s) {
  if (s < 0 || s >= (int)ctx->states.size()) ea::fail(EAADC_ERR_ARG, "state index out of range (build states first)");
  return *ctx->states[s];
}

bool all_finite(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}
}  // namespace

extern "C" {

const char* eaadc_version(void) { return "eaadc-gb300 0.1 (sm_103a)"; }

long long eaadc_kernel_launches(void) { return __atomic_load_n(&ea::g_kernel_launches, __ATOMIC_RELAXED); }

eaadc_status eaadc_init(eaadc_ctx** out, int o, int v, int naux, const double* eps_occ, const double* eps_vir,
                        const double* B, int device, void* stream) {
  if (!out) { g_static_err = "out is NULL"; return EAADC_ERR_ARG; }
  *out = nullptr;
  if (o < 1 || v < 1 || naux < 1 || !eps_occ || !eps_vir || !B) {
    g_static_err = "invalid sizes or NULL input";
    return EAADC_ERR_ARG;
  }
  eaadc_ctx* ctx = new (std::nothrow) eaadc_ctx();
  if (!ctx) { g_static_err = "host allocation failed"; return EAADC_ERR_ALLOC; }
  eaadc_status st = guarded(ctx, [&] {
    const int n = o + v;
    if (!all_finite(eps_occ, o) || !all_finite(eps_vir, v)) ea::fail(EAADC_ERR_NONFINITE, "non-finite orbital energy");
    int ndev = 0;
    EA_CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) ea::fail(EAADC_ERR_ARG, "device index out of range");
    ctx->device = device;
    EA_CK(cudaSetDevice(device));
    ctx->stream = (cudaStream_t)stream;
    ctx->o = o; ctx->v = v; ctx->naux = naux;
    cudaStream_t s = ctx->stream;
    ctx->eo.alloc(o, s);
    ctx->ev.alloc(v, s);
    EA_CK(cudaMemcpyAsync(ctx->eo.p, eps_occ, sizeof(double) * o, cudaMemcpyHostToDevice, s));
    EA_CK(cudaMemcpyAsync(ctx->ev.p, eps_vir, sizeof(double) * v, cudaMemcpyHostToDevice, s));
    ctx->Boo.alloc((size_t)naux * o * o, s);
    ctx->Bov.alloc((size_t)naux * o * v, s);
    ctx->Bvv.alloc((size_t)naux * v * v, s);
    const size_t nn = (size_t)n * n;
    for (int Q = 0; Q < naux; ++Q) {
      const double* BQ = B + (size_t)Q * nn;
      EA_CK(cudaMemcpy2DAsync(ctx->Boo.p + (size_t)Q * o * o, sizeof(double) * o, BQ, sizeof(double) * n,
                              sizeof(double) * o, o, cudaMemcpyHostToDevice, s));
      EA_CK(cudaMemcpy2DAsync(ctx->Bov.p + (size_t)Q * o * v, sizeof(double) * v, BQ + o, sizeof(double) * n,
                              sizeof(double) * v, o, cudaMemcpyHostToDevice, s));
      EA_CK(cudaMemcpy2DAsync(ctx->Bvv.p + (size_t)Q * v * v, sizeof(double) * v, BQ + (size_t)o * n + o,
                              sizeof(double) * n, sizeof(double) * v, v, cudaMemcpyHostToDevice, s));
    }
    EA_CK(cudaStreamSynchronize(s));
  });
  if (st != EAADC_OK) {
    g_static_err = ctx->err;
    delete ctx;
    return st;
  }
  *out = ctx;
  return EAADC_OK;
}

eaadc_status eaadc_build_canonical(eaadc_ctx* ctx, int adc_order, double x3) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (adc_order != 2 && adc_order != 3) ea::fail(EAADC_ERR_ARG, "adc_order must be 2 or 3");
    if (!std::isfinite(x3)) ea::fail(EAADC_ERR_ARG, "x3 must be finite");
    set_device(ctx);
    cudaStream_t s = ctx->stream;
    for (auto* p : ctx->states) delete p;
    ctx->states.clear();
    auto* st = new ea::State();
    ctx->states.push_back(st);
    st->o = ctx->o; st->v = ctx->v; st->naux = ctx->naux;
    st->order = adc_order; st->x3 = x3; st->build_prec = ctx->build_prec;
    const int o = ctx->o, v = ctx->v, naux = ctx->naux;
    st->eo.alloc(o, s); st->ev.alloc(v, s);
    st->Boo.alloc((size_t)naux * o * o, s);
    st->Bov.alloc((size_t)naux * o * v, s);
    st->Bvv.alloc((size_t)naux * v * v, s);
    EA_CK(cudaMemcpyAsync(st->eo.p, ctx->eo.p, sizeof(double) * o, cudaMemcpyDeviceToDevice, s));
    EA_CK(cudaMemcpyAsync(st->ev.p, ctx->ev.p, sizeof(double) * v, cudaMemcpyDeviceToDevice, s));
    EA_CK(cudaMemcpyAsync(st->Boo.p, ctx->Boo.p, sizeof(double) * st->Boo.n, cudaMemcpyDeviceToDevice, s));
    EA_CK(cudaMemcpyAsync(st->Bov.p, ctx->Bov.p, sizeof(double) * st->Bov.n, cudaMemcpyDeviceToDevice, s));
    EA_CK(cudaMemcpyAsync(st->Bvv.p, ctx->Bvv.p, sizeof(double) * st->Bvv.n, cudaMemcpyDeviceToDevice, s));
    ea::build_state_intermediates(ctx, *st);
  });
}

namespace {
eaadc_davidson_opts inner_opts(const eaadc_davidson_opts* o) {
  if (o) {
    if (!(o->tol > 0) || o->maxit < 1) ea::fail(EAADC_ERR_ARG, "bad Davidson options");
    if (o->prec != EAADC_FP64 && o->prec != EAADC_MIXED_BF16 && o->prec != EAADC_MIXED_BF16X3)
      ea::fail(EAADC_ERR_ARG, "unknown precision");
    return *o;
  }
  eaadc_davidson_opts d;
  d.tol = 1e-8; d.etol = 1e-10; d.maxit = 300; d.max_sub = 40; d.prec = EAADC_FP64; d.refine = 0;
  d.precond = 0; d.trace = 0;
  return d;
}
}  // namespace

eaadc_status eaadc_set_build_precision(eaadc_ctx* ctx, int prec) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (prec != EAADC_FP64 && prec != EAADC_MIXED_BF16 && prec != EAADC_MIXED_BF16X3)
      ea::fail(EAADC_ERR_ARG, "unknown precision");
    ctx->build_prec = prec;
  });
}

eaadc_status eaadc_build_states(eaadc_ctx* ctx, int nstates, const double* fno_thresh, const double* naf_thresh,
                                int adc_order, double x3, const eaadc_davidson_opts* can_opts) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (nstates < 1 || !fno_thresh || !naf_thresh) ea::fail(EAADC_ERR_ARG, "bad state count or NULL thresholds");
    if (adc_order != 2 && adc_order != 3) ea::fail(EAADC_ERR_ARG, "adc_order must be 2 or 3");
    if (!std::isfinite(x3)) ea::fail(EAADC_ERR_ARG, "x3 must be finite");
    if (!all_finite(fno_thresh, nstates) || !all_finite(naf_thresh, nstates))
      ea::fail(EAADC_ERR_NONFINITE, "non-finite threshold");
    set_device(ctx);
    ea::build_fno_states(ctx, nstates, fno_thresh, naf_thresh, adc_order, x3, inner_opts(can_opts));
  });
}

eaadc_status eaadc_ea_energies(eaadc_ctx* ctx, const eaadc_davidson_opts* opts, double* omega_uncorr,
                               double* omega_corr, double* omega2_can, double* omega2_fno) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (ctx->states.empty()) ea::fail(EAADC_ERR_STATE, "no states built");
    set_device(ctx);
    ea::ea_energies(ctx, inner_opts(opts), omega_uncorr, omega_corr, omega2_can, omega2_fno);
  });
}

eaadc_status eaadc_eigh_sym(int n, const double* a_dev, double* w_dev, double* v_dev, int device, void* stream) {
  return guarded(nullptr, [&] {
    if (n < 1 || !a_dev || !w_dev || !v_dev) ea::fail(EAADC_ERR_ARG, "bad size or NULL pointer");
    int ndev = 0;
    EA_CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) ea::fail(EAADC_ERR_ARG, "device index out of range");
    EA_CK(cudaSetDevice(device));
    ea::eigh_sym((cudaStream_t)stream, n, a_dev, w_dev, v_dev);
  });
}

eaadc_status eaadc_state_info(const eaadc_ctx* ctx, int state, int* vprime, int* nauxprime, long long* dim) {
  if (!ctx) return EAADC_ERR_ARG;
  if (state < 0 || state >= (int)ctx->states.size()) return EAADC_ERR_ARG;
  const ea::State& st = *ctx->states[state];
  if (vprime) *vprime = st.v;
  if (nauxprime) *nauxprime = st.naux;
  if (dim) *dim = st.dim;
  return EAADC_OK;
}

eaadc_status eaadc_sigma(eaadc_ctx* ctx, int state, int nvec, const double* x_dev, double* sigma_dev, int prec,
                         void* stream) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    set_device(ctx);
    ea::State& st = get_state(ctx, state);
    if (nvec < 0 || (nvec > 0 && (!x_dev || !sigma_dev))) ea::fail(EAADC_ERR_ARG, "bad vector arguments");
    if (prec != EAADC_FP64 && prec != EAADC_MIXED_BF16 && prec != EAADC_MIXED_BF16X3)
      ea::fail(EAADC_ERR_ARG, "unknown precision");
    if (nvec == 0) return;
    const char* xa = (const char*)x_dev;
    const char* ya = (const char*)sigma_dev;
    size_t bytes = sizeof(double) * (size_t)nvec * st.dim;
    if (xa < ya + bytes && ya < xa + bytes) ea::fail(EAADC_ERR_ARG, "x and sigma overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == EAADC_FP64) ea::sigma_fp64(s, st, nvec, x_dev, sigma_dev);
    else ea::sigma_mixed(s, st, nvec, x_dev, sigma_dev, prec == EAADC_MIXED_BF16X3);
  });
}

eaadc_status eaadc_sigma_host(eaadc_ctx* ctx, int state, int nvec, const double* x_host, double* sigma_host,
                              int prec) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    set_device(ctx);
    ea::State& st = get_state(ctx, state);
    if (nvec <= 0 || !x_host || !sigma_host) ea::fail(EAADC_ERR_ARG, "bad vector arguments");
    cudaStream_t s = ctx->stream;
    size_t n = (size_t)nvec * st.dim;
    ea::DArr<double> x(n, s), y(n, s);
    EA_CK(cudaMemcpyAsync(x.p, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    if (prec != EAADC_FP64 && prec != EAADC_MIXED_BF16 && prec != EAADC_MIXED_BF16X3)
      ea::fail(EAADC_ERR_ARG, "unknown precision");
    if (prec == EAADC_FP64) ea::sigma_fp64(s, st, nvec, x.p, y.p);
    else ea::sigma_mixed(s, st, nvec, x.p, y.p, prec == EAADC_MIXED_BF16X3);
    EA_CK(cudaMemcpyAsync(sigma_host, y.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    EA_CK(cudaStreamSynchronize(s));
    if (prec != EAADC_FP64) ea::check_device_error(s, st);
  });
}

eaadc_status eaadc_ladder(eaadc_ctx* ctx, int state, int nvec, const double* x_dev, float* out_dev, void* stream) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    set_device(ctx);
    ea::State& st = get_state(ctx, state);
    if (st.order < 3) ea::fail(EAADC_ERR_STATE, "the ladder is part of ADC(3) only");
    if (nvec <= 0 || !x_dev || !out_dev) ea::fail(EAADC_ERR_ARG, "bad vector arguments");
    ea::ladder_only((cudaStream_t)stream, st, nvec, x_dev, out_dev, true);
  });
}

eaadc_status eaadc_diagonal(eaadc_ctx* ctx, int state, double* diag_host) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    set_device(ctx);
    ea::State& st = get_state(ctx, state);
    if (!diag_host) ea::fail(EAADC_ERR_ARG, "NULL output");
    EA_CK(cudaMemcpyAsync(diag_host, st.diag.p, sizeof(double) * st.dim, cudaMemcpyDeviceToHost, ctx->stream));
    EA_CK(cudaStreamSynchronize(ctx->stream));
  });
}

eaadc_status eaadc_get_m11(eaadc_ctx* ctx, int state, double* m11_host) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    set_device(ctx);
    ea::State& st = get_state(ctx, state);
    if (!m11_host) ea::fail(EAADC_ERR_ARG, "NULL output");
    EA_CK(cudaMemcpyAsync(m11_host, st.M11.p, sizeof(double) * st.M11.n, cudaMemcpyDeviceToHost, ctx->stream));
    EA_CK(cudaStreamSynchronize(ctx->stream));
  });
}

eaadc_status eaadc_precond_load(eaadc_ctx* ctx, const float* weights, size_t bytes) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (!weights || bytes != sizeof(float) * (size_t)ea::kMlpParams)
      ea::fail(EAADC_ERR_ARG, "weights must be EAADC_MLP_PARAMS floats");
    for (long long i = 0; i < ea::kMlpParams; ++i)
      if (!std::isfinite(weights[i])) ea::fail(EAADC_ERR_NONFINITE, "non-finite weight");
    set_device(ctx);
    ea::mlp_load(ctx->stream, ctx->mlp, weights);
  });
}

eaadc_status eaadc_precond_get(eaadc_ctx* ctx, float* weights, size_t bytes) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (!weights || bytes != sizeof(float) * (size_t)ea::kMlpParams)
      ea::fail(EAADC_ERR_ARG, "weights must be EAADC_MLP_PARAMS floats");
    if (!ctx->mlp.ready) ea::fail(EAADC_ERR_STATE, "no weights loaded");
    set_device(ctx);
    EA_CK(cudaMemcpyAsync(weights, ctx->mlp.w.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    EA_CK(cudaStreamSynchronize(ctx->stream));
  });
}

eaadc_status eaadc_precond_pairs(eaadc_ctx* ctx, int state, int nvec, const double* y_dev, const double* r_dev,
                                 const double* theta_host, const double* ystar_dev, float* feat_dev, float* rr_dev,
                                 float* base_dev, float* target_dev, void* stream) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    set_device(ctx);
    ea::State& st = get_state(ctx, state);
    if (nvec < 1 || !y_dev || !r_dev || !theta_host || !feat_dev || !rr_dev || !base_dev)
      ea::fail(EAADC_ERR_ARG, "bad arguments");
    if ((ystar_dev == nullptr) != (target_dev == nullptr)) ea::fail(EAADC_ERR_ARG, "ystar and target go together");
    ea::precond_pairs((cudaStream_t)stream, st, nvec, y_dev, r_dev, theta_host, ystar_dev, feat_dev, rr_dev,
                      base_dev, target_dev);
  });
}

eaadc_status eaadc_mlp_forward(eaadc_ctx* ctx, long long n, const float* feat_dev, float* m_dev, void* stream) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (n < 1 || !feat_dev || !m_dev) ea::fail(EAADC_ERR_ARG, "bad arguments");
    set_device(ctx);
    ea::mlp_forward((cudaStream_t)stream, ctx->mlp, n, feat_dev, m_dev);
  });
}

eaadc_status eaadc_mlp_loss_grad(eaadc_ctx* ctx, int nseg, const int* seg_host, const float* feat_dev,
                                 const float* rr_dev, const float* base_dev, const float* target_dev,
                                 double* loss_host, float* grad_host, void* stream) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (nseg < 1 || !seg_host || !feat_dev || !rr_dev || !base_dev || !target_dev) ea::fail(EAADC_ERR_ARG, "bad arguments");
    set_device(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    const double L = ea::mlp_loss_grad(s, ctx->mlp, nseg, seg_host, feat_dev, rr_dev, base_dev, target_dev, 0.f, false);
    if (loss_host) *loss_host = L;
    if (grad_host) {
      EA_CK(cudaMemcpyAsync(grad_host, ctx->mlp.g.p, sizeof(float) * ea::kMlpParams, cudaMemcpyDeviceToHost, s));
      EA_CK(cudaStreamSynchronize(s));
    }
  });
}

eaadc_status eaadc_mlp_train_step(eaadc_ctx* ctx, int nseg, const int* seg_host, const float* feat_dev,
                                  const float* rr_dev, const float* base_dev, const float* target_dev, float lr,
                                  double* loss_host, void* stream) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    if (nseg < 1 || !seg_host || !feat_dev || !rr_dev || !base_dev || !target_dev || !(lr > 0))
      ea::fail(EAADC_ERR_ARG, "bad arguments");
    set_device(ctx);
    const double L = ea::mlp_loss_grad((cudaStream_t)stream, ctx->mlp, nseg, seg_host, feat_dev, rr_dev, base_dev,
                                       target_dev, lr, true);
    if (loss_host) *loss_host = L;
  });
}

eaadc_status eaadc_get_trace(eaadc_ctx* ctx, int state, int* niters, int* nroots, double* x_host, double* r_host,
                             double* theta_host) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    set_device(ctx);
    ea::State& st = get_state(ctx, state);
    if (niters) *niters = st.trN;
    if (nroots) *nroots = st.trK;
    const size_t cnt = (size_t)st.trN * st.trK;
    if (!cnt) return;
    if (x_host) EA_CK(cudaMemcpyAsync(x_host, st.trX.p, sizeof(double) * cnt * st.dim, cudaMemcpyDeviceToHost, ctx->stream));
    if (r_host) EA_CK(cudaMemcpyAsync(r_host, st.trR.p, sizeof(double) * cnt * st.dim, cudaMemcpyDeviceToHost, ctx->stream));
    if (theta_host) std::memcpy(theta_host, st.trTheta.data(), sizeof(double) * cnt);
    EA_CK(cudaStreamSynchronize(ctx->stream));
  });
}

int eaadc_num_states(const eaadc_ctx* ctx) { return ctx ? (int)ctx->states.size() : 0; }

eaadc_status eaadc_davidson(eaadc_ctx* ctx, int nroots, const eaadc_davidson_opts* opts, double* omega,
                            double* resnorm, int* iters) {
  if (!ctx) return EAADC_ERR_ARG;
  bool conv = true;
  eaadc_status st = guarded(ctx, [&] {
    set_device(ctx);
    if (ctx->states.empty()) ea::fail(EAADC_ERR_STATE, "no states built");
    if (nroots < 1 || !opts || !omega) ea::fail(EAADC_ERR_ARG, "bad arguments");
    if (!(opts->tol > 0) || opts->maxit < 1) ea::fail(EAADC_ERR_ARG, "bad Davidson options");
    if (opts->prec != EAADC_FP64 && opts->prec != EAADC_MIXED_BF16 && opts->prec != EAADC_MIXED_BF16X3)
      ea::fail(EAADC_ERR_ARG, "unknown precision");
    if (opts->precond != 0 && opts->precond != 1) ea::fail(EAADC_ERR_ARG, "unknown preconditioner");
    if (opts->refine < 0 || opts->refine > 3) ea::fail(EAADC_ERR_ARG, "refine must be 0..3");
    if (opts->trace < 0 || opts->trace > 10000) ea::fail(EAADC_ERR_ARG, "trace must be in [0, 10000]");
    ea::davidson(ctx, nroots, *opts, omega, resnorm, iters, &conv);
  });
  if (st == EAADC_OK && !conv) {
    ctx->err = "Davidson did not converge within maxit";
    return EAADC_ERR_NOCONV;
  }
  return st;
}

eaadc_status eaadc_get_eigvecs(eaadc_ctx* ctx, int state, double* vec_host) {
  if (!ctx) return EAADC_ERR_ARG;
  return guarded(ctx, [&] {
    set_device(ctx);
    ea::State& st = get_state(ctx, state);
    if (!vec_host) ea::fail(EAADC_ERR_ARG, "NULL output");
    if (!st.nvecs) ea::fail(EAADC_ERR_STATE, "no eigenvectors (run eaadc_davidson first)");
    EA_CK(cudaMemcpyAsync(vec_host, st.evecs.p, sizeof(double) * st.nvecs * st.dim, cudaMemcpyDeviceToHost,
                          ctx->stream));
    EA_CK(cudaStreamSynchronize(ctx->stream));
  });
}

void eaadc_destroy(eaadc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  delete ctx;
  cudaStreamSynchronize(s);
}

const char* eaadc_last_error(const eaadc_ctx* ctx) {
  if (!ctx) return g_static_err.c_str();
  return ctx->err.c_str();
}

}  // extern "C"
