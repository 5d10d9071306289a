/*
 * eaadc.h - C ABI of the GB300 (sm_103a) DF-EA-ADC(3) sigma/Davidson library.
 *
 * Method: non-Dyson EA-ADC(n) in the intermediate-state representation
 * (arXiv:2511.05897, Sec. II.A, Eq. 1-6), truncated by perturbation order
 * (Eq. 5), with density-fitted integrals (pq|rs) = sum_Q B^Q_pq B^Q_rs
 * (Sec. II.B, Eq. 25), state-specific frozen natural orbitals (Sec. II.C,
 * Eq. 9-17), natural auxiliary functions (Sec. II.D, Eq. 27-29) and the
 * perturbative truncation correction (Sec. II.E, Eq. 30).  The secular matrix
 * M is diagonalised by Davidson's method from sigma vectors sigma = M c
 * (Sec. II.A, last paragraph).
 *
 * Conventions for every entry point:
 *  - Every call returns an eaadc_status and never aborts; on failure
 *    eaadc_last_error(ctx) holds a one-line message (valid until the next call
 *    on that context).
 *  - Host arrays are owned by the caller and only read (or written, for
 *    outputs) during the call.
 *  - Device buffers passed to eaadc_sigma are owned by the caller; all other
 *    device memory is owned by the context and freed by eaadc_destroy.
 *  - A context is bound to one CUDA device; calls on one context must not run
 *    concurrently (thread-compatible, not thread-safe).
 *  - Device memory is taken from the stream-ordered allocator on the stream
 *    of the call; state buffers made during a call (the reduced-precision
 *    operand copies on the first such call, the learned-correction feature
 *    table) stay with the context and are released on that stream by
 *    eaadc_destroy: a stream passed to a call must outlive the context.
 *  - Vector layout of one attached-state vector of state s (dimension
 *    dim = v' + o*v'*v'): [1p part y[a], a < v'] followed by the 2p1h part
 *    w[k][b][c] (k < o, b, c < v', c fastest) in the orthonormal doublet
 *    representation: sym(w) in (b,c) is the pair-singlet and antisym(w) the
 *    pair-triplet coupled doublet, so M is symmetric.
 *  - Energies are in hartree; attachment energies omega, EA = -omega.
 */
#ifndef EAADC_H
#define EAADC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eaadc_ctx eaadc_ctx;

typedef enum {
  EAADC_OK = 0,
  EAADC_ERR_ARG = -1,       /* invalid argument (sizes, pointers, state index) */
  EAADC_ERR_ALLOC = -2,     /* device or host allocation failed */
  EAADC_ERR_CUDA = -3,      /* a CUDA runtime call or kernel failed */
  EAADC_ERR_NOCONV = -4,    /* Davidson reached maxit without convergence */
  EAADC_ERR_NONFINITE = -5, /* NaN/Inf in an input, sigma or residual */
  EAADC_ERR_TIMEOUT = -6,   /* a bounded device wait expired */
  EAADC_ERR_STATE = -7      /* call out of order (e.g. sigma before build) */
} eaadc_status;

typedef enum {
  EAADC_FP64 = 0,        /* every operation in FP64 */
  EAADC_MIXED_BF16 = 1,  /* every o*v^3 contraction (DF ladder, ring, second-
                            order coupling) on tcgen05 tensor cores with BF16
                            operands and FP32 accumulation; DF coupling pieces
                            in FP32, diagonal and 1p/1p block in FP64 */
  EAADC_MIXED_BF16X3 = 2 /* as EAADC_MIXED_BF16 with each tensor-core operand
                            split into two BF16 parts and three products
                            (about 16 significant bits, 3x the tensor work) */
} eaadc_prec;

typedef struct {
  double tol;     /* converged when every residual 2-norm <= tol ... */
  double etol;    /* ... and every Ritz value moved by <= etol */
  int maxit;      /* iteration limit */
  int max_sub;    /* subspace size limit per state (<= 96) */
  int prec;       /* eaadc_prec used for the sigma vectors inside the loop; a
                     reduced-precision phase stops at its noise floor (largest
                     residual shrinking by less than 2x in 8 iterations) */
  int refine;     /* after a reduced-precision phase (which stops at tol or at
                     its noise floor): 1 = FP64 Davidson iterations from its
                     Ritz vectors until tol is met in FP64; 2 = one FP64 sigma
                     of the Ritz vectors and a Rayleigh-Ritz step in their
                     span (Ritz values exact to second order in the error of
                     the vectors; resnorm reports the FP64 residuals); 3 = as
                     2 with the split-BF16 sigma (EAADC_MIXED_BF16X3, about
                     1e-5 relative) instead of FP64 */
  int precond;    /* 0: diagonal correction r/(theta - D); 1: learned
                     correction (weights from eaadc_precond_load), falling
                     back to the diagonal one, for the rest of the solve, for
                     a root whose residual norm grew after a learned step */
  int trace;      /* record the Ritz vectors, residuals and Ritz values of the
                     first `trace` iterations of each state (eaadc_get_trace);
                     0: none */
} eaadc_davidson_opts;

/* Library version string (static storage). */
const char* eaadc_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (instrumentation for benchmarks; the paper has no counterpart). */
long long eaadc_kernel_launches(void);

/* Create a context on `device` and upload the canonical problem.
 *  o, v, naux : occupied, virtual and auxiliary sizes (o >= 1, v >= 1, naux >= 1)
 *  eps_occ    : host [o] occupied orbital energies
 *  eps_vir    : host [v] virtual orbital energies
 *  B          : host [naux][o+v][o+v] row-major DF factor B^Q_pq in the MO
 *               basis (the paper's J^Q_pq of Eq. 26), symmetric in (p,q);
 *               only the oo, ov and vv blocks are read.
 *  stream     : cudaStream_t used for all internal work (NULL = legacy default)
 * Eq. 25 defines (pq|rs) from B.  On success *out owns device copies. */
eaadc_status eaadc_init(eaadc_ctx** out, int o, int v, int naux,
                        const double* eps_occ, const double* eps_vir, const double* B,
                        int device, void* stream);

/* Build one untruncated (canonical) state: state 0 uses the full virtual and
 * auxiliary spaces.  adc_order is 2 or 3; x3 scales the third-order 1p/1p
 * block (1.0 = ADC(3)).  Computes the first-order amplitudes, the 1p/1p block
 * through order adc_order and the stored (oo|vv) and (ov|ov) integrals. */
eaadc_status eaadc_build_canonical(eaadc_ctx* ctx, int adc_order, double x3);

/* Number of built states and the dimensions of state s. */
eaadc_status eaadc_state_info(const eaadc_ctx* ctx, int state, int* vprime, int* nauxprime,
                              long long* dim);

/* sigma = M x for nvec vectors of state `state`.
 *  x_dev, sigma_dev : caller-owned device buffers [nvec][dim] (FP64), must not
 *                     overlap; used on `stream` (cudaStream_t, NULL = legacy).
 *  prec             : eaadc_prec. */
eaadc_status eaadc_sigma(eaadc_ctx* ctx, int state, int nvec, const double* x_dev,
                         double* sigma_dev, int prec, void* stream);

/* In the reduced-precision modes, the first call for a given (state size,
 * nvec) shape also times the candidate chunk sizes of the ladder (each run
 * computes the full result) and keeps the fastest for later calls; that
 * first call waits for the stream.  The same holds for eaadc_ladder. */

/* Same as eaadc_sigma with host buffers [nvec][dim]; includes the copies. */
eaadc_status eaadc_sigma_host(eaadc_ctx* ctx, int state, int nvec, const double* x_host,
                              double* sigma_host, int prec);

/* The particle-particle ladder term alone (Sec. II.B: the four-virtual
 * integrals (bd|ce) = sum_Q B^Q_bd B^Q_ce are applied as two successive DF
 * contractions and never stored):
 *   out[n][k][c][b] = sum_Q sum_de B^Q_bd w_n[k][d][e] B^Q_ce
 * (note the transposed (c, b) order of the output) on the BF16/FP32
 * tensor-core path.
 *  x_dev   : device [nvec][dim] FP64 vectors (only their 2p1h parts are read)
 *  out_dev : device [nvec][o][v'][v'] FP32, caller-owned, overwritten
 *  stream  : cudaStream_t for the launches.  ADC(3) states only. */
eaadc_status eaadc_ladder(eaadc_ctx* ctx, int state, int nvec, const double* x_dev, float* out_dev,
                          void* stream);

/* Size in bytes of the one fixed device array that eaadc_ladder_noalloc works
 * in.  Every GPU that loads this library holds it until the process exits. */
#define EAADC_LADDER_NOALLOC_SCRATCH_BYTES (32u << 20)

/* eaadc_ladder that allocates no device memory.  The paper has no counterpart:
 * this is a service to callers that cannot allocate at the point of the call.
 * eaadc_ladder takes its working memory from the stream-ordered allocator on
 * every call; a process whose device memory already belongs to its own memory
 * manager (a framework's caching allocator, a server that reserves HBM at
 * start-up) may see that fail or force its manager to give memory back, and a
 * cudaFree synchronises the whole device, stalling the caller's other streams.
 * This entry point instead works in one fixed array of
 * EAADC_LADDER_NOALLOC_SCRATCH_BYTES and calls no allocator.
 *
 * Arguments, output layout and arithmetic are those of eaadc_ladder (the sum
 * over auxiliary functions is cut into blocks that fit the array, so results
 * agree with it to FP32 rounding).  out_dev must be 16-byte aligned.
 *
 * Limit: with r64(n) = n rounded up to a multiple of 64, the BF16 copy of the
 * 2p1h vectors (nvec*o*v'*r64(v')*2 bytes), for v' not a multiple of 4 an FP32
 * copy of the result (about nvec*o*v'*v'*4 bytes), and the intermediate of one
 * auxiliary function (nvec*o*v'*r64(pad8(v'))*2 bytes) must fit in the array;
 * larger nvec is rejected with EAADC_ERR_ARG and the sizes in
 * eaadc_last_error (o=20, v'=200 allows up to 8 vectors per call).
 *
 * Preconditions: the state's BF16 operands must exist; the first eaadc_ladder
 * or reduced-precision eaadc_sigma on the state makes them (those calls do
 * allocate).  Otherwise EAADC_ERR_STATE.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (with that device current) and keeps it.  Make that first call before any
 * stream capture on the device.
 *
 * Sharing: all calls on one device, from any context or thread, use the same
 * array, and it keeps what the last call left there; each call clears the
 * parts that must start at zero.  Calls whose GPU work can overlap (different
 * streams or contexts with no ordering between them) race on the array and
 * give wrong results: order them on one stream or with events. */
eaadc_status eaadc_ladder_noalloc(eaadc_ctx* ctx, int state, int nvec, const double* x_dev,
                                  float* out_dev, void* stream);

/* Davidson diagonal preconditioner values D (host [dim]): D_a = M_aa for the
 * 1p part, e_b + e_c - e_k for the 2p1h part. */
eaadc_status eaadc_diagonal(eaadc_ctx* ctx, int state, double* diag_host);

/* Precision of the pp-ladder of the first-order amplitudes inside M^(3)
 * (sum_Q B^Q tau_ij B^Q over the o^2 pairs, 4 o^2 v^3 naux flop: the largest
 * cost of building a state) for the states built next by
 * eaadc_build_canonical or eaadc_build_states: EAADC_FP64 (the default), or
 * the tensor-core ladder in EAADC_MIXED_BF16 or EAADC_MIXED_BF16X3 (about
 * 1e-5 relative; the state's reduced-precision operands are made then too).
 * Everything else in the build stays FP64. */
eaadc_status eaadc_set_build_precision(eaadc_ctx* ctx, int prec);

/* Per-state truncated spaces (Sec. II.C-E; the algorithm of Sec. III),
 * replacing any states built before.  Solves the canonical EA-ADC(2) problem
 * for its nstates lowest roots (FP64 Davidson with can_opts, or tol 1e-8,
 * maxit 300, max_sub 40 when NULL); root k defines state k:
 *   D^SS(k) = D^MP2 + D^EA(k) (Eq. 17; D^EA from the zeroth-order ISR of the
 *   root: y_a y_b + sum_kc (w_kac w_kbc + w_kca w_kcb), spin-summed),
 *   eigenvectors with occupation > fno_thresh[k] kept (Eq. 9-11; < 0 keeps
 *   all), semicanonicalised (Eq. 12-14); the DF factor transformed to that
 *   basis; W = J J^T over its vv block (Eq. 27-28), eigenvectors with
 *   eigenvalue >= naf_thresh[k] kept (< 0 keeps all), J~ = N~^T J (Eq. 29)
 *   for the oo, ov and vv blocks; then the ADC(adc_order) intermediates of
 *   the truncated problem, with x3 scaling M^(3) as in eaadc_build_canonical.
 * All eigenproblems run on the device (eaadc_eigh_sym).  eaadc_state_info
 * gives each state's v' and naux'; eaadc_davidson then solves every state and
 * records its target root: the Ritz vector whose 1p part overlaps most with
 * the canonical root's 1p part carried into the FNO basis (ties: lower root).
 *  fno_thresh, naf_thresh : host [nstates]
 * Errors: EAADC_ERR_ARG for a threshold that keeps nothing, EAADC_ERR_NOCONV
 * if the canonical roots do not converge. */
eaadc_status eaadc_build_states(eaadc_ctx* ctx, int nstates, const double* fno_thresh,
                                const double* naf_thresh, int adc_order, double x3,
                                const eaadc_davidson_opts* can_opts);

/* Eq. 30 for every state from eaadc_build_states, after eaadc_davidson:
 *   omega_corr = omega^(3)_FNO + omega^(2)_canonical - omega^(2)_FNO,
 * omega^(3)_FNO the target root of the last eaadc_davidson, omega^(2)_FNO the
 * target root of EA-ADC(2) solved here in the same truncated space (FP64
 * Davidson with opts, defaults as for eaadc_build_states; as many roots as the
 * last eaadc_davidson, and at least k + 2 for state k, whose canonical root is
 * the (k+1)-th).  Attachment energies in hartree (EA = -omega).
 * Each output is host [nstates] and may be NULL. */
eaadc_status eaadc_ea_energies(eaadc_ctx* ctx, const eaadc_davidson_opts* opts, double* omega_uncorr,
                               double* omega_corr, double* omega2_can, double* omega2_fno);

/* Dense FP64 symmetric eigensolver used for the FNO and NAF bases (Eq. 9, 13,
 * 28): a_dev [n][n] device, read only (its symmetric part is used);
 * eigenvalues ascending into w_dev [n], eigenvectors as the columns of v_dev
 * [n][n] (row-major).  Two-sided block Jacobi (32 x 32 blocks, pair
 * sub-problems solved in shared memory); n <= 96 in one CTA.  Works on the
 * given device and stream; allocates its own temporary device memory. */
eaadc_status eaadc_eigh_sym(int n, const double* a_dev, double* w_dev, double* v_dev, int device,
                            void* stream);

/* ---------------------------------------------- learned Davidson correction
 * Not in the paper: a per-element network that adds to the diagonal
 * correction.  For a root with Ritz value theta and residual r, element I of
 * the expansion vector is rr_I (1/(theta - D_I) + m_I), rr = r/||r||, D the
 * diagonal of eaadc_diagonal (|theta - D_I| >= 1e-8), m_I = MLP(f_I):
 *   h1 = tanh(W1 f + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3),
 *   m = w4 . h3 + b4   (width 256, FP32 on the device)
 * with the 16 features f_I (rr_I sqrt(dim), asinh(D_I - theta),
 * clip(1/(theta - D_I), +-100)/100, eps_k, asinh(eps_b) (1p: asinh(eps_a)),
 * asinh(eps_c), theta, log10 ||r||, [1p], [2p1h with b = c], (bb|cc) = the
 * ladder diagonal for 2p1h, 5 zeros).
 * Weights: EAADC_MLP_PARAMS floats, W1[256][16] b1[256] W2[256][256] b2
 * W3[256][256] b3 w4[256] b4[1].  Training minimises the mean over vectors of
 * 1 - cos^2(delta, t), t = (I - y y^T)(y* - y) the exact correction of the
 * Ritz vector y towards the converged eigenvector y* (sign-aligned). */
#define EAADC_MLP_FEATURES 16
#define EAADC_MLP_PARAMS 136193

/* Load (host FP32, bytes = 4 * EAADC_MLP_PARAMS) the network used by
 * eaadc_davidson when opts.precond = 1; resets the Adam moments. */
eaadc_status eaadc_precond_load(eaadc_ctx* ctx, const float* weights, size_t bytes);
/* Copy the current weights to the host. */
eaadc_status eaadc_precond_get(eaadc_ctx* ctx, float* weights, size_t bytes);

/* Training pairs for nvec Ritz vectors of a state: y_dev, r_dev device
 * [nvec][dim] FP64 (Ritz vectors, residuals), theta_host [nvec]; ystar_dev
 * [nvec][dim] the converged eigenvectors of the same roots (or NULL, then
 * target_dev must be NULL too).  Outputs (device FP32, row = (vector,
 * element)): feat_dev [nvec*dim][16], rr_dev and base_dev [nvec*dim] (rr and
 * rr/(theta - D)), target_dev [nvec*dim]. */
eaadc_status eaadc_precond_pairs(eaadc_ctx* ctx, int state, int nvec, const double* y_dev,
                                 const double* r_dev, const double* theta_host, const double* ystar_dev,
                                 float* feat_dev, float* rr_dev, float* base_dev, float* target_dev,
                                 void* stream);

/* m_dev[i] = MLP(feat_dev[i]) for n rows (device FP32). */
eaadc_status eaadc_mlp_forward(eaadc_ctx* ctx, long long n, const float* feat_dev, float* m_dev, void* stream);

/* Loss and gradient of a batch of nseg vectors: rows seg_host[j] ..
 * seg_host[j+1]-1 (seg_host host [nseg+1], seg_host[0] = 0, increasing) of
 * the device arrays from eaadc_precond_pairs.  loss_host (may be NULL) gets
 * the mean loss, grad_host (may be NULL) the EAADC_MLP_PARAMS gradient. */
eaadc_status eaadc_mlp_loss_grad(eaadc_ctx* ctx, int nseg, const int* seg_host, const float* feat_dev,
                                 const float* rr_dev, const float* base_dev, const float* target_dev,
                                 double* loss_host, float* grad_host, void* stream);

/* As eaadc_mlp_loss_grad, then one Adam step (beta 0.9/0.999, eps 1e-8) with
 * learning rate lr on the loaded weights. */
eaadc_status eaadc_mlp_train_step(eaadc_ctx* ctx, int nseg, const int* seg_host, const float* feat_dev,
                                  const float* rr_dev, const float* base_dev, const float* target_dev,
                                  float lr, double* loss_host, void* stream);

/* The trace of the last eaadc_davidson with opts.trace > 0: *niters
 * iterations of *nroots roots; x_host, r_host [niters][nroots][dim] (Ritz
 * vectors, residuals), theta_host [niters][nroots].  Pointers may be NULL
 * (query the sizes first). */
eaadc_status eaadc_get_trace(eaadc_ctx* ctx, int state, int* niters, int* nroots, double* x_host,
                             double* r_host, double* theta_host);

/* Copy the 1p/1p block M_ab of a state to host [v'][v']. */
eaadc_status eaadc_get_m11(eaadc_ctx* ctx, int state, double* m11_host);

/* Number of states currently built (0 for ctx == NULL). */
int eaadc_num_states(const eaadc_ctx* ctx);

/* Lowest nroots roots of every built state by Davidson.
 *  omega   : host [nstates][nroots] Ritz values (hartree)
 *  resnorm : host [nstates][nroots] final residual 2-norms (may be NULL)
 *  iters   : host [nstates] iterations used (may be NULL)
 * Returns EAADC_ERR_NOCONV (with results filled) if maxit was reached. */
eaadc_status eaadc_davidson(eaadc_ctx* ctx, int nroots, const eaadc_davidson_opts* opts,
                            double* omega, double* resnorm, int* iters);

/* Converged eigenvectors of state s from the last eaadc_davidson, host
 * [nroots][dim]. */
eaadc_status eaadc_get_eigvecs(eaadc_ctx* ctx, int state, double* vec_host);

/* Free everything owned by the context (NULL is ignored). */
void eaadc_destroy(eaadc_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); static for ctx==NULL. */
const char* eaadc_last_error(const eaadc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* EAADC_H */
