// Internal declarations of the EA-ADC library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>
#include <vector>
#include <initializer_list>
#include "eaadc.h"

namespace ea {

struct Error {
  eaadc_status st;
  std::string msg;
};

[[noreturn]] void fail(eaadc_status st, const std::string& msg);

#define EA_CK(x)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (x);                                                                \
    if (e_ != cudaSuccess)                                                               \
      ::ea::fail(EAADC_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_) +       \
                                     " at " + __FILE__ + ":" + std::to_string(__LINE__)); \
  } while (0)

// Counts every kernel launched by this library (instrumentation).
extern long long g_kernel_launches;
#define EA_LAUNCH()                                             \
  do {                                                          \
    __atomic_add_fetch(&::ea::g_kernel_launches, 1, __ATOMIC_RELAXED); \
    EA_CK(cudaGetLastError());                                  \
  } while (0)

// ------------------------------------------------------------ device memory
// Stream-ordered device array owned by its creator.
template <class T>
struct DArr {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DArr() = default;
  DArr(size_t n_, cudaStream_t s_) { alloc(n_, s_); }
  void alloc(size_t n_, cudaStream_t s_) {
    release();
    n = n_;
    s = s_;
    if (n) {
      cudaError_t e = cudaMallocAsync((void**)&p, n * sizeof(T), s);
      if (e != cudaSuccess) {
        p = nullptr;
        n = 0;
        cudaGetLastError();
        fail(EAADC_ERR_ALLOC, "device allocation of " + std::to_string(n_ * sizeof(T)) + " bytes failed");
      }
    }
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  ~DArr() { release(); }
  DArr(const DArr&) = delete;
  DArr& operator=(const DArr&) = delete;
  DArr(DArr&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  DArr& operator=(DArr&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
    return *this;
  }
};

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------- FP64 toolkit
// Row-major GEMM on CUDA cores: C = alpha * op(A) * op(B) + beta * C, op(X) = X
// or X^T.  A is M x K (or K x M if ta) with row stride lda; B is K x N (or N x K
// if tb).  Two-level batch: batch index z = z1 * nb2 + z2 adds z1*s?1 + z2*s?2.
// T is double (the FP64 path) or float (DF pieces of the mixed path).
struct GemmBatch {
  int nb1 = 1, nb2 = 1;
  long long sA1 = 0, sA2 = 0, sB1 = 0, sB2 = 0, sC1 = 0, sC2 = 0;
};
template <class T>
void gemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, long long lda, const T* B,
          long long ldb, T beta, T* C, long long ldc, const GemmBatch& bt);
inline void dgemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha, const double* A, long long lda,
                  const double* B, long long ldb, double beta, double* C, long long ldc,
                  const GemmBatch& bt = GemmBatch()) {
  gemm<double>(s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt);
}

// dst = alpha * permute(src) + beta * dst; src has dims sdims, dst axis i is src axis perm[i].
template <class T>
void permuteT(cudaStream_t s, const T* src, const std::vector<int>& sdims, const std::vector<int>& perm, T* dst,
              T alpha, T beta);
inline void permute(cudaStream_t s, const double* src, const std::vector<int>& sdims, const std::vector<int>& perm,
                    double* dst, double alpha = 1.0, double beta = 0.0) {
  permuteT<double>(s, src, sdims, perm, dst, alpha, beta);
}

// out[.., b, c] = alpha * (c1 * in[.., b, c] + c2 * in[.., c, b]) + beta * out[.., b, c]
// for `nmat` consecutive v x v matrices with strides (in_stride, out_stride).
template <class T>
void pair_combineT(cudaStream_t s, const T* in, long long in_stride, T* out, long long out_stride, int nmat, int v,
                   T c1, T c2, T alpha, T beta);
inline void pair_combine(cudaStream_t s, const double* in, long long in_stride, double* out, long long out_stride,
                         int nmat, int v, double c1, double c2, double alpha, double beta) {
  pair_combineT<double>(s, in, in_stride, out, out_stride, nmat, v, c1, c2, alpha, beta);
}

template <class T>
void fillT(cudaStream_t s, T* p, size_t n, T val);
template <class T>
void axpbyT(cudaStream_t s, size_t n, T a, const T* x, T b, T* y);  // y = a x + b y
inline void fill(cudaStream_t s, double* p, size_t n, double val) { fillT<double>(s, p, n, val); }
inline void axpby(cudaStream_t s, size_t n, double a, const double* x, double b, double* y) {
  axpbyT<double>(s, n, a, x, b, y);
}

// Two-operand tensor contraction (einsum without batch labels).
template <class T>
struct TensT {
  T* p;
  std::vector<int> dims;
  size_t size() const { size_t n = 1; for (int d : dims) n *= (size_t)d; return n; }
};
using Tens = TensT<double>;
template <class T>
void einsumT(cudaStream_t s, const char* spec, T alpha, const TensT<T>& A, const TensT<T>& B, T beta,
             const TensT<T>& C);
inline void einsum(cudaStream_t s, const char* spec, double alpha, const Tens& A, const Tens& B, double beta,
                   const Tens& C) {
  einsumT<double>(s, spec, alpha, A, B, beta, C);
}

// ------------------------------------------------------------- problem data
struct State {
  int o = 0, v = 0, naux = 0;
  long long dim = 0;
  int order = 3;
  double x3 = 1.0;
  int build_prec = EAADC_FP64;  // precision of the pp-ladder of the amplitudes in M^(3)
  DArr<double> eo, ev;            // [o], [v]
  DArr<double> Boo, Bov, Bvv;     // [naux][o][o], [naux][o][v], [naux][v][v]
  DArr<double> tau;               // [o][o][v][v]  (ia|jb)/D
  DArr<double> Kmat, Jmat;        // [(k,b)][(l,d)] = (bd|lk) ; [(k,c)][(l,d)] = (ck|ld)
  DArr<double> M11;               // [v][v]
  DArr<double> diag;              // [dim] Davidson diagonal
  // mixed-precision operands (built lazily)
  DArr<bf16> Bvv_bf, Bb_bf, Kmat_bf, Jmat_bf;  // Bb_bf[b][Q][d] = B^Q_bd
  DArr<bf16> tauA_bf, tauB_bf, tauC_bf, tauD_bf, tm2A_bf, tm2C_bf;  // (ov x ov) coupling operands
  DArr<float> Boo32, Bov32, Bvv32, tau32;     // FP32 copies for the DF coupling pieces
  DArr<bf16> Bvv_lo, Bb_lo, Kmat_lo, Jmat_lo, tauA_lo, tm2A_lo;  // low parts (split-BF16 mode)
  bool x3_ready = false;
  // per-state FNO/NAF data (states from eaadc_build_states)
  DArr<double> ref1p;                          // canonical ADC(2) root's 1p part in this basis [v']
  double omega2_can = 0.0;                     // that canonical ADC(2) root
  int vfull = 0, nauxfull = 0;                 // untruncated sizes
  std::vector<double> omega;                   // roots of the last Davidson
  int target = -1;                             // index of the target root
  // Davidson trace (opts.trace > 0): Ritz vectors, residuals and values per iteration
  DArr<double> trX, trR;
  std::vector<double> trTheta;
  int trN = 0, trK = 0;
  DArr<double> lad_diag;                       // (bb|cc) [v'][v'], a feature of the learned correction
  long long bvv_pitch = 0, bb_pitch = 0;      // row pitches (elements) of Bvv_bf and Bb_bf
  DArr<int> err;                              // device error word of bounded waits
  bool mixed_ready = false;
  // last Davidson solution
  DArr<double> evecs;             // [nroots][dim]
  int nvecs = 0;
};

// Learned Davidson correction: per-element MLP (16 features -> 3 x 256 tanh
// -> 1), FP32 master weights with Adam moments, flat layout
// W1[256][16] b1 W2[256][256] b2 W3[256][256] b3 w4[256] b4.
constexpr int kMlpF = 16, kMlpW = 256;
constexpr long long kMlpParams = 136193;
struct Mlp {
  DArr<float> w, g, mom, vel;
  int step = 0;
  bool ready = false;
};
// m[i] = MLP(feat[i]) for n rows (activations allocated on s).
void mlp_forward(cudaStream_t s, const Mlp& net, long long n, const float* feat, float* m);
// Features, normalised residual rr and diagonal term base = rr / (theta - D)
// of nvec residual vectors R (rows of length st.dim) with Ritz values theta.
void precond_features(cudaStream_t s, State& st, int nvec, const double* R, const double* theta_dev,
                      const double* rnorm_dev, float* feat, float* rr, float* base);
void precond_pairs(cudaStream_t s, State& st, int nvec, const double* Y, const double* R,
                   const double* theta_host, const double* Ys, float* feat, float* rr, float* base, float* T);
double mlp_loss_grad(cudaStream_t s, Mlp& net, int nseg, const int* segs_host, const float* feat, const float* rr,
                     const float* base, const float* T, float lr, bool update);
void mlp_load(cudaStream_t s, Mlp& net, const float* host);

}  // namespace ea

struct eaadc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int o = 0, v = 0, naux = 0;
  ea::DArr<double> eo, ev, Boo, Bov, Bvv;
  std::vector<ea::State*> states;
  ea::Mlp mlp;
  int build_prec = EAADC_FP64;  // for the states built next (eaadc_set_build_precision)
  std::string err;
  ~eaadc_ctx();
};

namespace ea {
void build_state_intermediates(eaadc_ctx* ctx, State& st);
// out[m] (FP64 [v][v], stride v*v) = sum_Q B^Q T[m] B^Q for nmat matrices T
// (FP64 [v][v]) on the tensor cores (BF16, or split BF16 when x3).
void ladder_pairs_tc(cudaStream_t s, State& st, const double* T, int nmat, bool x3, double* out);
void sigma_fp64(cudaStream_t s, State& st, int nvec, const double* x, double* y);
void sigma_mixed(cudaStream_t s, State& st, int nvec, const double* x, double* y, bool x3);
void sigma_base_fp64(cudaStream_t s, State& st, int nvec, const double* x, double* y, bool ring, bool ladder);
void check_device_error(cudaStream_t s, State& st);
void diag_and_m11(cudaStream_t s, State& st, int nvec, const double* x, double* y);
template <class T>
struct CoupOps {
  int o, v, naux, order;
  const T *Boo, *Bov, *Bvv, *tau;
};
template <class T>
void couple12(cudaStream_t s, const CoupOps<T>& c, const T* y, T* outA, const T* tm2, bool big, T* Fo, T* Go);
template <class T>
void couple21(cudaStream_t s, const CoupOps<T>& c, const T* V, T* sy, const T* tm2, const T* H1g, const T* H2g,
              const T* H3g);
void couple_1p_to_2p1h(cudaStream_t s, State& st, const double* y, double* outA, const double* tm2, bool big,
                       double* Fo, double* Go);
void couple_2p1h_to_1p(cudaStream_t s, State& st, const double* V, double* sy, const double* tm2,
                       const double* H1g, const double* H2g, const double* H3g);
void ladder_only(cudaStream_t s, State& st, int nvec, const double* x, float* out, bool mixed);
void make_diagonal(cudaStream_t s, State& st);
// Lowest nroots roots of one state (Ritz vectors into st.evecs, values into
// st.omega); returns true if converged.
bool davidson_state(cudaStream_t s, State& st, int nroots, const eaadc_davidson_opts& opt, double* omega,
                    double* resnorm, int* iters, const Mlp* mlp = nullptr);
// Target root of an FNO state: largest |overlap| of the 1p part with ref1p.
void pick_target(cudaStream_t s, State& st);
// Per-state FNO/NAF truncated states replacing ctx->states (Sec. III) and
// the Eq. 30 energies of the target roots.
void build_fno_states(eaadc_ctx* ctx, int nstates, const double* fno_thr, const double* naf_thr, int order, double x3,
                      const eaadc_davidson_opts& copts);
void ea_energies(eaadc_ctx* ctx, const eaadc_davidson_opts& opts, double* w_uncorr, double* w_corr, double* w2_can,
                 double* w2_fno);
void davidson(eaadc_ctx* ctx, int nroots, const eaadc_davidson_opts& opt, double* omega,
              double* resnorm, int* iters, bool* converged);
// Dense symmetric eigensolver (cyclic Jacobi, one CTA per matrix, m <= 96):
// nbatch matrices A [m][m] (read only), eigenvalues ascending into w[m],
// eigenvectors as columns of U [m][m].
void jacobi_eigh(cudaStream_t s, int m, double* A, double* w, double* U, int nbatch = 1);
// Dense symmetric eigensolver of any order n (FP64, two-sided block Jacobi):
// A [n][n] on the device (read only), eigenvalues ascending into w[n],
// eigenvectors as columns of V [n][n].
void eigh_sym(cudaStream_t s, int n, const double* A, double* w, double* V);
}  // namespace ea
