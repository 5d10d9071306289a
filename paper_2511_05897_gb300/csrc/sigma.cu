// sigma = M x for restricted EA-ADC(2)/(3) in the orthonormal doublet
// representation (FP64 path).
//
// With W the 2p1h part and S(Z) = sym(Z) + sqrt(3) antisym(Z) over (b, c):
//   sigma_1p   = M11 y + sum_kbc C_A[k,b,c,a] S(W)[k,b,c]
//   sigma_2p1h = (e_b + e_c - e_k) W + S(C_A y)
//              + sum_Q B^Q W_k B^Q                        (pp ladder, ADC(3))
//              + S(ring_A(S^-1 W))                         (ph terms, ADC(3))
// C_A is the 1p/2p1h coupling on the alpha-beta-beta determinant block:
// first order (ab|kc); second order from tau and integrals with three
// virtual indices, evaluated through B^Q (Sec. II.B: three- and four-virtual
// integrals are built on the fly).
#include "internal.cuh"

#include <cmath>

namespace ea {

void ladder_fp64(cudaStream_t s, const double* Bvv, int naux, int v, const double* T, long long tstride,
                 int nb1, long long tstride1, int nb2, double* out, long long ostride1, long long ostride2,
                 double alpha, double beta);

namespace {
const double kS1 = 0.5 * (1.0 + 1.7320508075688772935);   // S: c1
const double kS2 = 0.5 * (1.0 - 1.7320508075688772935);   // S: c2
const double kI1 = 0.5 * (1.0 + 0.57735026918962576451);  // S^-1: c1
const double kI2 = 0.5 * (1.0 - 0.57735026918962576451);  // S^-1: c2

// y[n][v + (k,b,c)] = (e_b + e_c - e_k) x[n][v + (k,b,c)]
__global__ void diag2p1h_kernel(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ eo,
                                const double* __restrict__ ev, int o, int v, long long dim, int nvec) {
  long long n2 = (long long)o * v * v;
  long long total = n2 * nvec;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long n = idx / n2, r = idx % n2;
    int c = r % v;
    long long q = r / v;
    int b = q % v;
    int k = (int)(q / v);
    long long off = n * dim + v + r;
    y[off] = (ev[b] + ev[c] - eo[k]) * x[off];
  }
}

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }
}  // namespace

// out (A-representation, [o][v][v]) = sum_a C_A[k,b,c,a] y_a.
// big = false skips the three o^2 v^3 tau contractions and instead returns the
// DF intermediates F[l][c][d] = sum_a (al|cd) y_a and G[b][l][d] = sum_a (ab|ld) y_a
// (when Fo/Go are given) for the tensor-core path.
template <class T>
void couple12(cudaStream_t s, const CoupOps<T>& c, const T* y, T* outA, const T* tm2, bool big, T* Fo, T* Go) {
  const int o = c.o, v = c.v, naux = c.naux;
  using TT = TensT<T>;
  TT Bov{(T*)c.Bov, {naux, o, v}}, Bvv{(T*)c.Bvv, {naux, v, v}}, Boo{(T*)c.Boo, {naux, o, o}};
  TT yt{(T*)y, {v}};
  TT out{outA, {o, v, v}};
  DArr<T> Qy((size_t)naux * v, s);
  TT Qyt{Qy.p, {naux, v}};
  einsumT<T>(s, "Qba,a->Qb", T(1), Bvv, yt, T(0), Qyt);  // B^Q symmetric
  einsumT<T>(s, "Qb,Qkc->kbc", T(1), Qyt, Bov, T(0), out);
  if (c.order < 3) return;
  TT tau{(T*)c.tau, {o, o, v, v}};
  DArr<T> Qo((size_t)naux * o, s), F, G, H((size_t)o * o * o, s);
  T* Fp = Fo;
  T* Gp = Go;
  if (!Fp) { F.alloc((size_t)o * v * v, s); Fp = F.p; }
  if (!Gp) { G.alloc((size_t)o * v * v, s); Gp = G.p; }
  TT Qot{Qo.p, {naux, o}}, Ft{Fp, {o, v, v}}, Gt{Gp, {v, o, v}}, Ht{H.p, {o, o, o}};
  einsumT<T>(s, "Qla,a->Ql", T(1), Bov, yt, T(0), Qot);
  einsumT<T>(s, "Ql,Qcd->lcd", T(1), Qot, Bvv, T(0), Ft);
  einsumT<T>(s, "Qb,Qld->bld", T(1), Qyt, Bov, T(0), Gt);
  einsumT<T>(s, "Ql,Qkm->lkm", T(1), Qot, Boo, T(0), Ht);
  einsumT<T>(s, "lkm,lmbc->kbc", T(1), Ht, tau, T(1), out);
  if (!big) return;
  einsumT<T>(s, "lcd,lkbd->kbc", T(-1), Ft, tau, T(1), out);
  einsumT<T>(s, "bld,lkcd->kbc", T(-1), Gt, TT{(T*)tm2, {o, o, v, v}}, T(1), out);
  einsumT<T>(s, "lbd,lkdc->kbc", T(-1), Ft, tau, T(1), out);
}

// sy[a] += sum_kbc C_A[k,b,c,a] V[k,b,c].  With H1..H3 given (tensor-core
// path) the three o^2 v^3 contractions H1[l][d][c] = sum_kb t_lk^bd V_kbc,
// H2[b][l][d] = sum_kc (t_lk^cd - 2 t_lk^dc) V_kbc, H3[l][b][d] = sum_kc t_lk^dc V_kbc
// are taken from them instead of being formed here.
template <class T>
void couple21(cudaStream_t s, const CoupOps<T>& c, const T* V, T* sy, const T* tm2, const T* H1g, const T* H2g,
              const T* H3g) {
  const int o = c.o, v = c.v, naux = c.naux;
  using TT = TensT<T>;
  TT Bov{(T*)c.Bov, {naux, o, v}}, Bvv{(T*)c.Bvv, {naux, v, v}}, Boo{(T*)c.Boo, {naux, o, o}};
  TT Vt{(T*)V, {o, v, v}};
  TT out{sy, {v}};
  DArr<T> g((size_t)naux * v, s);
  TT gt{g.p, {naux, v}};
  einsumT<T>(s, "Qkc,kbc->Qb", T(1), Bov, Vt, T(0), gt);
  einsumT<T>(s, "Qba,Qb->a", T(1), Bvv, gt, T(1), out);  // B^Q symmetric
  if (c.order < 3) return;
  TT tau{(T*)c.tau, {o, o, v, v}};
  DArr<T> H, tt((size_t)naux * o, s), t2q((size_t)naux * v, s), H4((size_t)o * o * o, s);
  TT ttt{tt.p, {naux, o}}, t2qt{t2q.p, {naux, v}};
  const bool ext = H1g != nullptr;
  if (!ext) H.alloc((size_t)o * v * v, s);
  TT H1t{ext ? (T*)H1g : H.p, {o, v, v}};
  if (!ext) einsumT<T>(s, "lkbd,kbc->ldc", T(1), tau, Vt, T(0), H1t);
  einsumT<T>(s, "Qcd,ldc->Ql", T(-1), Bvv, H1t, T(0), ttt);
  TT H2t{ext ? (T*)H2g : H.p, {v, o, v}};
  if (!ext) einsumT<T>(s, "lkcd,kbc->bld", T(1), TT{(T*)tm2, {o, o, v, v}}, Vt, T(0), H2t);
  einsumT<T>(s, "Qld,bld->Qb", T(1), Bov, H2t, T(0), t2qt);
  einsumT<T>(s, "Qba,Qb->a", T(-1), Bvv, t2qt, T(1), out);
  TT H3t{ext ? (T*)H3g : H.p, {o, v, v}};
  if (!ext) einsumT<T>(s, "lkdc,kbc->lbd", T(1), tau, Vt, T(0), H3t);
  einsumT<T>(s, "Qbd,lbd->Ql", T(-1), Bvv, H3t, T(1), ttt);
  TT H4t{H4.p, {o, o, o}};
  einsumT<T>(s, "lmbc,kbc->lkm", T(1), tau, Vt, T(0), H4t);
  einsumT<T>(s, "Qkm,lkm->Ql", T(1), Boo, H4t, T(1), ttt);
  einsumT<T>(s, "Qla,Ql->a", T(1), Bov, ttt, T(1), out);
}

template void couple12<double>(cudaStream_t, const CoupOps<double>&, const double*, double*, const double*, bool,
                               double*, double*);
template void couple12<float>(cudaStream_t, const CoupOps<float>&, const float*, float*, const float*, bool, float*,
                              float*);
template void couple21<double>(cudaStream_t, const CoupOps<double>&, const double*, double*, const double*,
                               const double*, const double*, const double*);
template void couple21<float>(cudaStream_t, const CoupOps<float>&, const float*, float*, const float*, const float*,
                              const float*, const float*);

static CoupOps<double> ops64(State& st) {
  return CoupOps<double>{st.o, st.v, st.naux, st.order, st.Boo.p, st.Bov.p, st.Bvv.p, st.tau.p};
}

void couple_1p_to_2p1h(cudaStream_t s, State& st, const double* y, double* outA, const double* tm2, bool big,
                       double* Fo, double* Go) {
  couple12<double>(s, ops64(st), y, outA, tm2, big, Fo, Go);
}

void couple_2p1h_to_1p(cudaStream_t s, State& st, const double* V, double* sy, const double* tm2,
                       const double* H1g, const double* H2g, const double* H3g) {
  couple21<double>(s, ops64(st), V, sy, tm2, H1g, H2g, H3g);
}

// sigmaW += S(ring_A(S^-1 W)) for one vector; ring_A(A) =
//   -K A(.,.,c) - transpose_bc[ J (A - 2 A^T) + K A^T ]
static void ring_fp64(cudaStream_t s, State& st, const double* W, double* sW) {
  const int o = st.o, v = st.v;
  const long long ov = (long long)o * v, vv = (long long)v * v, n2 = ov * v;
  DArr<double> A((size_t)n2, s), At((size_t)n2, s), Bm((size_t)n2, s), T1((size_t)n2, s), T2((size_t)n2, s);
  pair_combine(s, W, vv, A.p, vv, o, v, kI1, kI2, 1.0, 0.0);
  pair_combine(s, A.p, vv, At.p, vv, o, v, 0.0, 1.0, 1.0, 0.0);
  pair_combine(s, A.p, vv, Bm.p, vv, o, v, 1.0, -2.0, 1.0, 0.0);
  dgemm(s, false, false, (int)ov, v, (int)ov, 1.0, st.Kmat.p, ov, A.p, v, 0.0, T1.p, v);
  dgemm(s, false, false, (int)ov, v, (int)ov, 1.0, st.Jmat.p, ov, Bm.p, v, 0.0, T2.p, v);
  dgemm(s, false, false, (int)ov, v, (int)ov, 1.0, st.Kmat.p, ov, At.p, v, 1.0, T2.p, v);
  // sigma_A = -T1 - T2^T   (reuse A)
  pair_combine(s, T2.p, vv, A.p, vv, o, v, 0.0, -1.0, 1.0, 0.0);
  axpby(s, (size_t)n2, -1.0, T1.p, 1.0, A.p);
  pair_combine(s, A.p, vv, sW, vv, o, v, kS1, kS2, 1.0, 1.0);
}

// Orbital-energy diagonal of the 2p1h block and the 1p/1p block (overwrites y).
void diag_and_m11(cudaStream_t s, State& st, int nvec, const double* x, double* y) {
  const int o = st.o, v = st.v;
  const long long dim = st.dim, n2 = (long long)o * v * v;
  diag2p1h_kernel<<<gridn(n2 * nvec), 256, 0, s>>>(x, y, st.eo.p, st.ev.p, o, v, dim, nvec);
  EA_LAUNCH();
  dgemm(s, false, false, nvec, v, v, 1.0, x, dim, st.M11.p, v, 0.0, y, dim);
}

// All terms except (optionally) the ring and ladder terms, FP64.
void sigma_base_fp64(cudaStream_t s, State& st, int nvec, const double* x, double* y, bool ring, bool ladder) {
  const int o = st.o, v = st.v;
  const long long dim = st.dim, vv = (long long)v * v, n2 = (long long)o * vv;
  diag2p1h_kernel<<<gridn(n2 * nvec), 256, 0, s>>>(x, y, st.eo.p, st.ev.p, o, v, dim, nvec);
  EA_LAUNCH();
  // 1p/1p block (M11 symmetric): sy = Y M11
  dgemm(s, false, false, nvec, v, v, 1.0, x, dim, st.M11.p, v, 0.0, y, dim);
  DArr<double> tm2;
  if (st.order >= 3) {
    // tau_lk^cd - 2 tau_lk^dc
    tm2.alloc((size_t)(n2 * o), s);
    permute(s, st.tau.p, {o, o, v, v}, {0, 1, 3, 2}, tm2.p, -2.0, 0.0);
    axpby(s, (size_t)(n2 * o), 1.0, st.tau.p, 1.0, tm2.p);
  }
  DArr<double> V((size_t)n2, s), CA((size_t)n2, s);
  for (int n = 0; n < nvec; ++n) {
    const double* xn = x + n * dim;
    double* yn = y + n * dim;
    // 2p1h -> 1p with V = S(W)
    pair_combine(s, xn + v, vv, V.p, vv, o, v, kS1, kS2, 1.0, 0.0);
    couple_2p1h_to_1p(s, st, V.p, yn, tm2.p, nullptr, nullptr, nullptr);
    // 1p -> 2p1h
    couple_1p_to_2p1h(s, st, xn, CA.p, tm2.p, true, nullptr, nullptr);
    pair_combine(s, CA.p, vv, yn + v, vv, o, v, kS1, kS2, 1.0, 1.0);
    if (ring && st.order >= 3) ring_fp64(s, st, xn + v, yn + v);
  }
  if (ladder && st.order >= 3)
    ladder_fp64(s, st.Bvv.p, st.naux, v, x + v, vv, nvec, dim, o, y + v, dim, vv, 1.0, 1.0);
}

void sigma_fp64(cudaStream_t s, State& st, int nvec, const double* x, double* y) {
  sigma_base_fp64(s, st, nvec, x, y, true, true);
}

}  // namespace ea
