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
void couple_1p_to_2p1h(cudaStream_t s, State& st, const double* y, double* outA, const double* tm2, bool big,
                       double* Fo, double* Go) {
  const int o = st.o, v = st.v, naux = st.naux;
  Tens Bov{st.Bov.p, {naux, o, v}}, Bvv{st.Bvv.p, {naux, v, v}}, Boo{st.Boo.p, {naux, o, o}};
  Tens yt{(double*)y, {v}};
  Tens out{outA, {o, v, v}};
  DArr<double> Qy((size_t)naux * v, s);
  Tens Qyt{Qy.p, {naux, v}};
  einsum(s, "Qba,a->Qb", 1.0, Bvv, yt, 0.0, Qyt);  // B^Q symmetric
  einsum(s, "Qb,Qkc->kbc", 1.0, Qyt, Bov, 0.0, out);
  if (st.order < 3) return;
  Tens tau{st.tau.p, {o, o, v, v}};
  DArr<double> Qo((size_t)naux * o, s), F, G, H((size_t)o * o * o, s);
  double* Fp = Fo;
  double* Gp = Go;
  if (!Fp) { F.alloc((size_t)o * v * v, s); Fp = F.p; }
  if (!Gp) { G.alloc((size_t)o * v * v, s); Gp = G.p; }
  Tens Qot{Qo.p, {naux, o}}, Ft{Fp, {o, v, v}}, Gt{Gp, {v, o, v}}, Ht{H.p, {o, o, o}};
  einsum(s, "Qla,a->Ql", 1.0, Bov, yt, 0.0, Qot);
  einsum(s, "Ql,Qcd->lcd", 1.0, Qot, Bvv, 0.0, Ft);
  einsum(s, "Qb,Qld->bld", 1.0, Qyt, Bov, 0.0, Gt);
  einsum(s, "Ql,Qkm->lkm", 1.0, Qot, Boo, 0.0, Ht);
  einsum(s, "lkm,lmbc->kbc", 1.0, Ht, tau, 1.0, out);
  if (!big) return;
  einsum(s, "lcd,lkbd->kbc", -1.0, Ft, tau, 1.0, out);
  einsum(s, "bld,lkcd->kbc", -1.0, Gt, Tens{(double*)tm2, {o, o, v, v}}, 1.0, out);
  einsum(s, "lbd,lkdc->kbc", -1.0, Ft, tau, 1.0, out);
}

// sy[a] += sum_kbc C_A[k,b,c,a] V[k,b,c].  With H1..H3 given (tensor-core
// path) the three o^2 v^3 contractions H1[l][d][c] = sum_kb t_lk^bd V_kbc,
// H2[b][l][d] = sum_kc (t_lk^cd - 2 t_lk^dc) V_kbc, H3[l][b][d] = sum_kc t_lk^dc V_kbc
// are taken from them instead of being formed here.
void couple_2p1h_to_1p(cudaStream_t s, State& st, const double* V, double* sy, const double* tm2,
                       const double* H1g, const double* H2g, const double* H3g) {
  const int o = st.o, v = st.v, naux = st.naux;
  Tens Bov{st.Bov.p, {naux, o, v}}, Bvv{st.Bvv.p, {naux, v, v}}, Boo{st.Boo.p, {naux, o, o}};
  Tens Vt{(double*)V, {o, v, v}};
  Tens out{sy, {v}};
  DArr<double> g((size_t)naux * v, s);
  Tens gt{g.p, {naux, v}};
  einsum(s, "Qkc,kbc->Qb", 1.0, Bov, Vt, 0.0, gt);
  einsum(s, "Qba,Qb->a", 1.0, Bvv, gt, 1.0, out);  // B^Q symmetric
  if (st.order < 3) return;
  Tens tau{st.tau.p, {o, o, v, v}};
  DArr<double> H, tt((size_t)naux * o, s), t2q((size_t)naux * v, s), H4((size_t)o * o * o, s);
  Tens ttt{tt.p, {naux, o}}, t2qt{t2q.p, {naux, v}};
  const bool ext = H1g != nullptr;
  if (!ext) H.alloc((size_t)o * v * v, s);
  Tens H1t{ext ? (double*)H1g : H.p, {o, v, v}};
  if (!ext) einsum(s, "lkbd,kbc->ldc", 1.0, tau, Vt, 0.0, H1t);
  einsum(s, "Qcd,ldc->Ql", -1.0, Bvv, H1t, 0.0, ttt);
  Tens H2t{ext ? (double*)H2g : H.p, {v, o, v}};
  if (!ext) einsum(s, "lkcd,kbc->bld", 1.0, Tens{(double*)tm2, {o, o, v, v}}, Vt, 0.0, H2t);
  einsum(s, "Qld,bld->Qb", 1.0, Bov, H2t, 0.0, t2qt);
  einsum(s, "Qba,Qb->a", -1.0, Bvv, t2qt, 1.0, out);
  Tens H3t{ext ? (double*)H3g : H.p, {o, v, v}};
  if (!ext) einsum(s, "lkdc,kbc->lbd", 1.0, tau, Vt, 0.0, H3t);
  einsum(s, "Qbd,lbd->Ql", -1.0, Bvv, H3t, 1.0, ttt);
  Tens H4t{H4.p, {o, o, o}};
  einsum(s, "lmbc,kbc->lkm", 1.0, tau, Vt, 0.0, H4t);
  einsum(s, "Qkm,lkm->Ql", 1.0, Boo, H4t, 1.0, ttt);
  einsum(s, "Qla,Ql->a", 1.0, Bov, ttt, 1.0, out);
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
