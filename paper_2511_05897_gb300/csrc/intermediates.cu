// Per-state intermediates of restricted EA-ADC(2)/(3) (FP64):
//   tau_ij^ab = (ia|jb) / D_ij^ab                     first-order amplitudes
//   Kmat[(k,b),(l,d)] = (bd|lk),  Jmat[(k,c),(l,d)] = (ck|ld)   stored <=2-virtual
//                                                     integrals (Sec. II.B: integrals
//                                                     with up to two virtual indices
//                                                     are stored)
//   M11 = diag(e) + M^(2) + x3 * M^(3)                 1p/1p block
// M^(2) and M^(3) are (L + L^T)/2 of the spin-integrated
// L_ab = <Psi_0| c_a [V_N, c_b^+] |Psi_0> through third order (ISR, Sec. II.A);
// three- and four-virtual integrals are never stored: they enter through the
// DF factor B^Q (Eq. 25) as two successive contractions.
#include "internal.cuh"

#include <cmath>

namespace ea {
namespace {

__global__ void tau_kernel(const double* __restrict__ ovov, const double* __restrict__ eo,
                           const double* __restrict__ ev, double* __restrict__ tau, int o, int v) {
  long long total = (long long)o * o * v * v;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int b = idx % v;
    long long r = idx / v;
    int a = r % v;
    r /= v;
    int j = r % o;
    int i = (int)(r / o);
    double num = ovov[(((long long)i * v + a) * o + j) * v + b];
    tau[idx] = num / (eo[i] + eo[j] - ev[a] - ev[b]);
  }
}

// x[i][j][a][b] /= D_ij^ab
__global__ void div_D_kernel(double* __restrict__ x, const double* __restrict__ eo,
                             const double* __restrict__ ev, int o, int v) {
  long long total = (long long)o * o * v * v;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int b = idx % v;
    long long r = idx / v;
    int a = r % v;
    r /= v;
    int j = r % o;
    int i = (int)(r / o);
    x[idx] /= (eo[i] + eo[j] - ev[a] - ev[b]);
  }
}

// x[i][a] /= (e_i - e_a)
__global__ void div_D1_kernel(double* __restrict__ x, const double* __restrict__ eo,
                              const double* __restrict__ ev, int o, int v) {
  int total = o * v;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int a = idx % v, i = idx / v;
    x[idx] /= (eo[i] - ev[a]);
  }
}

// M = diag(ev) + 0.5 * (L + L^T)   (add = false), or M += x3 * 0.5 * (L + L^T)
__global__ void sym_kernel(double* __restrict__ M, const double* __restrict__ L, const double* __restrict__ ev,
                           int v, double scale, int add) {
  int total = v * v;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int a = idx / v, b = idx % v;
    double s = scale * 0.5 * (L[a * v + b] + L[b * v + a]);
    if (add) M[idx] += s;
    else M[idx] = s + (a == b ? ev[a] : 0.0);
  }
}

__global__ void diag_kernel(double* __restrict__ D, const double* __restrict__ M11, const double* __restrict__ eo,
                            const double* __restrict__ ev, int o, int v) {
  long long total = (long long)v + (long long)o * v * v;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < v) {
      D[idx] = M11[idx * v + idx];
    } else {
      long long r = idx - v;
      int c = r % v;
      r /= v;
      int b = r % v;
      int k = (int)(r / v);
      D[idx] = ev[b] + ev[c] - eo[k];
    }
  }
}

int gridn(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

}  // namespace

// sum_Q Bvv[Q] T[m] Bvv[Q] for nmat v x v matrices T (stride tstride), accumulated
// into out (stride ostride) with out = beta*out + alpha*result.
void ladder_fp64(cudaStream_t s, const double* Bvv, int naux, int v, const double* T, long long tstride,
                 int nb1, long long tstride1, int nb2, double* out, long long ostride1, long long ostride2,
                 double alpha, double beta) {
  DArr<double> tmp((size_t)nb1 * nb2 * v * v, s);
  const long long vv = (long long)v * v;
  for (int Q = 0; Q < naux; ++Q) {
    GemmBatch b1;
    b1.nb1 = nb1; b1.nb2 = nb2;
    b1.sB1 = tstride1; b1.sB2 = tstride;
    b1.sC1 = (long long)nb2 * vv; b1.sC2 = vv;
    dgemm(s, false, false, v, v, v, 1.0, Bvv + Q * vv, v, T, v, 0.0, tmp.p, v, b1);
    GemmBatch b2;
    b2.nb1 = nb1; b2.nb2 = nb2;
    b2.sA1 = (long long)nb2 * vv; b2.sA2 = vv;
    b2.sC1 = ostride1; b2.sC2 = ostride2;
    dgemm(s, false, false, v, v, v, alpha, tmp.p, v, Bvv + Q * vv, v, (Q == 0) ? beta : 1.0, out, v, b2);
  }
}

void build_state_intermediates(eaadc_ctx* ctx, State& st) {
  cudaStream_t s = ctx->stream;
  const int o = st.o, v = st.v, naux = st.naux;
  const long long ov = (long long)o * v, oo = (long long)o * o, vv = (long long)v * v;
  st.dim = v + ov * v;
  // (ia|jb) as [(i,a)][(j,b)]: also the stored Jmat[(k,c),(l,d)] = (ck|ld)
  st.Jmat.alloc((size_t)(ov * ov), s);
  dgemm(s, true, false, (int)ov, (int)ov, naux, 1.0, st.Bov.p, ov, st.Bov.p, ov, 0.0, st.Jmat.p, ov);
  st.tau.alloc((size_t)(oo * vv), s);
  tau_kernel<<<gridn(oo * vv), 256, 0, s>>>(st.Jmat.p, st.eo.p, st.ev.p, st.tau.p, o, v);
  EA_LAUNCH();
  // (lk|bd) as [l][k][b][d]; Kmat[(k,b),(l,d)] = (bd|lk)
  DArr<double> oovv((size_t)(oo * vv), s);
  dgemm(s, true, false, (int)oo, (int)vv, naux, 1.0, st.Boo.p, oo, st.Bvv.p, vv, 0.0, oovv.p, vv);
  st.Kmat.alloc((size_t)(ov * ov), s);
  permute(s, oovv.p, {o, o, v, v}, {1, 2, 0, 3}, st.Kmat.p);

  Tens tau{st.tau.p, {o, o, v, v}};
  Tens ovov{st.Jmat.p, {o, v, o, v}};
  Tens oovvT{oovv.p, {o, o, v, v}};
  // t2 = 2 tau - tau(a<->b)
  DArr<double> t2d((size_t)(oo * vv), s);
  permute(s, st.tau.p, {o, o, v, v}, {0, 1, 3, 2}, t2d.p, -1.0, 0.0);
  axpby(s, (size_t)(oo * vv), 2.0, st.tau.p, 1.0, t2d.p);
  Tens t2{t2d.p, {o, o, v, v}};

  DArr<double> L((size_t)vv, s);
  Tens Lt{L.p, {v, v}};
  // M^(2): L_ab = -sum_klc (kb|lc)(2 tau_kl^ac - tau_kl^ca)
  einsum(s, "kblc,klac->ab", -1.0, ovov, t2, 0.0, Lt);
  st.M11.alloc((size_t)vv, s);
  sym_kernel<<<gridn(vv), 256, 0, s>>>(st.M11.p, L.p, st.ev.p, v, 1.0, 0);
  EA_LAUNCH();

  if (st.order >= 3 && st.x3 != 0.0) {
    // second-order doubles: pp-ladder, hh-ladder, ring terms
    DArr<double> lad((size_t)(oo * vv), s);
    if (st.build_prec == EAADC_FP64)
      ladder_fp64(s, st.Bvv.p, naux, v, st.tau.p, vv, 1, 0, (int)oo, lad.p, 0, vv, 1.0, 0.0);
    else  // tensor cores; the intermediates above are what the operand copies need
      ladder_pairs_tc(s, st, st.tau.p, (int)oo, st.build_prec == EAADC_MIXED_BF16X3, lad.p);
    DArr<double> oooo((size_t)(oo * oo), s), ooov((size_t)(oo * ov), s);
    dgemm(s, true, false, (int)oo, (int)oo, naux, 1.0, st.Boo.p, oo, st.Boo.p, oo, 0.0, oooo.p, oo);
    dgemm(s, true, false, (int)oo, (int)ov, naux, 1.0, st.Boo.p, oo, st.Bov.p, ov, 0.0, ooov.p, ov);
    DArr<double> ups2((size_t)(oo * vv), s), X0((size_t)(oo * vv), s);
    Tens U2{ups2.p, {o, o, v, v}}, X0t{X0.p, {o, o, v, v}};
    einsum(s, "kilj,klab->ijab", 1.0, Tens{oooo.p, {o, o, o, o}}, tau, 0.0, U2);
    axpby(s, (size_t)(oo * vv), 1.0, lad.p, 1.0, ups2.p);
    einsum(s, "ikac,kcjb->ijab", 1.0, t2, ovov, 0.0, X0t);
    einsum(s, "ikac,kjbc->ijab", -1.0, tau, oovvT, 1.0, X0t);
    einsum(s, "ikcb,kjac->ijab", -1.0, tau, oovvT, 1.0, X0t);
    axpby(s, (size_t)(oo * vv), 1.0, X0.p, 1.0, ups2.p);
    permute(s, X0.p, {o, o, v, v}, {1, 0, 3, 2}, ups2.p, 1.0, 1.0);
    div_D_kernel<<<gridn(oo * vv), 256, 0, s>>>(ups2.p, st.eo.p, st.ev.p, o, v);
    EA_LAUNCH();
    // second-order singles: sum_kcd (kc|ad) t2_ik^dc - sum_klc (kc|li) t2_kl^ca
    DArr<double> Y((size_t)naux * ov, s), ups1((size_t)ov, s);
    Tens Bov{st.Bov.p, {naux, o, v}}, Bvv{st.Bvv.p, {naux, v, v}}, Boo{st.Boo.p, {naux, o, o}};
    Tens Yt{Y.p, {naux, o, v}}, U1{ups1.p, {o, v}};
    einsum(s, "Qkc,ikdc->Qid", 1.0, Bov, t2, 0.0, Yt);
    einsum(s, "Qad,Qid->ia", 1.0, Bvv, Yt, 0.0, U1);
    einsum(s, "likc,klca->ia", -1.0, Tens{ooov.p, {o, o, o, v}}, t2, 1.0, U1);
    div_D1_kernel<<<gridn(ov), 256, 0, s>>>(ups1.p, st.eo.p, st.ev.p, o, v);
    EA_LAUNCH();

    DArr<double> L3((size_t)vv, s);
    Tens L3t{L3.p, {v, v}};
    // A: same form as M^(2) with the second-order doubles
    DArr<double> u2x((size_t)(oo * vv), s);
    permute(s, ups2.p, {o, o, v, v}, {0, 1, 3, 2}, u2x.p, -1.0, 0.0);
    axpby(s, (size_t)(oo * vv), 2.0, ups2.p, 1.0, u2x.p);
    einsum(s, "kblc,klac->ab", -1.0, ovov, Tens{u2x.p, {o, o, v, v}}, 0.0, L3t);
    // X + X^T with X_ab = sum_jc [2 (ab|jc) - (ac|jb)] u_j^c
    DArr<double> g((size_t)naux, s), Z((size_t)naux * vv, s), Xab((size_t)vv, s);
    Tens gt{g.p, {naux}}, Zt{Z.p, {naux, v, v}}, Xt{Xab.p, {v, v}};
    einsum(s, "Qjc,jc->Q", 1.0, Bov, U1, 0.0, gt);
    einsum(s, "Qab,Q->ab", 2.0, Bvv, gt, 0.0, Xt);
    einsum(s, "jc,Qjb->Qcb", 1.0, U1, Bov, 0.0, Zt);
    einsum(s, "Qac,Qcb->ab", -1.0, Bvv, Zt, 1.0, Xt);
    axpby(s, (size_t)vv, 1.0, Xab.p, 1.0, L3.p);
    permute(s, Xab.p, {v, v}, {1, 0}, L3.p, 1.0, 1.0);
    // MP2 density terms
    DArr<double> rv((size_t)vv, s), ro((size_t)oo, s), rvT((size_t)vv, s);
    Tens rvt{rv.p, {v, v}}, rot{ro.p, {o, o}};
    einsum(s, "ijce,ijde->cd", 1.0, tau, t2, 0.0, rvt);
    einsum(s, "kjcd,ljcd->kl", -1.0, tau, t2, 0.0, rot);
    einsum(s, "Qcd,cd->Q", 1.0, Bvv, rvt, 0.0, gt);
    einsum(s, "Qab,Q->ab", 2.0, Bvv, gt, 1.0, L3t);
    permute(s, rv.p, {v, v}, {1, 0}, rvT.p);
    ladder_fp64(s, st.Bvv.p, naux, v, rvT.p, 0, 1, 0, 1, L3.p, 0, 0, -1.0, 1.0);
    einsum(s, "klab,kl->ab", 2.0, oovvT, rot, 1.0, L3t);
    einsum(s, "lakb,kl->ab", -1.0, ovov, rot, 1.0, L3t);
    // ring-type t.g.t terms (five spin cases)
    DArr<double> Ta((size_t)(oo * vv), s);
    permute(s, st.tau.p, {o, o, v, v}, {0, 1, 3, 2}, Ta.p, -1.0, 0.0);
    axpby(s, (size_t)(oo * vv), 1.0, st.tau.p, 1.0, Ta.p);
    Tens Tat{Ta.p, {o, o, v, v}};
    DArr<double> Z14((size_t)(oo * vv), s), Z25((size_t)(oo * vv), s), Z3((size_t)(oo * vv), s);
    Tens Z14t{Z14.p, {v, o, v, o}}, Z25t{Z25.p, {v, o, v, o}}, Z3t{Z3.p, {v, o, v, o}};
    einsum(s, "ikce,ilae->ckal", 1.0, Tat, Tat, 0.0, Z14t);
    einsum(s, "kice,liae->ckal", 1.0, tau, tau, 1.0, Z14t);
    einsum(s, "ikec,ilae->ckal", 1.0, tau, Tat, 0.0, Z25t);
    einsum(s, "ikce,liae->ckal", 1.0, Tat, tau, 1.0, Z25t);
    einsum(s, "ikce,ilae->ckal", 1.0, tau, tau, 0.0, Z3t);
    axpby(s, (size_t)(oo * vv), 1.0, Z14.p, 1.0, Z3.p);    // Z3 <- Z14 + Z3
    axpby(s, (size_t)(oo * vv), 1.0, Z14.p, -1.0, Z25.p);  // Z25 <- Z14 - Z25
    einsum(s, "lkcb,ckal->ab", 1.0, oovvT, Z3t, 1.0, L3t);
    einsum(s, "kclb,ckal->ab", -1.0, ovov, Z25t, 1.0, L3t);
    // tau . (vvvv ladder of tau)
    DArr<double> lx((size_t)(oo * vv), s);
    permute(s, lad.p, {o, o, v, v}, {0, 1, 3, 2}, lx.p, -1.0, 0.0);
    axpby(s, (size_t)(oo * vv), 2.0, lad.p, 1.0, lx.p);
    einsum(s, "ijae,ijbe->ab", -1.0, tau, Tens{lx.p, {o, o, v, v}}, 1.0, L3t);
    sym_kernel<<<gridn(vv), 256, 0, s>>>(st.M11.p, L3.p, st.ev.p, v, st.x3, 1);
    EA_LAUNCH();
  }
  st.diag.alloc((size_t)st.dim, s);
  diag_kernel<<<gridn(st.dim), 256, 0, s>>>(st.diag.p, st.M11.p, st.eo.p, st.ev.p, o, v);
  EA_LAUNCH();
  EA_CK(cudaStreamSynchronize(s));
}

}  // namespace ea
