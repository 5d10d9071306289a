"""Closed-shell (restricted) EA-ADC(2)/(3) for doublet attached states, with
density-fitted integrals (pq|rs) = sum_Q B^Q_pq B^Q_rs (Sec. II.B, Eq. 25).

Space: 1p part y[a] (a alpha electron attached to virtual a) and 2p1h part
w[k, b, c] over ALL (b, c).  w is the orthonormal doublet representation: its
symmetric part in (b, c) is the pair-singlet-coupled doublet and its
antisymmetric part the pair-triplet-coupled doublet, each with unit metric, so
the secular matrix is symmetric in the Euclidean product and
sum_bc w_bc phi_b(1) phi_c(2) is the particles' spatial pair function.

Relation to determinants (Ms = +1/2): with A = S^-1(w) the coefficient of
c_{b alpha}^+ c_{c beta}^+ c_{k beta} |Phi_0> is A[k,b,c] and that of
c_{b alpha}^+ c_{c alpha}^+ c_{k alpha} |Phi_0> (b < c) is A[k,b,c] - A[k,c,b]
(the doublet condition S+ Psi = 0).  S(Z) = sym(Z) + sqrt(3) antisym(Z) over
the last two axes; S is self-adjoint, and sigma_w = S(sigma_A(S^-1 w)) for every
2p1h term, where sigma_A is the sigma of the alpha-beta-beta block.

In this representation the particle-particle ladder is exactly
sigma[k,b,c] += sum_de (bd|ce) w[k,d,e]  (S commutes with it).

The spin-orbital blocks these formulas are integrated from are listed in
``spinorb``; test P3 checks this restricted matrix against the spin-orbital
one projected onto the doublet space, element by element.

Spatial notation: i,j,k,l,m occupied; a..e virtual; D_ij^ab = e_i+e_j-e_a-e_b;
tau_ij^ab = (ia|jb) / D_ij^ab is the alpha-beta first-order amplitude (the
same-spin amplitude is tau_ij^ab - tau_ij^ba).
"""
from __future__ import annotations

import numpy as np

SQ3 = np.sqrt(3.0)


def _es(*args):
    return np.einsum(*args, optimize=True)


def S_map(Z):
    Zt = np.swapaxes(Z, -1, -2)
    return 0.5 * (Z + Zt) + SQ3 * 0.5 * (Z - Zt)


def Sinv_map(Z):
    Zt = np.swapaxes(Z, -1, -2)
    return 0.5 * (Z + Zt) + 0.5 * (Z - Zt) / SQ3


class Problem:
    """Orbital energies and DF factor split into oo/ov/vv blocks."""

    def __init__(self, eps_occ, eps_vir, B):
        self.eo = np.asarray(eps_occ, dtype=np.float64)
        self.ev = np.asarray(eps_vir, dtype=np.float64)
        self.o, self.v = self.eo.size, self.ev.size
        o = self.o
        B = np.asarray(B, dtype=np.float64)
        self.Boo = np.ascontiguousarray(B[:, :o, :o])
        self.Bov = np.ascontiguousarray(B[:, :o, o:])
        self.Bvv = np.ascontiguousarray(B[:, o:, o:])
        self.naux = B.shape[0]
        self.ovov = _es("Qia,Qjb->iajb", self.Bov, self.Bov)
        self.oovv = _es("Qij,Qab->ijab", self.Boo, self.Bvv)
        self.oooo = _es("Qij,Qkl->ijkl", self.Boo, self.Boo)
        self.ooov = _es("Qij,Qka->ijka", self.Boo, self.Bov)
        self._ovvv = None
        eo, ev = self.eo, self.ev
        self.D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
        self.tau = self.ovov.transpose(0, 2, 1, 3) / self.D2

    @property
    def ovvv(self):
        if self._ovvv is None:
            self._ovvv = _es("Qia,Qbc->iabc", self.Bov, self.Bvv)
        return self._ovvv

    def vvvv(self):
        return _es("Qab,Qcd->abcd", self.Bvv, self.Bvv)

    def ladder_pairs(self, T):
        """sum_cd (ac|bd) T[..., c, d] for a stack of v x v matrices (DF, Eq. 25)."""
        out = np.zeros_like(T)
        for Q in range(self.naux):
            BQ = self.Bvv[Q]
            out += BQ @ T @ BQ
        return out


# --------------------------------------------------------------------- 1p/1p
def m11_second(p: Problem):
    """M^(2)_ab = (L_ab + L_ba)/2, L_ab = -sum_klc (kb|lc)(2 tau_kl^ac - tau_kl^ca)."""
    t2 = 2 * p.tau - p.tau.swapaxes(2, 3)
    L = -_es("kblc,klac->ab", p.ovov, t2)
    return 0.5 * (L + L.T)


def mp2_densities(p: Problem):
    """Per-spin MP2 correlation densities rho_cd (vv) and rho_kl (oo)."""
    t2 = 2 * p.tau - p.tau.swapaxes(2, 3)
    rv = _es("ijce,ijde->cd", p.tau, t2)
    ro = -_es("kjcd,ljcd->kl", p.tau, t2)
    return rv, ro


def second_order_amplitudes(p: Problem, lad=None):
    """Second-order doubles ups_ij^ab (alpha-beta) and singles ups_i^a."""
    tau = p.tau
    if lad is None:
        lad = p.ladder_pairs(tau)
    hh = _es("kilj,klab->ijab", p.oooo, tau)
    t2 = 2 * tau - tau.swapaxes(2, 3)
    X0 = (_es("ikac,kcjb->ijab", t2, p.ovov)
          - _es("ikac,kjbc->ijab", tau, p.oovv)
          - _es("ikcb,kjac->ijab", tau, p.oovv))
    ups2 = (lad + hh + X0 + X0.transpose(1, 0, 3, 2)) / p.D2
    s1 = (_es("kcad,ikdc->ia", p.ovvv, t2)
          - _es("likc,klca->ia", p.ooov, t2))
    ups1 = s1 / (p.eo[:, None] - p.ev[None, :])
    return ups1, ups2, lad


def m11_third(p: Problem, lad=None):
    """M^(3)_ab = (L3_ab + L3_ba)/2 from the spin-orbital L^(3) integrated over spin."""
    tau = p.tau
    ups1, ups2, lad = second_order_amplitudes(p, lad)
    # same form as second order with the second-order doubles
    A = -_es("kblc,klac->ab", p.ovov, 2 * ups2 - ups2.swapaxes(2, 3))
    # second-order singles
    X = 2 * _es("jcab,jc->ab", p.ovvv, ups1) - _es("jbac,jc->ab", p.ovvv, ups1)
    # MP2 density terms
    rv, ro = mp2_densities(p)
    g = _es("Qcd,cd->Q", p.Bvv, rv)
    Dt = 2 * _es("Q,Qab->ab", g, p.Bvv)
    Dt -= sum(p.Bvv[Q] @ rv.T @ p.Bvv[Q] for Q in range(p.naux))
    Dt += 2 * _es("klab,kl->ab", p.oovv, ro) - _es("lakb,kl->ab", p.ovov, ro)
    # ring-type t.g.t term, five spin cases
    Ta = tau - tau.swapaxes(2, 3)
    Icb = p.oovv.transpose(2, 1, 0, 3)          # (cb|lk) as [c,k,l,b]
    Ick = p.ovov.transpose(1, 0, 2, 3)          # (ck|lb) as [c,k,l,b]
    E1 = (_es("cklb,ckal->ab", Icb - Ick, _es("ikce,ilae->ckal", Ta, Ta))
          + _es("cklb,ckal->ab", Ick, _es("ikec,ilae->ckal", tau, Ta))
          + _es("cklb,ckal->ab", Icb, _es("ikce,ilae->ckal", tau, tau))
          + _es("cklb,ckal->ab", Icb - Ick, _es("kice,liae->ckal", tau, tau))
          + _es("cklb,ckal->ab", Ick, _es("ikce,liae->ckal", Ta, tau)))
    # t . (vvvv ladder of t)
    E2 = -_es("ijae,ijbe->ab", tau, 2 * lad - lad.swapaxes(2, 3))
    L3 = A + X + X.T + Dt + E1 + E2
    return 0.5 * (L3 + L3.T)


def m11(p: Problem, order=3, x3=1.0, lad=None):
    M = np.diag(p.ev) + m11_second(p)
    if order >= 3 and x3 != 0.0:
        M = M + x3 * m11_third(p, lad)
    return M


# ------------------------------------------------------------------ coupling
def coupling_A(p: Problem, order=3):
    """C_A[k,b,c,a]: coupling of 1p (a alpha) to c_{b alpha}^+ c_{c beta}^+ c_{k beta}."""
    C = _es("kcab->kbca", p.ovvv).copy()                       # (ab|kc)
    if order >= 3:
        tau = p.tau
        C -= _es("lacd,lkbd->kbca", p.ovvv, tau)                 # (al|cd) t_lk^bd
        C -= _es("ldab,lkcd->kbca", p.ovvv, tau - 2 * tau.swapaxes(2, 3))
        C -= _es("labd,lkdc->kbca", p.ovvv, tau)                 # (al|bd) t_lk^dc
        C += _es("kmla,lmbc->kbca", p.ooov, tau)                 # (al|km) t_lm^bc
    return C


def coupling_w(p: Problem, order=3):
    """Coupling in the orthonormal representation, [k,b,c,a]."""
    C = coupling_A(p, order)
    return S_map(C.transpose(3, 0, 1, 2)).transpose(1, 2, 3, 0)


# ----------------------------------------------------------------- 2p1h/2p1h
def ring_A(p: Problem, A):
    """First-order particle-hole terms on the alpha-beta-beta block, A[k,b,c]."""
    return (-_es("lkbd,ldc->kbc", p.oovv, A)
            - _es("kcld,ldb->kbc", p.ovov, A - 2 * A.swapaxes(1, 2))
            - _es("lkcd,lbd->kbc", p.oovv, A))


def ring_w(p: Problem, W):
    return S_map(ring_A(p, Sinv_map(W)))


def ladder_w(p: Problem, W):
    return p.ladder_pairs(W)


def diag_2p1h(p: Problem):
    return p.ev[None, :, None] + p.ev[None, None, :] - p.eo[:, None, None]


# ------------------------------------------------------------ explicit matrix
def explicit_matrix(p: Problem, order=3, x3=1.0):
    """Dense M over [1p (v), 2p1h (o*v*v)] built from 4-index integrals."""
    o, v = p.o, p.v
    n2 = o * v * v
    M = np.zeros((v + n2, v + n2))
    M[:v, :v] = m11(p, order, x3)
    C = coupling_w(p, order).reshape(n2, v)
    M[v:, :v] = C
    M[:v, v:] = C.T
    M22 = np.diag(diag_2p1h(p).reshape(-1))
    if order >= 3:
        I_o, I_v = np.eye(o), np.eye(v)
        vvvv = p.vvvv()
        lad = _es("kl,bdce->kbclde", I_o, vvvv)                 # d_kl (bd|ce)
        RA = (-_es("lkbd,ce->kbclde", p.oovv, I_v)
              - _es("kcld,eb->kbclde", p.ovov, I_v)
              + 2 * _es("kcle,db->kbclde", p.ovov, I_v)
              - _es("lkce,db->kbclde", p.oovv, I_v))
        # S on the output pair (b,c), S^-1 on the input pair (d,e)
        RA = S_map(RA.transpose(0, 3, 4, 5, 1, 2)).transpose(0, 4, 5, 1, 2, 3)
        RA = Sinv_map(RA)
        M22 += (lad + RA).reshape(n2, n2)
    M[v:, v:] = M22
    return M


# -------------------------------------------------------------------- sigma
class Sigma:
    """Matrix-vector product sigma = M c with DF integrals, for Davidson."""

    def __init__(self, p: Problem, order=3, x3=1.0):
        self.p, self.order = p, order
        lad = p.ladder_pairs(p.tau) if order >= 3 else None
        self.M11 = m11(p, order, x3, lad)
        self.D2p1h = diag_2p1h(p)

    def diagonal(self):
        p = self.p
        d = [np.diag(self.M11), self.D2p1h.reshape(-1).copy()]
        return np.concatenate(d)

    def _couple_1p_to_2p1h(self, y):
        """(C_A y)[k,b,c]."""
        p = self.p
        Qy = _es("Qab,a->Qb", p.Bvv, y)                       # sum_a B^Q_ab y_a
        out = _es("Qb,Qkc->kbc", Qy, p.Bov)                    # (ab|kc) y_a
        if self.order >= 3:
            tau = p.tau
            Qo = _es("Qla,a->Ql", p.Bov, y)                   # sum_a B^Q_la y_a
            F = _es("Ql,Qcd->lcd", Qo, p.Bvv)                  # sum_a (al|cd) y_a
            G = _es("Qb,Qld->bld", Qy, p.Bov)                  # sum_a (ab|ld) y_a
            H = _es("Ql,Qkm->lkm", Qo, p.Boo)                  # sum_a (al|km) y_a
            out -= _es("lcd,lkbd->kbc", F, tau)
            out -= _es("bld,lkcd->kbc", G, tau - 2 * tau.swapaxes(2, 3))
            out -= _es("lbd,lkdc->kbc", F, tau)
            out += _es("lkm,lmbc->kbc", H, tau)
        return out

    def _couple_2p1h_to_1p(self, V):
        """sum_kbc C_A[k,b,c,a] V[k,b,c]."""
        p = self.p
        g = _es("Qkc,kbc->Qb", p.Bov, V)
        out = _es("Qab,Qb->a", p.Bvv, g)
        if self.order >= 3:
            tau = p.tau
            H1 = _es("lkbd,kbc->ldc", tau, V)                  # sum_kb t_lk^bd V_kbc
            out -= _es("Qla,Ql->a", p.Bov, _es("Qcd,ldc->Ql", p.Bvv, H1))
            H2 = _es("lkcd,kbc->bld", tau - 2 * tau.swapaxes(2, 3), V)
            out -= _es("Qab,Qb->a", p.Bvv, _es("Qld,bld->Qb", p.Bov, H2))
            H3 = _es("lkdc,kbc->lbd", tau, V)
            out -= _es("Qla,Ql->a", p.Bov, _es("Qbd,lbd->Ql", p.Bvv, H3))
            H4 = _es("lmbc,kbc->lkm", tau, V)
            out += _es("Qla,Ql->a", p.Bov, _es("Qkm,lkm->Ql", p.Boo, H4))
        return out

    def __call__(self, x):
        """x: [v + o*v*v] or [nvec, v + o*v*v]."""
        p = self.p
        x = np.asarray(x, dtype=np.float64)
        single = x.ndim == 1
        X = x[None] if single else x
        out = np.empty_like(X)
        v, o = p.v, p.o
        for n in range(X.shape[0]):
            y = X[n, :v]
            W = X[n, v:].reshape(o, v, v)
            sy = self.M11 @ y + self._couple_2p1h_to_1p(S_map(W))
            sW = self.D2p1h * W + S_map(self._couple_1p_to_2p1h(y))
            if self.order >= 3:
                sW = sW + p.ladder_pairs(W) + ring_w(p, W)
            out[n, :v] = sy
            out[n, v:] = sW.reshape(-1)
        return out[0] if single else out
