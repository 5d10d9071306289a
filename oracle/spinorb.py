"""EA-ADC(n) secular-matrix blocks in spin-orbital form, element by element.

The paper gives the working equations only in its supplementary material,
which is not available; the blocks below follow from the ISR definition of
Sec. II.A (Eq. 1-6) with the perturbation-order truncation of Eq. 5, for the
attachment classes 1p (c_a^+) and 2p1h (c_b^+ c_c^+ c_k, b < c) of Eq. 2.
Strict ADC(3) keeps the 1p/1p block through third order, the 1p/2p1h
coupling through second order and the 2p1h/2p1h block through first order;
ADC(2) keeps them through second, first and zeroth order.  Every factor and
sign here is pinned against the brute-force ISR of ``fci_isr`` (test P1).

Notation: i,j,k,l,m occupied and a,b,c,d,e virtual spin orbitals,
<pq||rs> antisymmetrised, D_ij^ab = e_i + e_j - e_a - e_b,
t_ij^ab = <ab||ij> / D_ij^ab (first-order doubles).

1p/1p: with L_ab = <Psi_0| c_a [V_N, c_b^+] |Psi_0>, the ISR gives
M_ab = e_a d_ab + (L_ab + L_ba)/2 through third order, where
  L^(2)_ab = 1/2 sum_klc <kl||bc> t_kl^ca
  L^(3)_ab = 1/2 sum_klc <kl||bc> u_kl^ca                     (2nd-order doubles)
           + sum_jc (<aj||bc> + <ac||bj>) u_j^c               (2nd-order singles)
           + sum_cd <ac||bd> rho_cd + sum_kl <ak||bl> rho_kl  (MP2 density)
           + sum_ckl <cl||bk> sum_ie t_ik^ce t_il^ae
           + 1/2 sum_ije t_ij^ea Y_ij^be,  Y_ij^be = 1/2 sum_cd <be||cd> t_ij^cd.
1p/2p1h: M_{a,kbc} = <ak||bc> + P(bc) sum_ld <ad||cl> t_kl^db
                     + 1/2 sum_lm <ak||lm> t_lm^bc.
2p1h/2p1h: (e_b + e_c - e_k) d + d_kl <bc||de>
           - d_ce <bl||dk> + d_be <cl||dk> + d_cd <bl||ek> - d_bd <cl||ek>.
"""
from __future__ import annotations

import itertools

import numpy as np


def _pp(x, a, b):
    """x - x with axes a and b swapped."""
    return x - np.swapaxes(x, a, b)


def amplitudes(eps_so, g, nocc):
    o, v = slice(0, nocc), slice(nocc, eps_so.size)
    eo, ev = eps_so[o], eps_so[v]
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    t = g[v, v, o, o].transpose(2, 3, 0, 1) / D2
    return t, D2


def second_order_wavefunction(eps_so, g, nocc, t, D2):
    """Second-order singles u_i^a and doubles u_ij^ab of the MP wave function."""
    o, v = slice(0, nocc), slice(nocc, eps_so.size)
    eo, ev = eps_so[o], eps_so[v]
    ring = np.einsum("kbcj,ikac->ijab", g[o, v, v, o], t)
    ring = _pp(_pp(ring, 0, 1), 2, 3)
    nd = (0.5 * np.einsum("abcd,ijcd->ijab", g[v, v, v, v], t)
          + 0.5 * np.einsum("klij,klab->ijab", g[o, o, o, o], t) + ring)
    u2 = nd / D2
    ns = (0.5 * np.einsum("kacd,kicd->ia", g[o, v, v, v], t)
          - 0.5 * np.einsum("klci,klca->ia", g[o, o, v, o], t))
    u1 = ns / (eo[:, None] - ev[None, :])
    return u1, u2


def blocks(eps_so, g, nocc, order=3):
    """Dense blocks of M in the basis {c_A^+} + {c_B^+ c_C^+ c_K, B<C}.

    Returns dict with M11 parts '11_0', '11_2', '11_3', coupling '12_1', '12_2',
    and 2p1h parts '22_0', '22_1'; parts beyond the requested order are zero.
    """
    nso = eps_so.size
    nv = nso - nocc
    o, v = slice(0, nocc), slice(nocc, nso)
    eo, ev = eps_so[o], eps_so[v]
    t, D2 = amplitudes(eps_so, g, nocc)
    out = {}
    out["11_0"] = np.diag(ev)
    L2 = 0.5 * np.einsum("klbc,klca->ab", g[o, o, v, v], t)
    out["11_2"] = 0.5 * (L2 + L2.T)
    if order >= 3:
        u1, u2 = second_order_wavefunction(eps_so, g, nocc, t, D2)
        rv = 0.5 * np.einsum("ijce,ijde->cd", t, t)
        ro = -0.5 * np.einsum("kjcd,ljcd->kl", t, t)
        Y = 0.5 * np.einsum("becd,ijcd->ijbe", g[v, v, v, v], t)
        Z = np.einsum("ikce,ilae->ckal", t, t)
        L3 = (0.5 * np.einsum("klbc,klca->ab", g[o, o, v, v], u2)
              + np.einsum("ajbc,jc->ab", g[v, o, v, v], u1)
              + np.einsum("acbj,jc->ab", g[v, v, v, o], u1)
              + np.einsum("acbd,cd->ab", g[v, v, v, v], rv)
              + np.einsum("akbl,kl->ab", g[v, o, v, o], ro)
              + np.einsum("clbk,ckal->ab", g[v, o, v, o], Z)
              + 0.5 * np.einsum("ijea,ijbe->ab", t, Y))
        out["11_3"] = 0.5 * (L3 + L3.T)
    else:
        out["11_3"] = np.zeros((nv, nv))
    basis = [(K, Bv, C) for K in range(nocc) for Bv, C in itertools.combinations(range(nv), 2)]
    kk = np.array([x[0] for x in basis])
    bb = np.array([x[1] for x in basis])
    cc = np.array([x[2] for x in basis])
    C1 = g[v, o, v, v]
    out["12_1"] = C1[:, kk, bb, cc]
    if order >= 3:
        F = np.einsum("adcl,kldb->akbc", g[v, v, v, o], t)
        C2 = F - np.swapaxes(F, 2, 3) + 0.5 * np.einsum("aklm,lmbc->akbc", g[v, o, o, o], t)
        out["12_2"] = C2[:, kk, bb, cc]
    else:
        out["12_2"] = np.zeros_like(out["12_1"])
    out["22_0"] = np.diag(ev[bb] + ev[cc] - eo[kk])
    if order >= 3:
        dk = (kk[:, None] == kk[None, :]).astype(float)
        gv = g[v, v, v, v]
        gvoov = g[v, o, v, o]          # <bl||dk> as [b,l,d,k]
        K_, L_ = kk[:, None], kk[None, :]
        B_, C_ = bb[:, None], cc[:, None]
        D_, E_ = bb[None, :], cc[None, :]
        M1 = dk * gv[B_, C_, D_, E_]
        M1 -= (C_ == E_) * gvoov[B_, L_, D_, K_]
        M1 += (B_ == E_) * gvoov[C_, L_, D_, K_]
        M1 += (C_ == D_) * gvoov[B_, L_, E_, K_]
        M1 -= (B_ == D_) * gvoov[C_, L_, E_, K_]
        out["22_1"] = M1
    else:
        out["22_1"] = np.zeros_like(out["22_0"])
    out["basis"] = basis
    return out


def matrix(eps_so, g, nocc, order=3, x3=1.0):
    """Full EA-ADC(order) matrix; x3 scales the third-order 1p/1p part."""
    b = blocks(eps_so, g, nocc, order)
    M11 = b["11_0"] + b["11_2"] + x3 * b["11_3"]
    M12 = b["12_1"] + b["12_2"]
    M22 = b["22_0"] + b["22_1"]
    return np.block([[M11, M12], [M12.T, M22]])
