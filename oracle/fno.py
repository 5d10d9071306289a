"""State-specific frozen natural orbitals (SS-FNO), natural auxiliary
functions (NAF) and the perturbative truncation correction (Sec. II.C-E and
the algorithm of Sec. III).

Steps per attached state k (Sec. III, steps 2-4):
  * MP2 virtual density D^MP2 (spin-summed) in the canonical basis;
  * canonical EA-ADC(2) roots; D^EA(k) from the zeroth-order ISR of root k;
  * D^SS(k) = D^MP2 + D^EA(k) (Eq. 17); D V = V eta (Eq. 9); keep
    eta > eta_crit (Eq. 10-11);
  * F~ = V~^T F V~ (Eq. 12), F~ Z~ = Z~ e~ (Eq. 13), B = V~ Z~ (Eq. 14);
  * NAF: W = J J^T from the vv block of the FNO-basis DF factor (Eq. 28),
    keep eigenvectors with eigenvalue >= threshold, J~ = J N~ (Eq. 29);
  * EA-ADC(2) and EA-ADC(3) in the truncated space; Eq. 30:
    w_corr = w^(3)_FNO + w^(2)_canonical - w^(2)_FNO.

Readings (the supplementary material with D^EA-ADC(2) is not available):
D^EA(k)_ab = y_a y_b + sum_kc (w_kac w_kbc + w_kca w_kcb) with (y, w) the
normalised canonical ADC(2) eigenvector in the orthonormal doublet
representation (spin-summed; trace |y|^2 + 2|w|^2); D^MP2 is spin-summed too;
a negative threshold keeps everything; the target root in a truncated space
is the one whose 1p part overlaps most with the canonical root's 1p part
carried into that space (ties to the lower root).
"""
from __future__ import annotations

import numpy as np

from . import restricted as R
from .davidson import davidson


def mp2_density(p: R.Problem):
    rv, _ = R.mp2_densities(p)
    return 2.0 * rv


def ea_density(y, W):
    return np.outer(y, y) + np.einsum("kac,kbc->ab", W, W) + np.einsum("kca,kcb->ab", W, W)


def fno_basis(D, eps_vir, thresh):
    """Returns (Bfno [v, v'], eps_fno [v'], occupations kept)."""
    eta, V = np.linalg.eigh(0.5 * (D + D.T))
    keep = np.ones_like(eta, dtype=bool) if thresh < 0 else eta > thresh
    Vt = V[:, keep]
    F = Vt.T @ (eps_vir[:, None] * Vt)
    e, Z = np.linalg.eigh(0.5 * (F + F.T))
    return Vt @ Z, e, eta[keep]


def naf_basis(Bvv, thresh):
    """N~ [naux, naux'] from W = J J^T over the vv block (Eq. 27-29)."""
    J = Bvv.reshape(Bvv.shape[0], -1)
    W = J @ J.T
    lam, N = np.linalg.eigh(0.5 * (W + W.T))
    keep = np.ones_like(lam, dtype=bool) if thresh < 0 else lam >= thresh
    return N[:, keep], lam[keep]


def truncated_problem(p: R.Problem, Bfno, eps_fno, naf_thresh):
    """DF factor of the FNO/NAF space assembled as one [naux', n', n'] array."""
    Bov = np.einsum("Qia,aA->QiA", p.Bov, Bfno)
    Bvv = np.einsum("aA,Qab,bB->QAB", Bfno, p.Bvv, Bfno, optimize=True)
    N, lam = naf_basis(Bvv, naf_thresh)
    o = p.o
    vp = eps_fno.size
    n = o + vp
    Bt = np.zeros((N.shape[1], n, n))
    Bt[:, :o, :o] = np.einsum("QP,Qij->Pij", N, p.Boo)
    Bt[:, :o, o:] = np.einsum("QP,Qia->Pia", N, Bov)
    Bt[:, o:, :o] = Bt[:, :o, o:].transpose(0, 2, 1)
    Bt[:, o:, o:] = np.einsum("QP,Qab->Pab", N, Bvv)
    return R.Problem(p.eo, eps_fno, Bt), N


def solve(p: R.Problem, nroots, order=3, x3=1.0, tol=1e-8, explicit=None):
    """Lowest roots of EA-ADC(order): dense diagonalisation when `explicit`
    (default: dimension <= 3000), Davidson with the DF sigma otherwise."""
    dim = p.v + p.o * p.v * p.v
    if explicit is None:
        explicit = dim <= 3000
    if explicit:
        M = R.explicit_matrix(p, order, x3)
        w, U = np.linalg.eigh(M)
        return w[:nroots], U[:, :nroots]
    sig = R.Sigma(p, order, x3)
    th, X, rn, it = davidson(sig, sig.diagonal(), nroots, tol=tol)
    return th, X


def ss_fno_ea(p: R.Problem, nstates, nroots, fno_thresh, naf_thresh, x3=1.0, tol=1e-8):
    """Full SS-FNO-EA-ADC(3) energies for the nstates lowest canonical ADC(2) roots.

    Returns dict with per-state arrays: omega3 (uncorrected), omega_corr,
    omega2_can, omega2_fno, vprime, nauxprime, and the per-state transforms.
    """
    w2c, X2c = solve(p, nstates, order=2, tol=tol)
    Dmp2 = mp2_density(p)
    v = p.v
    out = {k: [] for k in ("omega3", "omega_corr", "omega2_can", "omega2_fno", "vprime",
                           "nauxprime", "Bfno", "eps_fno", "Nnaf", "omega3_roots")}
    for k in range(nstates):
        y = X2c[:v, k]
        W = X2c[v:, k].reshape(p.o, v, v)
        nrm = np.sqrt(y @ y + np.sum(W * W))
        y, W = y / nrm, W / nrm
        Dss = Dmp2 + ea_density(y, W)
        th_f = fno_thresh[k] if np.ndim(fno_thresh) else fno_thresh
        th_n = naf_thresh[k] if np.ndim(naf_thresh) else naf_thresh
        Bfno, efno, _ = fno_basis(Dss, p.ev, th_f)
        pt, N = truncated_problem(p, Bfno, efno, th_n)
        ref = Bfno.T @ y
        w3, X3 = solve(pt, nroots, order=3, x3=x3, tol=tol)
        w2, X2 = solve(pt, nroots, order=2, tol=tol)
        vp = efno.size

        def pick(X):
            ov = np.abs(ref @ X[:vp])
            return int(np.argmax(ov + 1e-12 * np.arange(ov.size)[::-1]))

        r3, r2 = pick(X3), pick(X2)
        out["omega3"].append(w3[r3])
        out["omega2_fno"].append(w2[r2])
        out["omega2_can"].append(w2c[k])
        out["omega_corr"].append(w3[r3] + w2c[k] - w2[r2])
        out["vprime"].append(vp)
        out["nauxprime"].append(N.shape[1])
        out["Bfno"].append(Bfno)
        out["eps_fno"].append(efno)
        out["Nnaf"].append(N)
        out["omega3_roots"].append(w3)
    for k in ("omega3", "omega_corr", "omega2_can", "omega2_fno", "vprime", "nauxprime"):
        out[k] = np.array(out[k])
    return out
