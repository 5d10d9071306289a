"""Brute-force intermediate-state representation (ISR) of the (N+1)-electron
secular matrix, for pinning the analytic EA-ADC blocks.

Sec. II.A (Eq. 1-6): the correlated ground state Psi_0 is acted on by the
electron-attachment operators {c_a^+, c_b^+ c_c^+ c_k, ...} (Eq. 2); the
resulting precursor states are Gram-Schmidt orthogonalised against the lower
excitation class and then symmetrically orthonormalised within their class
(excitation-class-orthonormalised, ECO, states); M_AB = <Psi~_A|H - E_0|Psi~_B>
(Eq. 3).  Eq. 5 expands M in perturbation order.

Here everything is exact on tiny systems: H(lam) = H0 + lam*V in the full N and
N+1 electron determinant spaces, H0 the Moller-Plesset operator
sum_p e_p p^+ p, V = H - H0, with H the normal-ordered Hamiltonian whose Fock
matrix is diag(e) (Brillouin holds).  M(lam) is analytic near lam = 0; its
Taylor coefficients M^(n) come from a Cauchy contour integral evaluated with
the trapezoidal rule on |lam| = r.  For complex lam every inner product is the
bilinear (transpose) one, so every step is an analytic function of lam.

Spin-orbital index P = 2p + sigma (sigma = 0 alpha, 1 beta); occupied spatial
orbitals are 0..o-1, so spin orbitals 0..2o-1 are occupied in Phi_0.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla


def spinorb_integrals(eps: np.ndarray, B: np.ndarray):
    """Spin-orbital <PQ||RS> and orbital energies from spatial e_p, B^Q_pq.

    (pq|rs) = sum_Q B^Q_pq B^Q_rs (Eq. 25); <PQ|RS> = (pr|qs) d(sP,sR) d(sQ,sS).
    """
    n = eps.size
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)
    sp = np.repeat(np.arange(n), 2)
    sg = np.tile([0, 1], n)
    chem = eri[np.ix_(sp, sp, sp, sp)]
    same = (sg[:, None] == sg[None, :]).astype(float)
    chem = chem * same[:, :, None, None] * same[None, None, :, :]
    phys = chem.transpose(0, 2, 1, 3)            # <PQ|RS> = (PR|QS)
    g = phys - phys.transpose(0, 1, 3, 2)
    return np.repeat(eps, 2), g


def _sign_annihilate(det: int, P: int) -> int:
    return -1 if bin(det & ((1 << P) - 1)).count("1") & 1 else 1


def apply_string(ops, det: int):
    """Apply a product of operators (rightmost first) to a determinant.

    ops: list of (P, dagger) read left to right as written, e.g.
    [(b,1),(c,1),(k,0)] is c_b^+ c_c^+ c_k.  Returns (sign, det) or (0, None).
    """
    sign = 1
    for P, dag in reversed(ops):
        bit = 1 << P
        if dag:
            if det & bit:
                return 0, None
            sign *= _sign_annihilate(det, P)
            det |= bit
        else:
            if not det & bit:
                return 0, None
            sign *= _sign_annihilate(det, P)
            det &= ~bit
    return sign, det


def determinants(nso: int, nel: int):
    dets = []
    for occ in itertools.combinations(range(nso), nel):
        d = 0
        for P in occ:
            d |= 1 << P
        dets.append(d)
    return dets


def hamiltonian(dets, h: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Dense FCI matrix of sum h_PQ P^+Q + 1/4 sum <PQ||RS> P^+Q^+SR (Slater-Condon)."""
    nso = h.shape[0]
    index = {d: i for i, d in enumerate(dets)}
    H = np.zeros((len(dets), len(dets)))
    for col, d in enumerate(dets):
        occ = [P for P in range(nso) if d >> P & 1]
        vir = [P for P in range(nso) if not d >> P & 1]
        H[col, col] = sum(h[I, I] for I in occ) + 0.5 * sum(g[I, J, I, J] for I in occ for J in occ)
        for I in occ:
            for A in vir:
                s, d2 = apply_string([(A, 1), (I, 0)], d)
                val = h[A, I] + sum(g[A, J, I, J] for J in occ if J != I)
                H[index[d2], col] += s * val
        for I, J in itertools.combinations(occ, 2):
            for A, Bb in itertools.combinations(vir, 2):
                s, d2 = apply_string([(A, 1), (Bb, 1), (J, 0), (I, 0)], d)
                H[index[d2], col] += s * g[A, Bb, I, J]
    return H


def operator_matrix(ops, dets_in, dets_out) -> np.ndarray:
    index = {d: i for i, d in enumerate(dets_out)}
    M = np.zeros((len(dets_out), len(dets_in)))
    for col, d in enumerate(dets_in):
        s, d2 = apply_string(ops, d)
        if s:
            M[index[d2], col] = s
    return M


class ISRSystem:
    """Exact N and N+1 electron Hamiltonians of a tiny closed-shell system."""

    def __init__(self, o: int, eps: np.ndarray, B: np.ndarray):
        self.o = o
        self.n = eps.size
        self.eps_so, self.g = spinorb_integrals(eps, B)
        nso = 2 * self.n
        self.nso = nso
        nocc = 2 * o
        self.occ = list(range(nocc))
        self.vir = list(range(nocc, nso))
        # one-body part chosen so that the Fock matrix is exactly diag(e)
        h = np.diag(self.eps_so) - np.einsum("pIqI->pq", self.g[:, :nocc, :, :nocc])
        self.detN = determinants(nso, nocc)
        self.detN1 = determinants(nso, nocc + 1)
        self.phi0 = self.detN.index((1 << nocc) - 1)
        HN = hamiltonian(self.detN, h, self.g)
        HN1 = hamiltonian(self.detN1, h, self.g)
        e0N = np.array([sum(self.eps_so[P] for P in range(nso) if d >> P & 1) for d in self.detN])
        e0N1 = np.array([sum(self.eps_so[P] for P in range(nso) if d >> P & 1) for d in self.detN1])
        self.H0N, self.VN = np.diag(e0N), HN - np.diag(e0N)
        self.H0N1, self.VN1 = np.diag(e0N1), HN1 - np.diag(e0N1)
        self.E00 = e0N[self.phi0]
        # class 1: c_A^+ ; class 2: c_B^+ c_C^+ c_K with B < C
        self.one_p = list(self.vir)
        self.two_p1h = [(K, Bv, C) for K in self.occ for Bv, C in itertools.combinations(self.vir, 2)]
        self.P1 = [operator_matrix([(A, 1)], self.detN, self.detN1) for A in self.one_p]
        self.P2 = [operator_matrix([(Bv, 1), (C, 1), (K, 0)], self.detN, self.detN1)
                   for (K, Bv, C) in self.two_p1h]

    def ground_state(self, lam: complex):
        H = self.H0N + lam * self.VN
        w, U = sla.eig(H)
        k = int(np.argmin(np.abs(w - self.E00)))
        psi = U[:, k]
        psi = psi / np.sqrt(psi @ psi)
        if psi[self.phi0].real < 0:
            psi = -psi
        return w[k], psi

    def secular(self, lam: complex) -> np.ndarray:
        """ISR matrix over the 1p + 2p1h classes at coupling strength lam."""
        E0, psi = self.ground_state(lam)
        X1 = np.stack([Pm @ psi for Pm in self.P1], axis=1)
        X2 = np.stack([Pm @ psi for Pm in self.P2], axis=1)
        Q1 = X1 @ sla.fractional_matrix_power(X1.T @ X1, -0.5)
        X2g = X2 - Q1 @ (Q1.T @ X2)
        Q2 = X2g @ sla.fractional_matrix_power(X2g.T @ X2g, -0.5)
        Q = np.concatenate([Q1, Q2], axis=1)
        H = self.H0N1 + lam * self.VN1
        return Q.T @ (H @ Q) - E0 * (Q.T @ Q)

    def taylor(self, nmax: int = 3, r: float = 0.25, npts: int = 24):
        """Taylor coefficients M^(0..nmax) of the ISR matrix (Eq. 5)."""
        lams = r * np.exp(2j * np.pi * np.arange(npts) / npts)
        Ms = np.stack([self.secular(l) for l in lams])
        coef = []
        for nn in range(nmax + 1):
            c = np.tensordot(np.exp(-2j * np.pi * nn * np.arange(npts) / npts), Ms, axes=1) / (npts * r ** nn)
            coef.append(c)
        return coef
