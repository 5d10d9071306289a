"""Textbook Davidson eigensolver for the lowest roots of a symmetric matrix
given only its matrix-vector product (Sec. II.A: M is diagonalised by
Davidson's method from sigma vectors).

Readings where the paper is silent: guesses are unit vectors on the nroots
lowest diagonal entries; the correction is the diagonal (Davidson)
preconditioner r / (theta - D) with |theta - D| floored at 1e-8; new
directions are orthogonalised twice by classical Gram-Schmidt against the
subspace; the subspace restarts from the current 2*nroots Ritz vectors when it
would exceed max_sub; convergence when every ||r||_2 <= tol and every Ritz
value moved by at most etol.
"""
from __future__ import annotations

import numpy as np


def _block(matvec, V):
    """matvec on the columns of V; matvec takes [nvec, n] rows."""
    return np.asarray(matvec(np.ascontiguousarray(V.T))).T.copy()


def davidson(matvec, diag, nroots, tol=1e-6, etol=1e-10, max_sub=None, maxit=200, guess=None):
    n = diag.size
    nroots = min(nroots, n)
    if max_sub is None:
        max_sub = max(8 * nroots, 40)
    max_sub = min(max_sub, n)
    if guess is None:
        V = np.zeros((n, nroots))
        for c, i in enumerate(np.argsort(diag, kind="stable")[:nroots]):
            V[i, c] = 1.0
    else:
        V, _ = np.linalg.qr(np.asarray(guess, dtype=np.float64).reshape(n, -1))
    S = _block(matvec, V)
    theta_old = np.full(nroots, np.inf)
    for it in range(1, maxit + 1):
        G = V.T @ S
        G = 0.5 * (G + G.T)
        th, U = np.linalg.eigh(G)
        th, U = th[:nroots], U[:, :nroots]
        X = V @ U
        R = S @ U - X * th
        rn = np.linalg.norm(R, axis=0)
        if np.all(rn <= tol) and np.all(np.abs(th - theta_old) <= etol):
            return th, X, rn, it
        theta_old = th.copy()
        new = []
        for c in range(nroots):
            if rn[c] <= tol:
                continue
            den = th[c] - diag
            den = np.where(np.abs(den) < 1e-8, np.where(den < 0, -1e-8, 1e-8), den)
            new.append(R[:, c] / den)
        if V.shape[1] + len(new) > max_sub:
            keep = min(2 * nroots, V.shape[1])
            _, Uk = np.linalg.eigh(G)
            V = V @ Uk[:, :keep]
            S = S @ Uk[:, :keep]
        added = []
        for d in new:
            for _ in range(2):
                d = d - V @ (V.T @ d)
                for a in added:
                    d = d - a * (a @ d)
            nd = np.linalg.norm(d)
            if nd > 1e-10:
                added.append(d / nd)
        if not added:
            return th, X, rn, it
        A = np.stack(added, axis=1)
        V = np.concatenate([V, A], axis=1)
        S = np.concatenate([S, _block(matvec, A)], axis=1)
    return th, X, rn, maxit
