"""Learned Davidson correction: per-element MLP oracle (test infrastructure
only; never imported by the product path).

The correction of a Davidson root with Ritz value theta and residual r is the
diagonal one, delta_I = r_I / (theta - D_I) (|theta - D_I| < 1e-8 set to
+-1e-8), plus a learned term: delta_I = rr_I (1 / (theta - D_I) + m_I) with
rr = r / ||r|| and m_I = MLP(f_I), a network of three tanh layers of width 256
and a linear output, applied to each element's feature vector f_I:

  f0 = rr_I sqrt(dim)           f1 = asinh(D_I - theta)
  f2 = clip(1/(theta - D_I), +-100) / 100
  f3 = eps_k (2p1h; 0 for 1p)   f4 = asinh(eps_b) (1p: asinh(eps_a))
  f5 = asinh(eps_c) (1p: 0)     f6 = theta       f7 = log10 ||r||
  f8 = 1 for a 1p element       f9 = 1 for a 2p1h element with b = c
  f10..f15 = 0.

Training target (one per Ritz vector y of an iteration, with the converged
eigenvector y* of the same root, sign-aligned so that y . y* >= 0): the exact
correction projected off y, t = (I - y y^T)(y* - y).  Loss per vector: one
minus the squared cosine between delta and t (the expansion vector is
normalised, so only its direction matters); the batch loss is the mean.

With the output layer zero the correction is exactly the diagonal one.
"""
from __future__ import annotations

import numpy as np

NF = 16
WIDTH = 256
SHAPES = [("W1", (WIDTH, NF)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("w4", (WIDTH,)), ("b4", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    """Parameter dict from the flat FP32 layout W1, b1, W2, b2, W3, b3, w4, b4."""
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def guarded(den):
    den = np.array(den, dtype=np.float64)
    small = np.abs(den) < 1e-8
    den[small] = np.where(den[small] < 0, -1e-8, 1e-8)
    return den


def element_energies(o, v, eo, ev):
    """(eps_k, eps_b, eps_c, is_1p, is_diag) for every element of a vector."""
    dim = v + o * v * v
    ek = np.zeros(dim)
    eb = np.zeros(dim)
    ec = np.zeros(dim)
    one = np.zeros(dim)
    dg = np.zeros(dim)
    eb[:v] = ev
    one[:v] = 1.0
    k, b, c = np.meshgrid(np.arange(o), np.arange(v), np.arange(v), indexing="ij")
    ek[v:] = eo[k.ravel()]
    eb[v:] = ev[b.ravel()]
    ec[v:] = ev[c.ravel()]
    dg[v:] = (b.ravel() == c.ravel()).astype(float)
    return ek, eb, ec, one, dg


def ladder_diagonal(Bvv):
    """(bb|cc) = sum_Q B^Q_bb B^Q_cc, [v, v]."""
    d = np.einsum("Qbb->Qb", Bvv)
    return d.T @ d


def features(r, D, theta, o, v, eo, ev, lad=None):
    """Feature matrix [dim, 16], normalised residual rr and diagonal term
    rr/(theta - D); lad = ladder_diagonal(B_vv) (zeros when None)."""
    dim = v + o * v * v
    rn = np.linalg.norm(r)
    rr = r / rn
    den = guarded(theta - D)
    ek, eb, ec, one, dg = element_energies(o, v, eo, ev)
    f = np.zeros((dim, NF))
    f[:, 0] = rr * np.sqrt(dim)
    f[:, 1] = np.arcsinh(D - theta)
    f[:, 2] = np.clip(1.0 / den, -100.0, 100.0) / 100.0
    f[:, 3] = ek
    f[:, 4] = np.arcsinh(eb)
    f[:, 5] = np.where(one > 0, 0.0, np.arcsinh(ec))
    f[:, 6] = theta
    f[:, 7] = np.log10(rn)
    f[:, 8] = one
    f[:, 9] = dg
    if lad is not None:
        f[v:, 10] = np.broadcast_to(lad, (o, v, v)).ravel()
    return f, rr, rr / den


def target(y, ystar):
    """Exact correction projected off y, with y* sign-aligned to y."""
    if y @ ystar < 0:
        ystar = -ystar
    d = ystar - y
    return d - y * (y @ d)


def forward(p, F):
    """m = w4 . tanh(W3 tanh(W2 tanh(W1 f + b1) + b2) + b3) + b4 per row of F."""
    h1 = np.tanh(F @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    h3 = np.tanh(h2 @ p["W3"].T + p["b3"])
    return h3 @ p["w4"] + p["b4"][0], (h1, h2, h3)


def loss(p, segs, F, rr, base, T):
    """Mean over vectors (row ranges segs[j]:segs[j+1]) of 1 - cos^2(delta, t),
    delta = base + rr * m."""
    m, _ = forward(p, F)
    delta = base + rr * m
    L = 0.0
    for j in range(len(segs) - 1):
        a, b = segs[j], segs[j + 1]
        d, t = delta[a:b], T[a:b]
        L += 1.0 - (d @ t) ** 2 / ((d @ d) * (t @ t))
    return L / (len(segs) - 1)


def loss_grad(p, segs, F, rr, base, T):
    """Loss and its gradient (flat, same layout as pack) by backpropagation."""
    m, (h1, h2, h3) = forward(p, F)
    delta = base + rr * m
    nseg = len(segs) - 1
    gd = np.zeros_like(delta)
    L = 0.0
    for j in range(nseg):
        a, b = segs[j], segs[j + 1]
        d, t = delta[a:b], T[a:b]
        c, dd, tt = d @ t, d @ d, t @ t
        L += 1.0 - c * c / (dd * tt)
        gd[a:b] = (-2.0 * c / (dd * tt) * t + 2.0 * c * c / (dd * dd * tt) * d) / nseg
    L /= nseg
    gm = gd * rr
    g = {"w4": h3.T @ gm, "b4": np.array([gm.sum()])}
    gz3 = np.outer(gm, p["w4"]) * (1.0 - h3 ** 2)
    g["W3"] = gz3.T @ h2
    g["b3"] = gz3.sum(0)
    gz2 = (gz3 @ p["W3"]) * (1.0 - h2 ** 2)
    g["W2"] = gz2.T @ h1
    g["b2"] = gz2.sum(0)
    gz1 = (gz2 @ p["W2"]) * (1.0 - h1 ** 2)
    g["W1"] = gz1.T @ F
    g["b1"] = gz1.sum(0)
    return L, pack(g)


def adam(flat, grad, mom, vel, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) in place; step counts from 1."""
    mom[:] = b1 * mom + (1 - b1) * grad
    vel[:] = b2 * vel + (1 - b2) * grad * grad
    mh = mom / (1 - b1 ** step)
    vh = vel / (1 - b2 ** step)
    flat -= lr * mh / (np.sqrt(vh) + eps)
    return flat
