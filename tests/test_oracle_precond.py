"""Pins of the learned-correction oracle (CPU): backpropagation against
central finite differences, the zero-output network against the plain
diagonal correction, the loss against its closed form for parallel and
orthogonal directions, and the exact-correction target against its
defining properties."""
import numpy as np

from oracle import precond as P
from oracle import restricted as R
from synth import make_problem


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in P.SHAPES:
        p[name] = rng.standard_normal(shp) * scale / np.sqrt(shp[-1] if len(shp) > 1 else 4)
    return p


def _data(seed, nseg=3, rows=(7, 5, 9)):
    rng = np.random.default_rng(seed)
    n = sum(rows)
    F = rng.standard_normal((n, P.NF))
    rr = rng.standard_normal(n)
    base = rng.standard_normal(n)
    T = rng.standard_normal(n)
    segs = np.concatenate([[0], np.cumsum(rows)])
    return segs, F, rr, base, T


def test_backprop_matches_finite_differences():
    p = _params(1)
    segs, F, rr, base, T = _data(2)
    L, g = P.loss_grad(p, segs, F, rr, base, T)
    assert abs(L - P.loss(p, segs, F, rr, base, T)) < 1e-14
    flat = P.pack(p)
    rng = np.random.default_rng(3)
    # every bias and output weight, and random entries of each weight matrix
    offs, o = [], 0
    for name, shp in P.SHAPES:
        n = int(np.prod(shp))
        idx = np.arange(n) if len(shp) == 1 else rng.choice(n, 12, replace=False)
        offs += list(o + idx)
        o += n
    h = 1e-6
    for i in offs:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        num = (P.loss(P.unpack(fp), segs, F, rr, base, T) - P.loss(P.unpack(fm), segs, F, rr, base, T)) / (2 * h)
        assert abs(num - g[i]) <= 1e-7 + 1e-5 * abs(num), (i, num, g[i])


def test_zero_output_layer_is_the_diagonal_correction():
    pr = make_problem(2, 5, 9, 3.0, 4)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    sig = R.Sigma(p, 3)
    D = sig.diagonal()
    dim = D.size
    r = np.random.default_rng(0).standard_normal(dim)
    theta = D.min() + 0.01
    D[3] = theta + 1e-12  # the guarded denominator
    F, rr, base = P.features(r, D, theta, p.o, p.v, p.eo, p.ev, P.ladder_diagonal(p.Bvv))
    net = _params(5)
    net["w4"][:] = 0.0
    net["b4"][:] = 0.0
    m, _ = P.forward(net, F)
    delta = base + rr * m
    ref = r / P.guarded(theta - D) / np.linalg.norm(r)
    assert np.array_equal(m, np.zeros(dim))
    assert np.allclose(delta, ref, rtol=1e-15, atol=0)
    assert abs(delta[3] + rr[3] * 1e8) <= 1e-6 * abs(delta[3])  # theta - D = -1e-12 -> -1e-8
    # feature columns: element energies in the (k, b, c) layout
    k, b, c = 1, 3, 2
    i = p.v + (k * p.v + b) * p.v + c
    assert F[i, 3] == p.eo[k] and F[i, 4] == np.arcsinh(p.ev[b]) and F[i, 5] == np.arcsinh(p.ev[c])
    assert F[:p.v, 8].sum() == p.v and F[p.v:, 8].sum() == 0
    assert F[:, 9].sum() == p.o * p.v


def test_ladder_feature_is_the_ladder_diagonal():
    """Feature 10 of element (k, b, c) is the ladder's response to the unit
    vector at (k, b, c), read at (k, b, c)."""
    pr = make_problem(2, 4, 7, 3.0, 6)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    lad = P.ladder_diagonal(p.Bvv)
    dim = p.v + p.o * p.v * p.v
    F, _, _ = P.features(np.ones(dim), np.zeros(dim), -1.0, p.o, p.v, p.eo, p.ev, lad)
    for k, b, c in [(0, 0, 0), (1, 2, 3), (0, 3, 1)]:
        w = np.zeros((p.o, p.v, p.v))
        w[k, b, c] = 1.0
        resp = R.ladder_w(p, w)[k, b, c]
        assert abs(F[p.v + (k * p.v + b) * p.v + c, 10] - resp) < 1e-14
    assert not F[:p.v, 10].any()


def test_loss_closed_forms():
    net = _params(7)
    segs = np.array([0, 4, 8])
    F = np.random.default_rng(8).standard_normal((8, P.NF))
    m, _ = P.forward(net, F)
    rr = np.ones(8)
    t = np.random.default_rng(9).standard_normal(8)
    # delta parallel to t in segment 0 (loss 0), orthogonal in segment 1 (loss 1)
    T = np.concatenate([t[:4], t[4:]])
    d1 = np.array([t[5], -t[4], t[7], -t[6]])
    base = np.concatenate([3.0 * t[:4], d1]) - rr * m
    assert abs(P.loss(net, segs, F, rr, base, T) - 0.5) < 1e-14


def test_target_is_the_projected_exact_correction():
    rng = np.random.default_rng(11)
    ys = rng.standard_normal(50)
    ys /= np.linalg.norm(ys)
    y = ys + 0.1 * rng.standard_normal(50)
    y /= np.linalg.norm(y)
    t = P.target(y, -ys)  # sign of y* is irrelevant
    assert abs(y @ t) < 1e-14
    # y + t is y* up to its component along y
    a = ys @ y
    assert np.allclose(y + t, ys + y * (1.0 - a), atol=1e-14)
