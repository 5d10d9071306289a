"""GPU parity of the learned Davidson correction against its CPU oracle
(features, exact-correction targets, forward pass, loss and gradient), the
effect of GPU training, and what the trained network gains over the diagonal
correction inside the Davidson solver.

Tolerances: features and targets are FP64 values rounded to FP32 (relative
2^-24); the network runs FP32 GEMMs with 16- to n-term sums, held to 1e-5 of
the largest output and 2e-4 of the largest gradient component against the
FP64 oracle."""
import numpy as np
import pytest

from synth import make_problem
from oracle import precond as P
from oracle import restricted as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import __graft_entry__ as g

    g.build()
    import paper_2511_05897_gb300 as mod

    return mod


def _net(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in P.SHAPES:
        fan = shp[-1] if len(shp) > 1 else 16
        p[name] = rng.standard_normal(shp) * scale / np.sqrt(fan)
    return p


def _traced(E, o, v, naux, seed, nroots=3, trace=4):
    pr = make_problem(o, v, naux, 3.0, seed)
    ctx = E.eaadc_init(o, v, naux, pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    E.eaadc_build_canonical(ctx, 3, 1.0)
    E.eaadc_davidson(ctx, nroots, tol=1e-10, maxit=300, trace=trace)
    X, Rs, th = E.eaadc_get_trace(ctx, 0)
    Ys = E.eaadc_get_eigvecs(ctx, 0, nroots)
    return pr, ctx, X, Rs, th, Ys


def _pairs(E, ctx, y, r, th, ys):
    import torch

    nv, dim = y.shape
    d = lambda a: torch.tensor(a, device="cuda:0")  # noqa: E731
    yd, rd, ysd = d(y), d(r), d(ys)
    f = torch.empty((nv * dim, 16), dtype=torch.float32, device="cuda:0")
    a = torch.empty(nv * dim, dtype=torch.float32, device="cuda:0")
    b, t = torch.empty_like(a), torch.empty_like(a)
    E.eaadc_precond_pairs(ctx, 0, nv, yd.data_ptr(), rd.data_ptr(), th, ysd.data_ptr(), f.data_ptr(), a.data_ptr(),
                          b.data_ptr(), t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f, a, b, t


def test_pairs_and_forward_match_oracle(E):
    import torch

    o, v, naux = 2, 5, 9
    pr, ctx, X, Rs, th, Ys = _traced(E, o, v, naux, 4)
    try:
        p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
        D = E.eaadc_diagonal(ctx, 0)
        assert X.shape[0] == 4 and X.shape[1] == 3
        t_it = 2
        f, a, b, t = _pairs(E, ctx, X[t_it], Rs[t_it], th[t_it], Ys)
        dim = D.size
        for r in range(3):
            Fo, rro, baseo = P.features(Rs[t_it, r], D, th[t_it, r], o, v, p.eo, p.ev, P.ladder_diagonal(p.Bvv))
            sl = slice(r * dim, (r + 1) * dim)
            assert np.allclose(f[sl].cpu().numpy(), Fo, rtol=2e-7, atol=2e-7 * np.abs(Fo).max())
            assert np.allclose(a[sl].cpu().numpy(), rro, rtol=2e-7, atol=1e-12)
            assert np.allclose(b[sl].cpu().numpy(), baseo, rtol=2e-7, atol=1e-12)
            to = P.target(X[t_it, r], Ys[r])
            assert np.allclose(t[sl].cpu().numpy(), to, rtol=2e-7, atol=2e-7 * np.abs(to).max())
        # forward pass of a random network
        net = _net(1)
        E.eaadc_precond_load(ctx, P.pack(net).astype(np.float32))
        m = torch.empty(f.shape[0], dtype=torch.float32, device="cuda:0")
        E.eaadc_mlp_forward(ctx, f.shape[0], f.data_ptr(), m.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        w32 = P.unpack(P.pack(net).astype(np.float32))
        mo, _ = P.forward(w32, f.cpu().numpy().astype(np.float64))
        assert np.abs(m.cpu().numpy() - mo).max() <= 1e-5 * np.abs(mo).max()
    finally:
        E.eaadc_destroy(ctx)


def test_loss_and_gradient_match_oracle(E):
    o, v, naux = 2, 6, 10
    pr, ctx, X, Rs, th, Ys = _traced(E, o, v, naux, 6)
    try:
        y = np.concatenate([X[1], X[3]])
        r = np.concatenate([Rs[1], Rs[3]])
        thv = np.concatenate([th[1], th[3]])
        ys = np.concatenate([Ys, Ys])
        f, a, b, t = _pairs(E, ctx, y, r, thv, ys)
        dim = X.shape[2]
        segs = np.arange(0, 7) * dim
        net = _net(2, 0.7)
        w32 = P.pack(net).astype(np.float32)
        E.eaadc_precond_load(ctx, w32)
        L, g = E.eaadc_mlp_loss_grad(ctx, segs, f.data_ptr(), a.data_ptr(), b.data_ptr(), t.data_ptr())
        Lo, go = P.loss_grad(P.unpack(w32), segs, f.cpu().numpy().astype(np.float64), a.cpu().numpy().astype(np.float64),
                             b.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64))
        assert abs(L - Lo) <= 1e-5 * max(1.0, abs(Lo))
        assert np.abs(g - go).max() <= 2e-4 * np.abs(go).max()
        # a train step moves the weights against the gradient (Adam, first step: -lr * sign)
        E.eaadc_mlp_train_step(ctx, segs, f.data_ptr(), a.data_ptr(), b.data_ptr(), t.data_ptr(), 1e-3)
        w1 = E.eaadc_precond_get(ctx)
        big = np.abs(go) > 1e-3 * np.abs(go).max()
        assert np.allclose((w1 - w32)[big], -1e-3 * np.sign(go[big]), rtol=1e-3, atol=1e-7)
    finally:
        E.eaadc_destroy(ctx)


def test_bad_network_falls_back_to_the_diagonal(E):
    """A network with large random output weights: every root falls back and
    the solve still converges to the dense eigenvalues."""
    o, v, naux = 2, 6, 10
    pr = make_problem(o, v, naux, 3.0, 9)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    ref = np.linalg.eigvalsh(R.explicit_matrix(p, 3))[:3]
    ctx = E.eaadc_init(o, v, naux, pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    try:
        E.eaadc_build_canonical(ctx, 3, 1.0)
        with pytest.raises(E.EaadcError):  # no weights yet
            E.eaadc_davidson(ctx, 3, tol=1e-8, precond=1)
        net = _net(3, 50.0)
        E.eaadc_precond_load(ctx, P.pack(net).astype(np.float32))
        om, rn, it, st = E.eaadc_davidson(ctx, 3, tol=1e-8, maxit=300, precond=1)
        assert st == 0 and np.abs(om[0] - ref).max() <= 1e-8
    finally:
        E.eaadc_destroy(ctx)


def test_trained_network_against_diagonal(E, capsys):
    """Train on Davidson pairs of 8 seeds of the o=5, v=20, naux=60 problem,
    then solve 4 held-out seeds to ||r|| <= 1e-5 with and without it."""
    from paper_2511_05897_gb300 import precond_train as T

    data = T.make_pairs([(5, 20, 60, 15.0, s) for s in range(1, 9)], trace=30)
    w0 = T.init_weights(0)
    w = T.train(data, epochs=12, batch=32, lr=1e-3, weights=w0)
    pr0 = make_problem(1, 1, 1, 1.0, 1)
    ctx = E.eaadc_init(1, 1, 1, pr0["eps_occ"], pr0["eps_vir"], pr0["B"], 0)
    try:
        E.eaadc_precond_load(ctx, w0)
        l0 = T.loss(ctx, data)
        E.eaadc_precond_load(ctx, w)
        l1 = T.loss(ctx, data)
    finally:
        E.eaadc_destroy(ctx)
    assert l1 < l0  # training lowers the loss below the diagonal correction's
    its = {0: [], 1: []}
    for seed in range(1001, 1005):
        pr = make_problem(5, 20, 60, 15.0, seed)
        ctx = E.eaadc_init(5, 20, 60, pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
        try:
            E.eaadc_build_canonical(ctx, 3, 1.0)
            E.eaadc_precond_load(ctx, w)
            res = {}
            for pc in (0, 1):
                om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-5, etol=1e-6, maxit=300, precond=pc)
                assert st == 0
                res[pc] = om[0]
                its[pc].append(int(it[0]))
            assert np.abs(res[0] - res[1]).max() <= 1e-8
        finally:
            E.eaadc_destroy(ctx)
    with capsys.disabled():
        print(f"\nlearned correction: loss {l0:.4f} -> {l1:.4f}; Davidson iterations to 1e-5, "
              f"diagonal {its[0]} vs learned {its[1]}")
    assert sum(its[1]) <= sum(its[0]) + 4
