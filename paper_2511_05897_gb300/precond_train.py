"""Training of the learned Davidson correction on pairs the method generates.

For each seeded problem the GPU Davidson is run with its trace on; every
recorded Ritz vector y (with residual r and Ritz value theta) is paired with
the converged eigenvector y* of the same root, and eaadc_precond_pairs turns
the pair into per-element features, the diagonal term and the exact-correction
target.  Training runs eaadc_mlp_train_step (forward, backward and Adam in the
library's kernels) over mini-batches of whole vectors.  PyTorch only holds the
device buffers.

    from paper_2511_05897_gb300 import precond_train as T
    w = T.train(T.make_pairs([(5, 20, 60, 15.0, s) for s in range(1, 51)]))
"""
from __future__ import annotations

import numpy as np

from . import _lib as L


def init_weights(seed=0):
    """Glorot-uniform tanh layers; zero output layer, so the untrained network
    reproduces the diagonal correction exactly."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((256, L.MLP_FEATURES), (256, 256), (256, 256)):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        parts += [rng.uniform(-a, a, (fan_out, fan_in)).ravel(), np.zeros(fan_out)]
    parts += [np.zeros(256), np.zeros(1)]
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == L.MLP_PARAMS
    return w


def _problem(spec):
    from synth import make_problem

    return make_problem(*spec)


def make_pairs(specs, nroots=4, trace=30, tol=1e-9, order=3, device=0, min_overlap=0.5, min_resnorm=1e-7):
    """Training pairs from the problems in specs ((o, v, naux, decay, seed)
    tuples).  Returns a dict of device tensors feat [N,16], rr, base, target
    [N] and the vector boundaries segs (host int32 [nvec+1])."""
    import torch

    feats, rrs, bases, tgts, segs = [], [], [], [], [0]
    for spec in specs:
        pr = _problem(spec)
        ctx = L.eaadc_init(pr["o"], pr["v"], pr["naux"], pr["eps_occ"], pr["eps_vir"], pr["B"], device)
        try:
            L.eaadc_build_canonical(ctx, order, 1.0)
            L.eaadc_davidson(ctx, nroots, tol=tol, maxit=300, trace=trace)
            X, R, th = L.eaadc_get_trace(ctx, 0)
            Ys = L.eaadc_get_eigvecs(ctx, 0, nroots)
            dim = Ys.shape[1]
            keep = []
            for t in range(X.shape[0]):
                for r in range(X.shape[1]):
                    if abs(X[t, r] @ Ys[r]) >= min_overlap and np.linalg.norm(R[t, r]) >= min_resnorm:
                        keep.append((t, r))
            if not keep:
                continue
            y = torch.tensor(np.stack([X[t, r] for t, r in keep]), device="cuda")
            rr_ = torch.tensor(np.stack([R[t, r] for t, r in keep]), device="cuda")
            ys = torch.tensor(np.stack([Ys[r] for t, r in keep]), device="cuda")
            thv = np.array([th[t, r] for t, r in keep])
            nv = len(keep)
            f = torch.empty((nv * dim, L.MLP_FEATURES), dtype=torch.float32, device="cuda")
            a = torch.empty(nv * dim, dtype=torch.float32, device="cuda")
            b = torch.empty_like(a)
            tg = torch.empty_like(a)
            L.eaadc_precond_pairs(ctx, 0, nv, y.data_ptr(), rr_.data_ptr(), thv, ys.data_ptr(), f.data_ptr(),
                                  a.data_ptr(), b.data_ptr(), tg.data_ptr(), torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            feats.append(f)
            rrs.append(a)
            bases.append(b)
            tgts.append(tg)
            for _ in range(nv):
                segs.append(segs[-1] + dim)
        finally:
            L.eaadc_destroy(ctx)
    return {"feat": torch.cat(feats), "rr": torch.cat(rrs), "base": torch.cat(bases), "target": torch.cat(tgts),
            "segs": np.array(segs, dtype=np.int64)}


def _batch(data, lo, hi):
    s = data["segs"]
    a, b = int(s[lo]), int(s[hi])
    segs = (s[lo:hi + 1] - a).astype(np.int32)
    return segs, data["feat"][a:b], data["rr"][a:b], data["base"][a:b], data["target"][a:b]


def loss(ctx, data, batch=64):
    """Mean loss over all vectors of data with the loaded weights."""
    import torch

    nvec = len(data["segs"]) - 1
    tot = 0.0
    for lo in range(0, nvec, batch):
        hi = min(nvec, lo + batch)
        segs, f, a, b, t = _batch(data, lo, hi)
        Lb, _ = L.eaadc_mlp_loss_grad(ctx, segs, f.data_ptr(), a.data_ptr(), b.data_ptr(), t.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        tot += Lb * (hi - lo)
    return tot / nvec


def train(data, epochs=8, batch=64, lr=1e-3, seed=0, device=0, weights=None, log=None):
    """Trains from init_weights(seed) (or weights) and returns the FP32 weights."""
    import torch

    from synth import make_problem

    pr = make_problem(1, 1, 1, 1.0, 1)  # any context holds a network
    ctx = L.eaadc_init(1, 1, 1, pr["eps_occ"], pr["eps_vir"], pr["B"], device)
    try:
        L.eaadc_precond_load(ctx, init_weights(seed) if weights is None else weights)
        nvec = len(data["segs"]) - 1
        order = np.random.default_rng(seed).permutation((nvec + batch - 1) // batch)
        stream = torch.cuda.current_stream().cuda_stream
        for ep in range(epochs):
            tot = 0.0
            for bi in order:
                lo, hi = bi * batch, min(nvec, (bi + 1) * batch)
                segs, f, a, b, t = _batch(data, lo, hi)
                tot += (hi - lo) * L.eaadc_mlp_train_step(ctx, segs, f.data_ptr(), a.data_ptr(), b.data_ptr(),
                                                          t.data_ptr(), lr, stream)
            if log:
                log(f"epoch {ep}: mean loss {tot / nvec:.4f}")
        return L.eaadc_precond_get(ctx)
    finally:
        L.eaadc_destroy(ctx)
