"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  FP64 mode: elementwise to ~1e-12 relative for sigma and
the 1p/1p block, eigenvalues to 1e-8 Eh."""
import os

import numpy as np
import pytest

from synth import config_problem, make_problem
from oracle import restricted as R

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def E():
    import __graft_entry__ as g

    g.build()
    import paper_2511_05897_gb300 as mod

    return mod


def _ctx(E, pr, order=3, x3=1.0):
    ctx = E.eaadc_init(pr["o"], pr["v"], pr["naux"], pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    E.eaadc_build_canonical(ctx, order, x3)
    return ctx


# sizes: degenerate, ragged, several 64-wide GEMM tiles with a tail
CASES = [(1, 1, 1, 1.0, 2), (1, 2, 3, 2.0, 4), (2, 3, 5, 3.0, 6), (3, 9, 24, 6.0, 5), (4, 13, 40, 8.0, 9),
         (2, 70, 30, 10.0, 3), (5, 20, 60, 15.0, 1)]


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("o,v,naux,decay,seed", CASES)
def test_m11_and_sigma_match_oracle(E, o, v, naux, decay, seed, order):
    pr = make_problem(o, v, naux, decay, seed)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    sig = R.Sigma(p, order)
    ctx = _ctx(E, pr, order)
    try:
        m11 = E.eaadc_get_m11(ctx, 0)
        assert np.abs(m11 - sig.M11).max() <= 1e-12 * np.abs(sig.M11).max()
        vp, npx, dim = E.eaadc_state_info(ctx, 0)
        assert (vp, npx, dim) == (v, naux, v + o * v * v)
        x = np.random.default_rng(seed).standard_normal((3, dim))
        ref = sig(x)
        got = E.eaadc_sigma_host(ctx, 0, x)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        d = E.eaadc_diagonal(ctx, 0)
        assert np.abs(d - sig.diagonal()).max() <= 1e-14 * np.abs(d).max()
    finally:
        E.eaadc_destroy(ctx)


def test_sigma_device_pointers_and_x3(E):
    """eaadc_sigma on caller-owned device buffers; x3 scales only M^(3)."""
    import torch

    pr = make_problem(3, 9, 24, 6.0, 11)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    ctx = _ctx(E, pr, 3, 0.5)
    try:
        M = R.explicit_matrix(p, 3, 0.5)
        x = torch.randn(2, M.shape[0], dtype=torch.float64, device="cuda:0")
        y = torch.empty_like(x)
        E.eaadc_sigma(ctx, 0, 2, x.data_ptr(), y.data_ptr(), E.EAADC_FP64,
                      torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        ref = x.cpu().numpy() @ M
        assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        E.eaadc_destroy(ctx)


def test_davidson_tiny_equals_dense(E):
    pr = config_problem("tiny")
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    ref = np.linalg.eigvalsh(R.explicit_matrix(p, 3))[:4]
    ctx = _ctx(E, pr)
    try:
        om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-8)
        assert st == 0
        assert np.abs(om[0] - ref).max() <= 1e-8
        vecs = E.eaadc_get_eigvecs(ctx, 0, 4)
        assert np.abs(vecs @ vecs.T - np.eye(4)).max() < 1e-10
    finally:
        E.eaadc_destroy(ctx)


def test_davidson_edge_one_virtual(E):
    pr = make_problem(1, 1, 1, 1.0, 2)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    ref = np.linalg.eigvalsh(R.explicit_matrix(p, 3))
    ctx = _ctx(E, pr)
    try:
        om, rn, it, st = E.eaadc_davidson(ctx, 2, tol=1e-10)
        assert np.abs(om[0] - ref[:2]).max() <= 1e-10
    finally:
        E.eaadc_destroy(ctx)


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLD, "canonical-200.npz")), reason="golden file missing")
@pytest.mark.parametrize("order", [2, 3])
def test_canonical_200_fp64_against_oracle(E, order):
    """o=20, v=200, naux=600, 4 roots: 1p/1p block and sampled sigma of seeded
    probes elementwise; FP64 GPU Davidson roots vs the oracle to 1e-8 Eh."""
    import sys
    sys.path.insert(0, GOLD)
    from make_golden import probes

    g = np.load(os.path.join(GOLD, "canonical-200.npz"))
    pr = config_problem("canonical-200")
    ctx = _ctx(E, pr, order)
    try:
        m11 = E.eaadc_get_m11(ctx, 0)
        ref = g[f"m11_{order}"]
        assert np.abs(m11 - ref).max() <= 1e-11 * np.abs(ref).max()
        v, naux, dim = E.eaadc_state_info(ctx, 0)
        x, idx = probes(dim, v)
        assert np.array_equal(idx, g["sample_index"])
        s = E.eaadc_sigma_host(ctx, 0, x)[:, idx]
        sref = g[f"sigma_probe{order}"]
        assert np.abs(s - sref).max() <= 1e-11 * np.abs(sref).max()
        om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-7, max_sub=40, maxit=300)
        assert st == 0
        assert np.abs(om[0] - g[f"omega{order}"]).max() <= 1e-8
    finally:
        E.eaadc_destroy(ctx)


# ---------------------------------------------------------------- mixed path
MIXED_CASES = [(1, 2, 3, 2.0, 4), (4, 13, 40, 8.0, 9), (2, 70, 30, 10.0, 3), (5, 20, 60, 15.0, 1),
               (3, 136, 90, 20.0, 7)]


@pytest.mark.parametrize("o,v,naux,decay,seed", MIXED_CASES)
def test_ladder_tensor_core_vs_oracle(E, o, v, naux, decay, seed):
    """a1 on tcgen05 (BF16 operands, FP32 accumulation) vs the FP64 DF ladder.

    Tolerance: BF16 keeps 8 significant bits (relative rounding 2^-9) on B, on
    w and on the stage-1 intermediate; with FP32 accumulation the error of each
    output stays below ~3 * 2^-9 of the largest |term|, bounded here by 2e-2 of
    max |ladder| for unit-variance inputs."""
    import torch

    pr = make_problem(o, v, naux, decay, seed)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    ctx = _ctx(E, pr)
    try:
        dim = v + o * v * v
        x = np.random.default_rng(seed).standard_normal((2, dim))
        xd = torch.tensor(x, device="cuda:0")
        out = torch.empty((2, o, v, v), dtype=torch.float32, device="cuda:0")
        E.eaadc_ladder(ctx, 0, 2, xd.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        for n in range(2):
            ref = R.ladder_w(p, x[n, v:].reshape(o, v, v)).transpose(0, 2, 1)  # output is [k][c][b]
            assert np.abs(got[n] - ref).max() <= 2e-2 * np.abs(ref).max()
    finally:
        E.eaadc_destroy(ctx)


@pytest.mark.parametrize("o,v,naux,decay,seed", MIXED_CASES)
def test_mixed_sigma_vs_fp64(E, o, v, naux, decay, seed):
    pr = make_problem(o, v, naux, decay, seed)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    ctx = _ctx(E, pr)
    try:
        dim = v + o * v * v
        x = np.random.default_rng(seed + 1).standard_normal((3, dim))
        s64 = E.eaadc_sigma_host(ctx, 0, x, E.EAADC_FP64)
        smx = E.eaadc_sigma_host(ctx, 0, x, E.EAADC_MIXED_BF16)
        scale = max(np.abs(R.ladder_w(p, x[n, v:].reshape(o, v, v)) + R.ring_w(p, x[n, v:].reshape(o, v, v))).max()
                    for n in range(3))
        assert np.abs(smx - s64).max() <= 2e-2 * scale
        # the 1p part only sees BF16 through the second-order coupling contractions
        assert np.abs(smx[:, :v] - s64[:, :v]).max() <= 1e-4 * np.abs(s64[:, :v]).max()
        # split-BF16: each operand carries ~16 significant bits (representation
        # error <= 2^-17 relative), the dropped lo*lo product is ~2^-18, and the
        # re-split stage-1 intermediate adds the same again: 2e-4 of the scale
        sx3 = E.eaadc_sigma_host(ctx, 0, x, E.EAADC_MIXED_BF16X3)
        err3 = np.abs(sx3 - s64).max()
        print(f"mixed err {np.abs(smx - s64).max() / scale:.2e}  x3 err {err3 / scale:.2e}")
        assert err3 <= 2e-4 * scale
        # a BF16 sigma after an x3 one rebuilds nothing and stays as before
        assert np.array_equal(E.eaadc_sigma_host(ctx, 0, x, E.EAADC_MIXED_BF16), smx)
    finally:
        E.eaadc_destroy(ctx)


def test_mixed_davidson_tiny(E):
    pr = config_problem("tiny")
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    ref = np.linalg.eigvalsh(R.explicit_matrix(p, 3))[:4]
    ctx = _ctx(E, pr)
    try:
        om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-6, prec=E.EAADC_MIXED_BF16, refine=0)
        assert np.abs(om[0] - ref).max() <= 1e-5       # reduced-precision target
        om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-8, prec=E.EAADC_MIXED_BF16, refine=1)
        assert st == 0 and np.abs(om[0] - ref).max() <= 1e-8  # after FP64 refinement
        om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-6, prec=E.EAADC_MIXED_BF16X3, refine=0)
        assert np.abs(om[0] - ref).max() <= 1e-7       # split-BF16 target
        om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-8, prec=E.EAADC_MIXED_BF16X3, refine=1)
        assert st == 0 and np.abs(om[0] - ref).max() <= 1e-8
    finally:
        E.eaadc_destroy(ctx)


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLD, "canonical-200.npz")), reason="golden file missing")
@pytest.mark.parametrize("prec", ["EAADC_MIXED_BF16", "EAADC_MIXED_BF16X3"])
def test_canonical_200_mixed_refined_against_oracle(E, prec):
    g = np.load(os.path.join(GOLD, "canonical-200.npz"))
    pr = config_problem("canonical-200")
    ctx = _ctx(E, pr)
    try:
        om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-7, prec=getattr(E, prec), refine=1, max_sub=40, maxit=300)
        print(f"{prec}: iters {it[0]} resnorm {rn[0].max():.1e}")
        assert st == 0
        assert np.abs(om[0] - g["omega3"]).max() <= 1e-8
    finally:
        E.eaadc_destroy(ctx)


@pytest.mark.parametrize("o,v,naux,decay,seed", [(4, 13, 40, 8.0, 9), (3, 136, 90, 20.0, 7)])
def test_tensor_core_build_of_m11(E, o, v, naux, decay, seed):
    """M^(3) with its amplitude ladder on the tensor cores (split BF16) against
    the FP64 build: the ladder term carries ~1e-5 relative error, held to
    1e-4 of max |M_ab| and 1e-6 Eh in the roots."""
    pr = make_problem(o, v, naux, decay, seed)
    ctx = E.eaadc_init(o, v, naux, pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    try:
        E.eaadc_build_canonical(ctx, 3, 1.0)
        m64 = E.eaadc_get_m11(ctx, 0)
        w64 = E.eaadc_davidson(ctx, 3, tol=1e-8)[0][0]
        E.eaadc_set_build_precision(ctx, E.EAADC_MIXED_BF16X3)
        E.eaadc_build_canonical(ctx, 3, 1.0)
        mx = E.eaadc_get_m11(ctx, 0)
        wx = E.eaadc_davidson(ctx, 3, tol=1e-8)[0][0]
        print(f"tensor-core build: M11 rel err {np.abs(mx - m64).max() / np.abs(m64).max():.1e}, "
              f"roots {np.abs(wx - w64).max():.1e} Eh")
        assert np.abs(mx - m64).max() <= 1e-4 * np.abs(m64).max()
        assert np.abs(wx - w64).max() <= 1e-6
    finally:
        E.eaadc_destroy(ctx)


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLD, "canonical-200.npz")), reason="golden file missing")
def test_canonical_200_tensor_core_build_against_oracle(E):
    """Whole reduced-precision pipeline: split-BF16 amplitude ladder in the
    build, BF16 Davidson, FP64 Ritz step: roots within 1e-5 Eh of the oracle."""
    g = np.load(os.path.join(GOLD, "canonical-200.npz"))
    pr = config_problem("canonical-200")
    ctx = E.eaadc_init(pr["o"], pr["v"], pr["naux"], pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    try:
        E.eaadc_set_build_precision(ctx, E.EAADC_MIXED_BF16X3)
        E.eaadc_build_canonical(ctx, 3, 1.0)
        m11 = E.eaadc_get_m11(ctx, 0)
        assert np.abs(m11 - g["m11_3"]).max() <= 1e-4 * np.abs(g["m11_3"]).max()
        om, rn, it, st = E.eaadc_davidson(ctx, 4, tol=1e-5, prec=E.EAADC_MIXED_BF16, refine=2, max_sub=40, maxit=300)
        print(f"tensor-core build, BF16 Davidson + FP64 Ritz: max err {np.abs(om[0] - g['omega3']).max():.1e} Eh")
        assert np.abs(om[0] - g["omega3"]).max() <= 1e-5
    finally:
        E.eaadc_destroy(ctx)
