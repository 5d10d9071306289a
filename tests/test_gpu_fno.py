"""GPU parity of the per-state FNO/NAF build (Sec. II.C-E, Sec. III) and of
the Eq. 30 correction against the CPU oracle, and of the device eigensolver
those bases rest on against LAPACK (numpy.linalg.eigh).

Thresholds are placed in the middle (geometric) of a gap of the oracle's own
occupation / auxiliary-metric spectra, so that both sides keep the same
functions; the energies are then compared to 1e-8 Eh (FP64 on both sides,
Davidson converged to residual 1e-8)."""
import numpy as np
import pytest

from synth import make_problem
from oracle import fno as F
from oracle import restricted as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import __graft_entry__ as g

    g.build()
    import paper_2511_05897_gb300 as mod

    return mod


def _eigh_gpu(E, A):
    import torch

    n = A.shape[0]
    a = torch.tensor(A, device="cuda:0")
    w = torch.empty(n, dtype=torch.float64, device="cuda:0")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda:0")
    E.eaadc_eigh_sym(n, a.data_ptr(), w.data_ptr(), V.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return w.cpu().numpy(), V.cpu().numpy()


@pytest.mark.parametrize("n,kind", [(1, "rand"), (7, "rand"), (96, "rand"), (97, "rand"), (130, "degenerate"),
                                    (333, "rand"), (260, "lowrank")])
def test_eigh_sym_matches_lapack(E, n, kind):
    rng = np.random.default_rng(n)
    if kind == "rand":
        G = rng.standard_normal((n, n))
        A = G + G.T
    elif kind == "degenerate":  # eigenvalues in repeated pairs
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        A = (Q * np.repeat(np.arange(n // 2), 2)[:n]) @ Q.T
    else:  # J J^T of rank n/4, like the auxiliary metric: many zero eigenvalues
        J = rng.standard_normal((n, n // 4))
        A = J @ J.T
    w, V = _eigh_gpu(E, A)
    ref = np.linalg.eigvalsh(A)
    scale = np.abs(ref).max()
    assert np.abs(w - ref).max() <= 1e-12 * scale * max(1, np.sqrt(n) / 4)
    assert np.abs(A @ V - V * w).max() <= 1e-11 * scale
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-11


def _gap_threshold(values, keep):
    """A threshold between the keep-th and (keep+1)-th largest values (geometric
    mean, away from both), adjusted to the nearest gap of at least 2 %."""
    w = np.sort(values)[::-1]
    w = w[w > 1e-8 * w[0]]  # below that: the numerical null space (W = J J^T has rank <= v'^2)
    keep = min(keep, len(w) - 1)
    for j in list(range(keep, len(w))) + list(range(keep - 1, 0, -1)):
        hi, lo = w[j - 1], w[j]
        if hi > 1.02 * lo:
            return float(np.sqrt(hi * lo))
    raise AssertionError("no usable gap")


def _thresholds(p, nstates, frac_v, frac_aux):
    """Per-state FNO and NAF thresholds keeping about frac of the functions,
    from the oracle's spectra."""
    w2, X2 = F.solve(p, nstates, order=2, tol=1e-10)
    Dmp2 = F.mp2_density(p)
    fno, naf = [], []
    for k in range(nstates):
        y = X2[:p.v, k]
        W = X2[p.v:, k].reshape(p.o, p.v, p.v)
        nrm = np.sqrt(y @ y + np.sum(W * W))
        D = Dmp2 + F.ea_density(y / nrm, W / nrm)
        eta = np.linalg.eigvalsh(0.5 * (D + D.T))
        tf = _gap_threshold(eta, max(1, int(round(frac_v * p.v))))
        Bfno, efno, _ = F.fno_basis(D, p.ev, tf)
        Bvv = np.einsum("aA,Qab,bB->QAB", Bfno, p.Bvv, Bfno, optimize=True)
        _, lam = F.naf_basis(Bvv, -1.0)
        naf.append(_gap_threshold(lam, max(1, int(round(frac_aux * p.naux)))))
        fno.append(tf)
    return np.array(fno), np.array(naf)


CASES = [  # o, v, naux, decay, seed, nstates, nroots
    (2, 12, 100, 25.0, 3, 2, 3),     # auxiliary metric 100 x 100: block-Jacobi path
    (1, 100, 40, 10.0, 5, 2, 3),     # virtual density 100 x 100: block-Jacobi path
    (3, 20, 60, 15.0, 1, 3, 3),
]


@pytest.mark.parametrize("o,v,naux,decay,seed,nstates,nroots", CASES)
def test_fno_states_and_eq30_match_oracle(E, o, v, naux, decay, seed, nstates, nroots):
    pr = make_problem(o, v, naux, decay, seed)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    fno_t, naf_t = _thresholds(p, nstates, 0.6, 0.6)
    ref = F.ss_fno_ea(p, nstates, nroots, fno_t, naf_t, tol=1e-10)
    ctx = E.eaadc_init(o, v, naux, pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    try:
        E.eaadc_build_states(ctx, nstates, fno_t, naf_t, 3, 1.0)
        for k in range(nstates):
            vp, npx, dim = E.eaadc_state_info(ctx, k)
            assert (vp, npx) == (ref["vprime"][k], ref["nauxprime"][k])
            assert vp < v and npx < naux
        om, rn, it, st = E.eaadc_davidson(ctx, nroots, tol=1e-8)
        assert st == 0
        for k in range(nstates):
            assert np.abs(om[k] - ref["omega3_roots"][k][:nroots]).max() <= 1e-8
        got = E.eaadc_ea_energies(ctx)
        for key, rkey in (("omega_uncorr", "omega3"), ("omega_corr", "omega_corr"), ("omega2_can", "omega2_can"),
                          ("omega2_fno", "omega2_fno")):
            assert np.abs(got[key] - ref[rkey]).max() <= 1e-8, key
    finally:
        E.eaadc_destroy(ctx)


def test_zero_thresholds_reproduce_canonical(E):
    """Keeping every function: each state's target root is a canonical ADC(3)
    root and Eq. 30 adds nothing."""
    o, v, naux = 2, 9, 30
    pr = make_problem(o, v, naux, 6.0, 8)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    can3 = np.linalg.eigvalsh(R.explicit_matrix(p, 3))
    can2 = np.linalg.eigvalsh(R.explicit_matrix(p, 2))
    ctx = E.eaadc_init(o, v, naux, pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    try:
        E.eaadc_build_states(ctx, 3, -1.0, -1.0, 3, 1.0)
        for k in range(3):
            assert E.eaadc_state_info(ctx, k)[:2] == (v, naux)
        E.eaadc_davidson(ctx, 2, tol=1e-9)  # fewer roots than states: Eq. 30 still finds state 2's root
        got = E.eaadc_ea_energies(ctx)
        assert np.abs(got["omega2_can"] - can2[:3]).max() <= 1e-9
        assert np.abs(got["omega2_fno"] - got["omega2_can"]).max() <= 1e-9
        assert np.abs(got["omega_corr"] - got["omega_uncorr"]).max() <= 1e-9
        for w in got["omega_uncorr"]:
            assert np.abs(can3 - w).min() <= 1e-9
    finally:
        E.eaadc_destroy(ctx)


def test_build_states_rejects_bad_thresholds(E):
    pr = make_problem(1, 4, 6, 2.0, 4)
    ctx = E.eaadc_init(1, 4, 6, pr["eps_occ"], pr["eps_vir"], pr["B"], 0)
    try:
        with pytest.raises(E.EaadcError) as err:
            E.eaadc_build_states(ctx, 1, 1e6, -1.0, 3, 1.0)  # keeps no virtual
        assert err.value.status == E.EAADC_ERR_ARG
        with pytest.raises(E.EaadcError) as err:
            E.eaadc_build_states(ctx, 1, np.nan, -1.0, 3, 1.0)
        assert err.value.status == E.EAADC_ERR_NONFINITE
        with pytest.raises(E.EaadcError) as err:
            E.eaadc_ea_energies(ctx)  # no states yet
        assert err.value.status == E.EAADC_ERR_STATE
    finally:
        E.eaadc_destroy(ctx)
