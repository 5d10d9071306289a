"""Pins of the CPU oracle against things other than itself (CPU only).

P1  brute-force ISR (exact FCI, Sec. II.A Eq. 1-6) Taylor coefficients (Eq. 5)
    equal the analytic spin-orbital EA-ADC(3) blocks, every block and order;
P2  first-order blocks equal Slater-Condon CI elements of the determinants;
P3  the restricted doublet matrix equals the spin-orbital matrix projected
    onto the doublet (Ms = +1/2) space, and that space is invariant;
P4  Hermiticity of the explicit matrix;
P5  dense diagonalisation equals the Davidson roots;
P6  zero FNO/NAF thresholds reproduce canonical roots; orbital/auxiliary
    rotations leave the roots unchanged; Eq. 30 reduces to omega^(3);
P7  without two-electron integrals the roots are the virtual energies;
P8  the DF two-step ladder equals the explicit four-index contraction;
P9  the state density equals the spin-summed density of the determinant
    expansion; the MP2 density equals the second-order Taylor coefficient of
    the exact ground-state density.
"""
import itertools

import numpy as np
import pytest

from synth import config_problem, make_problem
from oracle import fci_isr, spinorb, restricted as R, fno
from oracle.davidson import davidson


def _tiny(o, v, naux=10, decay=4.0, seed=3, tmax=0.05):
    return make_problem(o, v, naux, decay, seed, tmax=tmax)


def _eps(pr):
    return np.concatenate([pr["eps_occ"], pr["eps_vir"]])


# ----------------------------------------------------------------------- P1
@pytest.mark.parametrize("o,v,seed,tmax", [(1, 2, 7, 0.05), (2, 3, 7, 0.05), (2, 3, 11, 0.1)])
def test_p1_bruteforce_isr_taylor(o, v, seed, tmax):
    pr = _tiny(o, v, 12, 4.0, seed, tmax)
    sysm = fci_isr.ISRSystem(o, _eps(pr), pr["B"])
    coef = sysm.taylor(3, r=0.25, npts=24)
    assert max(np.abs(c.imag).max() for c in coef) < 1e-10
    c = [x.real for x in coef]
    b = spinorb.blocks(sysm.eps_so, sysm.g, 2 * o, 3)
    n1 = 2 * v
    pairs = [
        (c[0][:n1, :n1], b["11_0"]), (c[1][:n1, :n1], 0 * b["11_0"]),
        (c[2][:n1, :n1], b["11_2"]), (c[3][:n1, :n1], b["11_3"]),
        (c[0][:n1, n1:], 0 * b["12_1"]), (c[1][:n1, n1:], b["12_1"]), (c[2][:n1, n1:], b["12_2"]),
        (c[0][n1:, n1:], b["22_0"]), (c[1][n1:, n1:], b["22_1"]),
    ]
    for ref, got in pairs:
        scale = max(np.abs(ref).max(), 1e-3)
        assert np.abs(ref - got).max() <= 1e-9 * scale
    # the third-order 1p block is really exercised
    assert np.abs(b["11_3"]).max() > 1e-4


# ----------------------------------------------------------------------- P2
def test_p2_ci_identity():
    o, v = 2, 3
    pr = _tiny(o, v, 12, 4.0, 5)
    sysm = fci_isr.ISRSystem(o, _eps(pr), pr["B"])
    HN1 = sysm.H0N1 + sysm.VN1
    HN = sysm.H0N + sysm.VN
    Ehf = HN[sysm.phi0, sysm.phi0]
    phi0 = np.zeros(len(sysm.detN))
    phi0[sysm.phi0] = 1.0
    X1 = np.stack([P @ phi0 for P in sysm.P1], 1)
    X2 = np.stack([P @ phi0 for P in sysm.P2], 1)
    X = np.concatenate([X1, X2], 1)
    Mci = X.T @ HN1 @ X - Ehf * np.eye(X.shape[1])
    b = spinorb.blocks(sysm.eps_so, sysm.g, 2 * o, 3)
    n1 = 2 * v
    assert np.abs(Mci[:n1, :n1] - b["11_0"]).max() < 1e-12
    assert np.abs(Mci[:n1, n1:] - b["12_1"]).max() < 1e-12
    assert np.abs(Mci[n1:, n1:] - b["22_0"] - b["22_1"]).max() < 1e-12


# ----------------------------------------------------------------------- P3
def doublet_embedding(o, v, basis):
    """Isometry from the restricted [1p, 2p1h] space into the spin-orbital basis."""
    idx = {x: i for i, x in enumerate(basis)}
    n1 = 2 * v
    nr = v + o * v * v
    E = np.zeros((n1 + len(basis), nr))
    for a in range(v):
        E[2 * a, a] = 1.0
    for col in range(o * v * v):
        w = np.zeros(o * v * v)
        w[col] = 1.0
        A = R.Sinv_map(w.reshape(o, v, v))
        for k, b_, c_ in itertools.product(range(o), range(v), range(v)):
            val = A[k, b_, c_]
            if val == 0.0:
                continue
            Ka, Kb, Ba, Cb = 2 * k, 2 * k + 1, 2 * b_, 2 * c_ + 1
            if Ba < Cb:
                E[n1 + idx[(Kb, Ba, Cb)], v + col] += val
            else:
                E[n1 + idx[(Kb, Cb, Ba)], v + col] -= val
            if b_ < c_:
                E[n1 + idx[(Ka, 2 * b_, 2 * c_)], v + col] += A[k, b_, c_] - A[k, c_, b_]
    return E


@pytest.mark.parametrize("o,v,seed", [(1, 2, 3), (2, 3, 3), (3, 2, 9)])
@pytest.mark.parametrize("order", [2, 3])
def test_p3_restricted_equals_projected_spinorbital(o, v, seed, order):
    pr = _tiny(o, v, 10, 4.0, seed)
    eso, g = fci_isr.spinorb_integrals(_eps(pr), pr["B"])
    Mso = spinorb.matrix(eso, g, 2 * o, order)
    basis = spinorb.blocks(eso, g, 2 * o, 1)["basis"]
    E = doublet_embedding(o, v, basis)
    assert np.abs(E.T @ E - np.eye(E.shape[1])).max() < 1e-14
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    Mr = R.explicit_matrix(p, order)
    assert np.abs(Mr - E.T @ Mso @ E).max() < 1e-12 * np.abs(Mr).max()
    assert np.abs(Mso @ E - E @ Mr).max() < 1e-12 * np.abs(Mr).max()
    # the restricted roots are the doublet subset of the spin-orbital roots
    wso = np.linalg.eigvalsh(Mso)
    for w in np.linalg.eigvalsh(Mr):
        assert np.min(np.abs(wso - w)) < 1e-10


# ----------------------------------------------------------------------- P4/P5
@pytest.fixture(scope="module")
def tiny_cfg():
    pr = config_problem("tiny")
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    return pr, p, R.explicit_matrix(p, 3)


def test_p4_hermitian(tiny_cfg):
    _, p, M = tiny_cfg
    assert M.shape == (2020, 2020)
    assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()
    M2 = R.explicit_matrix(p, 2)
    assert np.abs(M2 - M2.T).max() <= 1e-13 * np.abs(M2).max()


def test_p5_dense_equals_davidson(tiny_cfg):
    _, p, M = tiny_cfg
    w = np.linalg.eigvalsh(M)
    sig = R.Sigma(p, 3)
    x = np.random.default_rng(1).standard_normal(M.shape[0])
    assert np.abs(sig(x) - M @ x).max() < 1e-12 * np.abs(M @ x).max()
    th, X, rn, it = davidson(sig, sig.diagonal(), 4, tol=1e-9)
    assert np.all(rn <= 1e-9)
    assert np.abs(th - w[:4]).max() <= 1e-10


# ----------------------------------------------------------------------- P6
def test_p6_zero_thresholds_and_eq30(tiny_cfg):
    _, p, M = tiny_cfg
    w3 = np.linalg.eigvalsh(M)
    r = fno.ss_fno_ea(p, 2, 3, -1.0, -1.0)
    assert np.all(r["vprime"] == p.v) and np.all(r["nauxprime"] == p.naux)
    for k in range(2):
        assert np.min(np.abs(w3 - r["omega3"][k])) < 1e-10
        assert np.abs(r["omega_corr"][k] - r["omega3"][k]) < 1e-10
        assert np.abs(r["omega2_fno"][k] - r["omega2_can"][k]) < 1e-10


def test_p6_rotation_invariance():
    pr = _tiny(2, 4, 12, 5.0, 21)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    w = np.linalg.eigvalsh(R.explicit_matrix(p, 3))[:6]
    rng = np.random.default_rng(5)
    # random orthogonal virtual rotation, then semicanonicalisation (Eq. 12-14)
    Qv, _ = np.linalg.qr(rng.standard_normal((p.v, p.v)))
    Bfno, efno, _ = fno.fno_basis(Qv @ np.diag(np.arange(p.v, 0, -1.0)) @ Qv.T, p.ev, -1.0)
    pt, _ = fno.truncated_problem(p, Bfno, efno, -1.0)
    assert np.abs(np.linalg.eigvalsh(R.explicit_matrix(pt, 3))[:6] - w).max() < 1e-11
    # random orthogonal auxiliary rotation
    Qa, _ = np.linalg.qr(rng.standard_normal((p.naux, p.naux)))
    p2 = R.Problem(pr["eps_occ"], pr["eps_vir"], np.einsum("QP,Qpq->Ppq", Qa, pr["B"]))
    assert np.abs(np.linalg.eigvalsh(R.explicit_matrix(p2, 3))[:6] - w).max() < 1e-12


# ----------------------------------------------------------------------- P7
def test_p7_no_interaction_limit():
    pr = _tiny(2, 3, 8, 4.0, 2)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], 0.0 * pr["B"])
    w = np.linalg.eigvalsh(R.explicit_matrix(p, 3))
    ref = np.sort(np.concatenate([pr["eps_vir"], R.diag_2p1h(p).reshape(-1)]))
    assert np.abs(w - ref).max() < 1e-13


def test_p7_second_order_self_energy_limit():
    """For weak interaction the lowest root is e_a + M2_aa + sum_J C1_aJ^2/(e_a - D_J) + O(s^6)."""
    pr = _tiny(2, 3, 8, 4.0, 4)
    errs = []
    for s in (0.2, 0.1):
        p = R.Problem(pr["eps_occ"], pr["eps_vir"], s * pr["B"])
        w = np.linalg.eigvalsh(R.explicit_matrix(p, 3))[0]
        ea = pr["eps_vir"][0]
        C = R.coupling_w(p, 2).reshape(-1, p.v)[:, 0]
        D = R.diag_2p1h(p).reshape(-1)
        pred = ea + R.m11_second(p)[0, 0] + np.sum(C * C / (ea - D))
        errs.append(abs(w - pred) / s ** 4)
    # error / s^4 shrinks like s^2
    assert errs[1] < 0.3 * errs[0]


# ----------------------------------------------------------------------- P8
def test_p8_df_ladder_equals_four_index():
    pr = _tiny(2, 6, 14, 5.0, 8)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    W = np.random.default_rng(2).standard_normal((p.o, p.v, p.v))
    ref = np.einsum("bdce,kde->kbc", p.vvvv(), W)
    got = R.ladder_w(p, W)
    assert np.abs(ref - got).max() <= 1e-12 * np.abs(ref).max()


# ----------------------------------------------------------------------- P9
def test_p9_state_density_from_determinants():
    o, v = 2, 3
    pr = _tiny(o, v, 10, 4.0, 6)
    eso, g = fci_isr.spinorb_integrals(_eps(pr), pr["B"])
    basis = spinorb.blocks(eso, g, 2 * o, 1)["basis"]
    E = doublet_embedding(o, v, basis)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(v + o * v * v)
    x /= np.linalg.norm(x)
    y, W = x[:v], x[v:].reshape(o, v, v)
    D = fno.ea_density(y, W)
    assert abs(np.trace(D) - (y @ y + 2 * np.sum(W * W))) < 1e-13
    # determinant expansion of the same state and its spin-summed vv density
    sysm = fci_isr.ISRSystem(o, _eps(pr), pr["B"])
    phi0 = np.zeros(len(sysm.detN))
    phi0[sysm.phi0] = 1.0
    X = np.concatenate([np.stack([P @ phi0 for P in sysm.P1], 1),
                        np.stack([P @ phi0 for P in sysm.P2], 1)], 1)
    psi = X @ (E @ x)
    ref = np.zeros((v, v))
    for a in range(v):
        for b in range(v):
            for s in range(2):
                A, B = sysm.vir[2 * a + s], sysm.vir[2 * b + s]
                op = fci_isr.operator_matrix([(A, 1), (B, 0)], sysm.detN1, sysm.detN1)
                ref[a, b] += psi @ op @ psi
    assert np.abs(ref - D).max() < 1e-13


def test_p9_mp2_density_is_second_order_exact_density():
    o, v = 2, 3
    pr = _tiny(o, v, 10, 4.0, 12)
    sysm = fci_isr.ISRSystem(o, _eps(pr), pr["B"])
    ops = {}
    for a in range(v):
        for b in range(v):
            for s in range(2):
                A, B = sysm.vir[2 * a + s], sysm.vir[2 * b + s]
                ops[(a, b, s)] = fci_isr.operator_matrix([(A, 1), (B, 0)], sysm.detN, sysm.detN)
    r, npts = 0.25, 16
    acc = np.zeros((v, v), dtype=complex)
    for m in range(npts):
        lam = r * np.exp(2j * np.pi * m / npts)
        _, psi = sysm.ground_state(lam)
        dens = np.zeros((v, v), dtype=complex)
        for (a, b, s), op in ops.items():
            dens[a, b] += psi @ op @ psi
        acc += dens * np.exp(-2j * np.pi * 2 * m / npts)
    D2 = (acc / (npts * r ** 2)).real
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    Dmp2 = fno.mp2_density(p)
    assert np.abs(Dmp2).max() > 1e-5
    assert np.abs(D2 - Dmp2).max() < 1e-10 * max(1.0, np.abs(Dmp2).max())


# ---------------------------------------------------------------------- R13
def test_r13_sm_scale_multiplies_third_order_block_only():
    """sm-ADC reading: x scales M^(3)_ab only. With x = 0 the 1p/1p block is
    the second-order one, the second-order coupling and the first-order
    2p1h block stay; x is linear in the 1p/1p block."""
    pr = _tiny(2, 3, 8, 4.0, 6)
    p = R.Problem(pr["eps_occ"], pr["eps_vir"], pr["B"])
    v = p.v
    M3 = R.explicit_matrix(p, 3, 1.0)
    M0 = R.explicit_matrix(p, 3, 0.0)
    Mh = R.explicit_matrix(p, 3, 0.5)
    M2 = R.explicit_matrix(p, 2)
    assert np.abs(M0[:v, :v] - M2[:v, :v]).max() < 1e-14
    assert np.abs(M0[v:, :] - M3[v:, :]).max() < 1e-14          # coupling and 2p1h block unchanged
    assert np.abs(M0[v:, :v] - M2[v:, :v]).max() > 1e-6          # C^(2) kept, not ADC(2)
    assert np.abs(Mh[:v, :v] - 0.5 * (M0[:v, :v] + M3[:v, :v])).max() < 1e-14
