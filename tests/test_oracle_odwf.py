"""Pins of the oracle's 5D ODWF operator, its site-local part M, the even-odd Schur
operator and the normal-equation CG, against facts fixed outside the oracle:

* Sec. 2: with c = 1, d = 0 the 4D effective operator (P^-1 D(m_PV)^-1 D(m_q) P)_11 with
  m_PV = 2 m0 equals (1 + r)/2 + (1 - r)/2 gamma_5 S(H_w), r = m_q/(2 m0), with S the shifted
  Zolotarev approximation built from R_Z's coefficients (not from the weights);
* Eq. (1)-(2): det D(m_q)/det D(m_PV) = det D_eff;
* dense adjoints, dense Schur complements, dense LU solves and positivity of D^dag D.
"""
import numpy as np
import pytest

import odwf_synth as syn
import oracle
from oracle import dense, zolotarev

M0 = 1.3


@pytest.fixture(scope="module")
def small():
    dims = (2, 2, 2, 2)
    U = syn.gauge_field(dims, 0.5, 1)
    return dims, U


@pytest.mark.parametrize("shifted", [True, False])
@pytest.mark.parametrize("mq", [0.01, 0.3])
def test_effective_operator_is_zolotarev_overlap(oracle_lib, small, shifted, mq):
    dims, U = small
    ns = 4
    w, _ = zolotarev.omega(ns, 0.05, 6.0, shifted)
    deff5, D, Dpv = dense.effective_from_5d(U, ns, M0, mq, w)
    dz, lam = dense.effective_zolotarev(U, ns, M0, mq, 0.05, 6.0, shifted)
    assert np.abs(deff5 - dz).max() < 1e-11
    # Eq. (1)-(2): the determinant ratio against the Pauli-Villars operator m_PV = 2 m0
    s1, l1 = np.linalg.slogdet(D)
    s2, l2 = np.linalg.slogdet(Dpv)
    s3, l3 = np.linalg.slogdet(dz)
    assert abs((l1 - l2) - l3) < 1e-9
    assert abs(s1 / s2 - s3) < 1e-9


def test_effective_operator_wrong_mass_fails(oracle_lib, small):
    """A Pauli-Villars mass other than 2 m0 (or r other than m_q/(2 m0)) breaks the identity."""
    dims, U = small
    ns = 4
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    mq = 0.2
    deff5, _, _ = dense.effective_from_5d(U, ns, M0, mq, w)
    wrong, _ = dense.effective_zolotarev(U, ns, M0, 2 * mq, 0.05, 6.0, True)
    assert np.abs(deff5 - wrong).max() > 1e-2


@pytest.mark.parametrize("ns", [2, 4])
def test_d5_dagger_is_adjoint_dense(oracle_lib, small, ns):
    dims, U = small
    w = np.linspace(0.3, 1.7, ns)  # generic, non-symmetric weights
    D = dense.dense_d5(U, ns, M0, 0.07, w)
    Dd = dense.dense_d5(U, ns, M0, 0.07, w, dagger=True)
    assert np.abs(Dd - D.conj().T).max() < 1e-14
    # rho != sigma (c = 1, d != 0) stays adjoint too
    rho, sig = w + 0.1, w - 0.1
    n = D.shape[0]
    e = np.eye(n, dtype=np.complex128)
    A = np.stack([oracle.d5(U, e[j].reshape(ns, 2, 2, 2, 2, 4, 3), M0, 0.07, rho=rho, sigma=sig).reshape(-1)
                  for j in range(n)], axis=1)
    Ad = np.stack([oracle.d5(U, e[j].reshape(ns, 2, 2, 2, 2, 4, 3), M0, 0.07, dagger=True, rho=rho,
                             sigma=sig).reshape(-1) for j in range(n)], axis=1)
    assert np.abs(Ad - A.conj().T).max() < 1e-14


def test_adjoint_identity_large(oracle_lib):
    dims = (4, 4, 4, 4)
    ns = 8
    U = syn.gauge_field(dims, 0.3, 2)
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    psi = syn.gaussian_spinor(ns, dims, 3)
    phi = syn.gaussian_spinor(ns, dims, 4)
    lhs = np.vdot(phi, oracle.d5(U, psi, M0, 0.01, w))
    rhs = np.vdot(oracle.d5(U, phi, M0, 0.01, w, dagger=True), psi)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_m5_is_site_local_part_of_d5(oracle_lib):
    """M applied directly equals D with all links set to zero; M M^-1 = 1 and M^dag M^-dag = 1."""
    dims = (2, 2, 2, 4)
    ns = 8
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    lx, ly, lz, lt = dims
    U0 = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    psi = syn.gaussian_spinor(ns, dims, 5)
    m = oracle.m5(psi, M0, 0.04, w, oracle.M)
    assert np.abs(m - oracle.d5(U0, psi, M0, 0.04, w)).max() < 1e-13
    md = oracle.m5(psi, M0, 0.04, w, oracle.MDAG)
    assert np.abs(md - oracle.d5(U0, psi, M0, 0.04, w, dagger=True)).max() < 1e-13
    assert np.abs(oracle.m5(oracle.m5(psi, M0, 0.04, w, oracle.MINV), M0, 0.04, w, oracle.M) - psi).max() < 1e-12
    assert np.abs(oracle.m5(oracle.m5(psi, M0, 0.04, w, oracle.MINVDAG), M0, 0.04, w, oracle.MDAG) - psi).max() < 1e-12


def test_schur_is_dense_schur_complement(oracle_lib, small):
    dims, U = small
    ns = 4
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    mq = 0.05
    D = dense.dense_d5(U, ns, M0, mq, w)
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    ev = syn.even_sites(dims)
    od = np.setdiff1d(np.arange(V), ev)

    def idx(sites):
        return np.array([((s * V + x) * 12 + k) for s in range(ns) for x in sites for k in range(12)])

    ie, io = idx(ev), idx(od)
    Dee, Deo, Doe, Doo = D[np.ix_(ie, ie)], D[np.ix_(ie, io)], D[np.ix_(io, ie)], D[np.ix_(io, io)]
    S_dense = np.eye(len(ie)) - np.linalg.solve(Dee, Deo @ np.linalg.solve(Doo, Doe))
    S = dense.dense_schur(U, ns, M0, mq, w)
    Sd = dense.dense_schur(U, ns, M0, mq, w, dagger=True)
    assert np.abs(S - S_dense).max() < 1e-12
    assert np.abs(Sd - S.conj().T).max() < 1e-12
    # det D = det(M_ee) det(M_oo) det(S)
    l_full = np.linalg.slogdet(D)[1]
    l_parts = np.linalg.slogdet(Dee)[1] + np.linalg.slogdet(Doo)[1] + np.linalg.slogdet(S)[1]
    assert abs(l_full - l_parts) < 1e-9


def test_cg_matches_dense_lu_and_is_hpd(oracle_lib, small):
    dims, U = small
    ns = 4
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    mq = 0.01
    S = dense.dense_schur(U, ns, M0, mq, w)
    A = S.conj().T @ S
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    assert ev.min() > 0
    b = syn.gaussian_spinor_even(ns, dims, 21)
    x_lu = np.linalg.solve(A, b.reshape(-1))
    x, it, res = oracle.cg(U, b, M0, mq, w, tol=1e-13)
    assert it > 0 and res <= 1e-12
    kappa = ev.max() / ev.min()
    assert np.linalg.norm(x.reshape(-1) - x_lu) <= 1e-12 * kappa * np.linalg.norm(x_lu) * 10
    # full-lattice normal equations D^dag D x = b
    D = dense.dense_d5(U, ns, M0, mq, w)
    bf = syn.gaussian_spinor(ns, dims, 22)
    xf_lu = np.linalg.solve(D.conj().T @ D, bf.reshape(-1))
    # the CG stops on its recursed residual; the recomputed one may sit a little above it
    xf, itf, resf = oracle.cg(U, bf, M0, mq, w, system=oracle.FULL_NORMAL, tol=1e-13)
    assert itf > 0 and resf <= 1e-12
    assert np.linalg.norm(xf.reshape(-1) - xf_lu) <= 1e-8 * np.linalg.norm(xf_lu)


def test_even_odd_full_solve_reconstruction(oracle_lib, small):
    """D x = eta through the Schur system: x_e from S x_e = M^-1(eta_e - H_eo M^-1 eta_o),
    x_o = M^-1 (eta_o - H_oe x_e); D x reproduces eta."""
    dims, U = small
    ns = 4
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    mq = 0.1
    eta = syn.gaussian_spinor(ns, dims, 30)
    D = dense.dense_d5(U, ns, M0, mq, w)
    x = np.linalg.solve(D, eta.reshape(-1)).reshape(eta.shape)
    ee = oracle.to_parity(eta, dims, 0)
    eo = oracle.to_parity(eta, dims, 1)
    minv_eo = oracle.m5(eo, M0, mq, w, oracle.MINV)
    heo = oracle.to_parity(oracle.d5(U, oracle.from_parity(minv_eo, dims, 1), M0, mq, w), dims, 0)
    rhs = oracle.m5(ee - heo, M0, mq, w, oracle.MINV)
    S = dense.dense_schur(U, ns, M0, mq, w)
    xe = np.linalg.solve(S, rhs.reshape(-1)).reshape(rhs.shape)
    hoe = oracle.to_parity(oracle.d5(U, oracle.from_parity(xe, dims, 0), M0, mq, w), dims, 1)
    xo = oracle.m5(eo - hoe, M0, mq, w, oracle.MINV)
    assert np.abs(xe - oracle.to_parity(x, dims, 0)).max() < 1e-11
    assert np.abs(xo - oracle.to_parity(x, dims, 1)).max() < 1e-11


def test_lanczos_extremes_match_dense_eigenvalues(oracle_lib, small):
    """The CG coefficients recorded by oracle.cg give, through the Lanczos tridiagonal matrix,
    the extreme eigenvalues of S^dag S: checked against a dense eigendecomposition on 2^4 x 4
    (with enough iterations the Ritz values converge to the ends of the spectrum)."""
    dims, U = small
    ns = 4
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    mq = 0.05
    S = dense.dense_schur(U, ns, M0, mq, w)
    A = S.conj().T @ S
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    b = syn.gaussian_spinor_even(ns, dims, 23)
    coefs = np.zeros(2 * 4000)
    x, it, res = oracle.cg(U, b, M0, mq, w, tol=1e-13, max_iter=4000, coefs=coefs)
    assert it > 0
    lmin, lmax = oracle.lanczos_extremes(coefs, it)
    assert abs(lmax - ev.max()) <= 1e-6 * ev.max()
    assert abs(lmin - ev.min()) <= 1e-3 * ev.min()
    # a truncated run sees the spectrum from inside
    lmin5, lmax5 = oracle.lanczos_extremes(coefs, 5)
    assert ev.min() * (1 - 1e-9) <= lmin5 and lmax5 <= ev.max() * (1 + 1e-9)


@pytest.mark.parametrize("ns", [4, 8])
def test_b5_is_the_chiral_shift_of_d5(oracle_lib, small, ns):
    """oracle.b5 against three independent routes (generic rho != sigma, both masses):
    (1) with U = 0 the Wilson operator is the constant 4 - m0, so D(m0 = 3) - D(m0 = 4) at the
        same r = m_q/(2 m0) is exactly B (D = D_w B + 1 - L);
    (2) B^dag is the adjoint of B: <phi, B psi> = <B^dag phi, psi>;
    (3) the site-local M = (4 - m0) B + 1 - L built densely by oracle.m5, with L = (B - rho)/sigma."""
    dims, _ = small
    rho = np.linspace(0.4, 1.9, ns)
    sig = np.linspace(1.2, 0.3, ns)
    U0 = np.zeros((4, 2, 2, 2, 2, 3, 3), dtype=np.complex128)
    psi = syn.gaussian_spinor(ns, dims, 40)
    phi = syn.gaussian_spinor(ns, dims, 41)
    for r in (0.02, 0.4):
        d3 = oracle.d5(U0, psi, 3.0, 2 * 3.0 * r, tbc=False, rho=rho, sigma=sig)
        d4 = oracle.d5(U0, psi, 4.0, 2 * 4.0 * r, tbc=False, rho=rho, sigma=sig)
        b = oracle.b5(psi, M0, 2 * M0 * r, rho=rho, sigma=sig)
        assert np.abs(b - (d3 - d4)).max() < 1e-13
        bd = oracle.b5(phi, M0, 2 * M0 * r, dagger=True, rho=rho, sigma=sig)
        lhs = np.vdot(phi.reshape(-1), b.reshape(-1))
        rhs = np.vdot(bd.reshape(-1), psi.reshape(-1))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
        m = oracle.m5(psi, M0, 2 * M0 * r, rho=rho, sigma=sig, op=oracle.M)
        lpsi = (b - rho[:, None, None, None, None, None, None] * psi) / sig[:, None, None, None, None, None, None]
        assert np.abs(m - ((4 - M0) * b + psi - lpsi)).max() < 1e-13


@pytest.mark.parametrize("tbc", [True, False])
def test_hop_w_composes_to_the_parity_blocks_of_d5(oracle_lib, tbc):
    """-1/2 W B is the parity-coupling part H of D (D = D_w B + 1 - L, D_w = 4 - m0 - W/2):
    hop_w(b5(psi_e)) is the odd part of D applied to the even-embedded psi, and
    b5^dag(hop_w^dag(phi_o)) the even part of D^dag applied to the odd-embedded phi."""
    dims, ns, mq = (4, 2, 2, 4), 4, 0.3
    U = syn.gauge_field(dims, 0.5, 3)
    w = np.linspace(0.3, 1.7, ns)
    pe = syn.gaussian_spinor_even(ns, dims, 42)
    po = syn.gaussian_spinor_even(ns, dims, 43)  # any half field, used as odd
    got = oracle.hop_w(U, oracle.b5(pe, M0, mq, w), 0, M0, tbc)
    ref = oracle.to_parity(oracle.d5(U, oracle.from_parity(pe, dims, 0), M0, mq, w, tbc), dims, 1)
    assert np.abs(got - ref).max() < 1e-13
    got = oracle.b5(oracle.hop_w(U, po, 1, M0, tbc, dagger=True), M0, mq, w, dagger=True)
    ref = oracle.to_parity(oracle.d5(U, oracle.from_parity(po, dims, 1), M0, mq, w, tbc, dagger=True), dims, 0)
    assert np.abs(got - ref).max() < 1e-13


def test_residual_mass_vanishes_for_exact_sign_and_shrinks_with_ns(oracle_lib, small):
    """The residual-mass reading of the effective operator: exactly zero (to rounding) when the
    sign function is exact (D_c then anticommutes with gamma_5), positive and O(d_Z) for the
    shifted Zolotarev approximation, and smaller at larger N_s (smaller d_Z)."""
    dims, U = small
    mq = 0.05
    ex = dense.effective_dense(U, 4, M0, mq, 0.05, 6.2, exact_sign=True)
    m_ex, num, den, _ = dense.residual_mass(ex, M0, mq, 3)
    assert abs(m_ex) < 1e-12 * abs(num / den)
    res = {}
    for ns in (4, 8):
        d = dense.effective_dense(U, ns, M0, mq, 0.05, 6.2)
        res[ns] = dense.residual_mass(d, M0, mq, 3)[0]
    assert abs(res[8]) < abs(res[4])
    _, dz4 = zolotarev.omega(4, 0.05, 6.2, True)
    assert 0 < abs(res[4]) < 10 * dz4


def test_effective_propagator_solves_the_effective_operator(oracle_lib, small):
    """D_eff^-1 b from the dense 4D operator equals the 5D route [P^-1 D(m_q)^-1 D(m_PV) P (b x e_1)]_1
    built from the dense 5D operators (the identity of Sec. 2 applied to a vector)."""
    dims, U = small
    ns, mq = 4, 0.1
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    Deff = dense.effective_dense(U, ns, M0, mq, 0.05, 6.0)
    b4 = syn.gaussian_spinor(1, dims, 77)[0]
    x = dense.effective_propagator(Deff, b4)
    D = dense.dense_d5(U, ns, M0, mq, w)
    Dpv = dense.dense_d5(U, ns, M0, 2 * M0, w)
    V = 16
    P = dense.chiral_perm(ns, V)
    v5 = np.zeros(12 * ns * V, dtype=np.complex128)
    v5[:12 * V] = b4.reshape(-1)
    y = np.linalg.solve(P, np.linalg.solve(D, Dpv @ (P @ v5)))[:12 * V]
    assert np.abs(y - x.reshape(-1)).max() < 1e-11 * np.abs(x).max()
