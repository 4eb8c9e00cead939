"""Two-flavour pseudofermion action of the ODWF operator, its force, the Wilson gauge action and
force, and a molecular-dynamics step (Sec. 2: the HMC's two-flavour parts with mass
preconditioning, the Wilson plaquette gauge action at beta = 6.20, the Omelyan integrator).

TEST INFRASTRUCTURE ONLY (see the package docstring).  numpy and the C oracle in fp64.

Reading (the paper cites the action's formula, Eq. 14 of its reference, which is not available):
det D(m) = det(M(m))^2 det S(m) for the even-odd split, and M (site-local, no links) does not
depend on the gauge field, so the two-flavour factor det[D(m1)^+ D(m1)] / det[D(m2)^+ D(m2)] is,
up to a constant, det[S1^+ S1] / det[S2^+ S2] with S_i = S(m_i) the Schur operator on even sites.
It is represented by the pseudofermion action on even-site fields

    S_pf = phi^+ S2^+ (S1^+ S1)^-1 S2 phi = | S1 X |^2,   X = (S1^+ S1)^-1 S2 phi.

m2 = m_PV = 2 m0 gives the plain two-flavour term; mass preconditioning (Hasenbusch) is the
product of such ratios over a chain m_q -> m_H1 -> m_H2 -> m_PV.

Force.  For a link U_mu(x) -> exp(eps T) U_mu(x), T traceless anti-Hermitian, every function
here returns Pi_mu(x), traceless anti-Hermitian, with dS/deps = tr(T Pi).  With
H = -1/2 W B (the hopping term of D = D_w B + 1 - L, D_w = 4 - m0 - W/2):

    dS = 2 Re<X, dS2 phi> - 2 Re<Y, dS1 X>,   Y = S1 X,
    <A, dS psi> = 1/2 <L1, dW (B R1)> + 1/2 <L2, dW (B psi)>,
        L1 = M^-+ A,  R1 = M^-1 H_oe psi,  L2 = M^-+ H_eo^+ M^-+ A,

and for full-lattice fields Lf, Rf, d<Lf, W Rf>/deps = tr(T G) per link with
    G_mu(x) = U_mu(x) K1 - K2 U_mu(x)^+,
    K1 = sum_{s,spin} Rf_s(x+mu) conj((1 - gamma_mu) Lf_s(x)),
    K2 = sum_{s,spin} Rf_s(x) conj((1 + gamma_mu) Lf_s(x+mu))
(colour outer products, first index from Rf), times -1 on t-links across the antiperiodic
boundary.  Pi = ta(G_total) since tr(T ta(G)) = Re tr(T G) for traceless anti-Hermitian T.

Molecular dynamics: momenta P_mu(x) traceless anti-Hermitian, kinetic energy
K = -sum tr(P^2), H = K + S; Hamilton's equations dU/dt = P U, dP/dt = Pi / 2.  Multiple time
scales (Sexton-Weingarten, Sec. 2): the outer integrator kicks with the pseudofermion forces and
each of its drifts is n_inner steps of the same integrator under the gauge force alone.
Parity status: pinned by tests/test_oracle_hmc.py (central finite differences of both actions
along all eight generators, the heat-bath identity S(phi(eta)) = |eta|^2, reversibility and
second-order energy conservation of the integrators, and the two limits in which the nested
integrator is a single-scale one: no pseudofermion term, and beta = 0).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

from . import M, MDAG, MINV, MINVDAG, b5, cg, from_parity, gammas, hop_w, m5, schur, to_parity
from . import flow as fl

EYE4 = np.eye(4, dtype=np.int64)
OMELYAN_LAMBDA = 0.1931833275037836


def _dims(U):
    lt, lz, ly, lx = U.shape[1:5]
    return (lx, ly, lz, lt)


def ta(X):
    A = 0.5 * (X - np.conj(np.swapaxes(X, -1, -2)))
    tr = np.trace(A, axis1=-2, axis2=-1)
    return A - (tr / 3.0)[..., None, None] * np.eye(3)


# ------------------------------------------------------------------ pseudofermion action
def solve_normal(U, b, m0, m, omega, tbc=True, tol=1e-13):
    """(S^+ S)^-1 b for even-site b (the oracle's FP64 CG)."""
    x, it, _ = cg(U, b, m0, m, omega, tbc, tol=tol, max_iter=200000)
    assert it >= 0, "oracle CG did not converge"
    return x


def pf_action(U, phi, m0, m1, m2, omega, tbc=True):
    """phi^+ S2^+ (S1^+ S1)^-1 S2 phi (real)."""
    psi = schur(U, phi, m0, m2, omega, tbc)
    X = solve_normal(U, psi, m0, m1, omega, tbc)
    return float(np.vdot(psi, X).real)


def heatbath_phi(U, eta, m0, m1, m2, omega, tbc=True):
    """phi = S2^-1 S1^+ eta, so that S_pf(phi) = |eta|^2 (S2 phi = b solved as S2^+ S2 phi = S2^+ b)."""
    b = schur(U, eta, m0, m1, omega, tbc, dagger=True)
    return solve_normal(U, schur(U, b, m0, m2, omega, tbc, dagger=True), m0, m2, omega, tbc)


def _hop_contract(U, Lf, Rf, tbc=True):
    """G_mu(x) with d<Lf, W(exp(eps T) U) Rf>/deps = sum_links tr(T G), for full 5D fields."""
    g = gammas()
    dims = _dims(U)
    lt = dims[3]
    ax = {0: 4, 1: 3, 2: 2, 3: 1}  # site axes of a (s, t, z, y, x, spin, col) field
    G = np.zeros(U.shape, dtype=np.complex128)
    one = np.eye(4)
    for mu in range(4):
        Rn = np.roll(Rf, -1, axis=ax[mu])  # R(x + mu)
        Ln = np.roll(Lf, -1, axis=ax[mu])  # L(x + mu)
        wm = np.einsum("ab,s...bc->s...ac", one - g[mu], Lf)  # (1 - gamma_mu) L(x)
        wp = np.einsum("ab,s...bc->s...ac", one + g[mu], Ln)  # (1 + gamma_mu) L(x + mu)
        K1 = np.einsum("s...ib,s...ia->...ba", Rn, np.conj(wm))
        K2 = np.einsum("s...ib,s...ia->...ba", Rf, np.conj(wp))
        Gm = U[mu] @ K1 - K2 @ np.conj(np.swapaxes(U[mu], -1, -2))
        if mu == 3 and tbc:
            Gm[lt - 1] *= -1.0
        G[mu] = Gm
    return G


def _dschur_contract(U, A, psi, m0, m, omega, tbc=True):
    """G with Re <A, dS(m) psi> = Re sum tr(T G): the two hop terms of dS = -M^-1 (dH_eo M^-1 H_oe
    + H_eo M^-1 dH_oe) on even fields A, psi, each contracting dW between B R and L."""
    dims = _dims(U)
    L1 = m5(A, m0, m, omega, MINVDAG)                                  # even
    R1 = m5(hop_w(U, b5(psi, m0, m, omega), 0, m0, tbc), m0, m, omega, MINV)  # odd: M^-1 H_oe psi
    L2 = m5(b5(hop_w(U, L1, 0, m0, tbc, dagger=True), m0, m, omega, dagger=True), m0, m, omega, MINVDAG)  # odd
    BR1 = b5(R1, m0, m, omega)
    Bpsi = b5(psi, m0, m, omega)
    G = _hop_contract(U, from_parity(L1, dims, 0), from_parity(BR1, dims, 1), tbc)
    G += _hop_contract(U, from_parity(L2, dims, 1), from_parity(Bpsi, dims, 0), tbc)
    return 0.5 * G


def pf_force(U, phi, m0, m1, m2, omega, tbc=True):
    """Pi_mu(x) (traceless anti-Hermitian, shape of U) with dS_pf/deps = tr(T Pi) for
    U_mu(x) -> exp(eps T) U_mu(x); also returns S_pf."""
    psi = schur(U, phi, m0, m2, omega, tbc)
    X = solve_normal(U, psi, m0, m1, omega, tbc)
    Y = schur(U, X, m0, m1, omega, tbc)
    G = 2.0 * _dschur_contract(U, X, phi, m0, m2, omega, tbc) - 2.0 * _dschur_contract(U, Y, X, m0, m1, omega, tbc)
    return ta(G), float(np.vdot(Y, Y).real)


# ------------------------------------------------------------------ gauge action
def gauge_action(U, beta):
    """Wilson plaquette action beta sum_p (1 - Re tr P / 3)."""
    return beta / 6.0 * fl.wilson_action(U)


def gauge_force(U, beta):
    """Pi with dS_g/deps = tr(T Pi): beta/3 times the flow force -ta(U S)."""
    Z = fl.force(U).reshape(U.shape)
    return beta / 3.0 * Z


# ------------------------------------------------------------------ molecular dynamics
def kinetic(P):
    return float(-np.einsum("...ab,...ba->...", P, P).real.sum())


def _force_total(U, terms, beta):
    Pi = gauge_force(U, beta) if beta else np.zeros(U.shape, dtype=np.complex128)
    for phi, m0, m1, m2, omega in terms:
        Pi = Pi + pf_force(U, phi, m0, m1, m2, omega)[0]
    return Pi


def hamiltonian(U, P, terms, beta):
    Hh = kinetic(P) + (gauge_action(U, beta) if beta else 0.0)
    for phi, m0, m1, m2, omega in terms:
        Hh += pf_action(U, phi, m0, m1, m2, omega)
    return Hh


def md_leapfrog(U, P, eps, nsteps, terms, beta):
    """P(eps/2) U(eps) P(eps/2) steps of dU/dt = P U, dP/dt = Pi/2."""
    U = U.copy()
    P = P.copy()
    for _ in range(nsteps):
        P = P + 0.25 * eps * _force_total(U, terms, beta)
        U = expm(eps * P) @ U
        P = P + 0.25 * eps * _force_total(U, terms, beta)
    return U, P


def md_omelyan(U, P, eps, nsteps, terms, beta, lam=OMELYAN_LAMBDA):
    """Second-order minimum-norm (Omelyan) steps: P(lam eps) U(eps/2) P((1-2lam) eps) U(eps/2) P(lam eps)."""
    U = U.copy()
    P = P.copy()
    for _ in range(nsteps):
        P = P + 0.5 * lam * eps * _force_total(U, terms, beta)
        U = expm(0.5 * eps * P) @ U
        P = P + 0.5 * (1.0 - 2.0 * lam) * eps * _force_total(U, terms, beta)
        U = expm(0.5 * eps * P) @ U
        P = P + 0.5 * lam * eps * _force_total(U, terms, beta)
    return U, P


def _inner(U, P, h, n_inner, beta, integrator, lam):
    """n_inner steps of the integrator over time h under the gauge force alone."""
    d = h / n_inner
    for _ in range(n_inner):
        if integrator == "omelyan":
            P = P + 0.5 * lam * d * gauge_force(U, beta)
            U = expm(0.5 * d * P) @ U
            P = P + 0.5 * (1.0 - 2.0 * lam) * d * gauge_force(U, beta)
            U = expm(0.5 * d * P) @ U
            P = P + 0.5 * lam * d * gauge_force(U, beta)
        else:
            P = P + 0.25 * d * gauge_force(U, beta)
            U = expm(d * P) @ U
            P = P + 0.25 * d * gauge_force(U, beta)
    return U, P


def md_nested(U, P, eps, nsteps, terms, beta, n_inner, integrator="omelyan", lam=OMELYAN_LAMBDA):
    """Sexton-Weingarten multiple time scales: outer steps of size eps kick with the pseudofermion
    forces only; every drift of the outer step (eps/2 twice for Omelyan, eps once for leapfrog)
    is _inner over that time with the gauge force."""
    U = U.copy()
    P = P.copy()

    def ff(U):
        return _force_total(U, terms, 0.0)

    for _ in range(nsteps):
        if integrator == "omelyan":
            P = P + 0.5 * lam * eps * ff(U)
            U, P = _inner(U, P, 0.5 * eps, n_inner, beta, integrator, lam)
            P = P + 0.5 * (1.0 - 2.0 * lam) * eps * ff(U)
            U, P = _inner(U, P, 0.5 * eps, n_inner, beta, integrator, lam)
            P = P + 0.5 * lam * eps * ff(U)
        else:
            P = P + 0.25 * eps * ff(U)
            U, P = _inner(U, P, eps, n_inner, beta, integrator, lam)
            P = P + 0.25 * eps * ff(U)
    return U, P
