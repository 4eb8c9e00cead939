"""Pins of the oracle's two-flavour pseudofermion action and force, the Wilson gauge force and
the molecular-dynamics integrators (oracle/hmc.py) against facts fixed outside those functions:

* the force is the derivative of the action: central finite differences of the action (each
  value a fresh FP64 CG solve to 1e-13) along all eight generators at several links, for the
  plain two-flavour term (m2 = m_PV = 2 m0) and a mass-preconditioning ratio, both time
  boundaries; the same for the Wilson gauge action at beta = 6.2;
* the heat-bath field phi = S2^-1 S1^+ eta has S_pf(phi) = |eta|^2;
* leapfrog and Omelyan steps are reversible, conserve H to second order in the step, and Omelyan
  violates it less than leapfrog at the same step;
* the nested (Sexton-Weingarten) integrator is a single-scale one in its two limits: without
  pseudofermion terms it is 2 n_inner (Omelyan) or n_inner (leapfrog) gauge steps per outer
  step, and at beta = 0 its inner drifts compose to the outer drift (exp(aP) exp(bP) =
  exp((a + b) P)); it is reversible and second order.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import odwf_synth as syn
from oracle import hmc, zolotarev

M0 = 1.3


def _case(dims, ns, seed=1, eps=0.5):
    U = syn.gauge_field(dims, eps, seed)
    w, _ = zolotarev.omega(ns, 0.05, 6.0, True)
    return U, w


@pytest.mark.parametrize("m1,m2,tbc", [(0.1, 2 * M0, True), (0.05, 0.5, False)])
def test_pf_force_is_the_derivative_of_the_action(oracle_lib, m1, m2, tbc):
    dims, ns = (2, 2, 2, 4), 4
    U, w = _case(dims, ns)
    phi = syn.gaussian_spinor_even(ns, dims, 3)
    Pi, S = hmc.pf_force(U, phi, M0, m1, m2, w, tbc)
    assert abs(S - hmc.pf_action(U, phi, M0, m1, m2, w, tbc)) < 1e-9 * abs(S)
    T = 1j * syn.gell_mann() / 2
    h = 1e-4
    rng = np.random.default_rng(4)
    worst, scale = 0.0, np.abs(Pi).max()
    for _ in range(4):
        mu = int(rng.integers(0, 4))
        site = tuple(int(rng.integers(0, L)) for L in dims)
        x, y, z, t = site
        for a in range(8):
            vals = []
            for sgn in (1, -1):
                Ud = U.copy()
                Ud[mu, t, z, y, x] = expm(sgn * h * T[a]) @ U[mu, t, z, y, x]
                vals.append(hmc.pf_action(Ud, phi, M0, m1, m2, w, tbc))
            fd = (vals[0] - vals[1]) / (2 * h)
            worst = max(worst, abs(fd - np.trace(T[a] @ Pi[mu, t, z, y, x]).real))
    assert worst < 1e-5 * scale, (worst, scale)
    assert scale > 1.0


def test_gauge_force_is_the_derivative_of_the_action():
    dims, beta = (2, 2, 2, 4), 6.2
    U, _ = _case(dims, 4, seed=5, eps=0.8)
    Pi = hmc.gauge_force(U, beta)
    T = 1j * syn.gell_mann() / 2
    h = 1e-5
    for mu, site in ((0, (1, 0, 1, 2)), (3, (0, 1, 0, 3))):
        x, y, z, t = site
        for a in range(8):
            Up, Um = U.copy(), U.copy()
            Up[mu, t, z, y, x] = expm(h * T[a]) @ U[mu, t, z, y, x]
            Um[mu, t, z, y, x] = expm(-h * T[a]) @ U[mu, t, z, y, x]
            fd = (hmc.gauge_action(Up, beta) - hmc.gauge_action(Um, beta)) / (2 * h)
            assert abs(fd - np.trace(T[a] @ Pi[mu, t, z, y, x]).real) < 1e-7


def test_heatbath_field_has_gaussian_action(oracle_lib):
    dims, ns = (2, 2, 2, 4), 4
    U, w = _case(dims, ns, seed=6)
    eta = syn.gaussian_spinor_even(ns, dims, 7)
    for m1, m2 in ((0.02, 0.3), (0.3, 2 * M0)):
        phi = hmc.heatbath_phi(U, eta, M0, m1, m2, w)
        S = hmc.pf_action(U, phi, M0, m1, m2, w)
        assert abs(S - np.vdot(eta, eta).real) < 1e-9 * S


def _terms(U, ns, w):
    dims = hmc._dims(U)
    return [(syn.gaussian_spinor_even(ns, dims, 11), M0, 0.1, 0.5, w),
            (syn.gaussian_spinor_even(ns, dims, 12), M0, 0.5, 2 * M0, w)]


@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
def test_md_is_reversible(oracle_lib, integrator):
    dims, ns = (2, 2, 2, 4), 4
    U, w = _case(dims, ns, seed=8)
    P = syn.gaussian_momenta(dims, 9)
    step = hmc.md_leapfrog if integrator == "leapfrog" else hmc.md_omelyan
    terms = _terms(U, ns, w)
    U1, P1 = step(U, P, 0.05, 3, terms, 6.2)
    U2, P2 = step(U1, -P1, 0.05, 3, terms, 6.2)
    assert np.abs(U2 - U).max() < 1e-9 and np.abs(P2 + P).max() < 1e-9
    assert np.abs(U1 - U).max() > 1e-2  # the trajectory moved


def test_md_conserves_energy_to_second_order(oracle_lib):
    dims, ns = (2, 2, 2, 4), 4
    U, w = _case(dims, ns, seed=10, eps=0.3)
    P = syn.gaussian_momenta(dims, 13)
    terms = _terms(U, ns, w)
    H0 = hmc.hamiltonian(U, P, terms, 6.2)
    tau = 0.2
    dH = {}
    for name, step in (("leapfrog", hmc.md_leapfrog), ("omelyan", hmc.md_omelyan)):
        dH[name] = []
        for n in (16, 32):  # steps small against the fermion force (max |Pi| ~ 190 here)
            U1, P1 = step(U, P, tau / n, n, terms, 6.2)
            dH[name].append(abs(hmc.hamiltonian(U1, P1, terms, 6.2) - H0))
        r = dH[name][0] / dH[name][1]
        assert 3.0 < r < 5.5, (name, dH[name], r)
    assert dH["omelyan"][1] < 0.5 * dH["leapfrog"][1], dH


@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
def test_nested_integrator_limits(oracle_lib, integrator):
    dims, ns = (2, 2, 2, 4), 4
    U, w = _case(dims, ns, seed=14, eps=0.4)
    P = syn.gaussian_momenta(dims, 15)
    single = hmc.md_leapfrog if integrator == "leapfrog" else hmc.md_omelyan
    k = 1 if integrator == "leapfrog" else 2
    # gauge only: the inner integrator alone, n_inner (x2 for Omelyan's two drifts) per outer step
    U1, P1 = hmc.md_nested(U, P, 0.08, 2, [], 6.2, 3, integrator)
    U2, P2 = single(U, P, 0.08 / (k * 3), 2 * k * 3, [], 6.2)
    assert np.abs(U1 - U2).max() < 1e-13 and np.abs(P1 - P2).max() < 1e-12
    # no gauge force: the inner drifts compose to the outer one
    terms = _terms(U, ns, w)
    U1, P1 = hmc.md_nested(U, P, 0.05, 2, terms, 0.0, 3, integrator)
    U2, P2 = single(U, P, 0.05, 2, terms, 0.0)
    assert np.abs(U1 - U2).max() < 1e-12 and np.abs(P1 - P2).max() < 1e-10
    assert np.abs(U1 - U).max() > 1e-2


def test_nested_integrator_is_reversible_and_second_order(oracle_lib):
    dims, ns = (2, 2, 2, 4), 4
    U, w = _case(dims, ns, seed=10, eps=0.3)
    P = syn.gaussian_momenta(dims, 13)
    terms = _terms(U, ns, w)
    U1, P1 = hmc.md_nested(U, P, 0.05, 3, terms, 6.2, 2)
    U2, P2 = hmc.md_nested(U1, -P1, 0.05, 3, terms, 6.2, 2)
    assert np.abs(U2 - U).max() < 1e-9 and np.abs(P2 + P).max() < 1e-9
    H0 = hmc.hamiltonian(U, P, terms, 6.2)
    dH = []
    for n in (16, 32):
        U1, P1 = hmc.md_nested(U, P, 0.2 / n, n, terms, 6.2, 2)
        dH.append(abs(hmc.hamiltonian(U1, P1, terms, 6.2) - H0))
    assert 3.0 < dH[0] / dH[1] < 5.5, dH


def test_kinetic_energy_closed_form():
    """K = -sum tr P^2 = 1/2 sum_a p_a^2 for P = sum_a p_a T_a, T_a = i lambda_a / 2
    (tr(lambda_a lambda_b) = 2 delta_ab)."""
    dims = (2, 2, 2, 4)
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(31)
    p = rng.standard_normal((4, lt, lz, ly, lx, 8))
    P = np.einsum("...a,aij->...ij", p, 1j * syn.gell_mann() / 2)
    assert abs(hmc.kinetic(P) - 0.5 * np.sum(p ** 2)) < 1e-12 * np.sum(p ** 2)
