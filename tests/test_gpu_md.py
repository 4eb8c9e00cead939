"""GPU parity of the Wilson gauge action and force (odwf_gauge_force) and of the molecular-dynamics
trajectory (odwf_md_trajectory, Sec. 2's HMC: Wilson gauge action at beta = 6.2, two-flavour
pseudofermion terms with mass preconditioning, the Omelyan integrator) against the FP64 oracle
(oracle/hmc.py), through the C ABI.  The oracle's forces are pinned to finite differences of its
actions and its integrators to reversibility and second-order energy conservation
(test_oracle_hmc.py).

Tolerances.  The gauge force and action are FP64 sums of a few hundred products of unit-size
numbers in another order than numpy's: 1e-12 of the largest component (force) and relative
(action).  A trajectory with pseudofermion terms inherits the inner solves' error (FP64 CG to
1e-12 against the oracle's 1e-13, amplified by at most the condition number ~1e3 of these small
cases) in every force evaluation; over a few steps of eps = 0.05 that moves U and P by at most
~1e-9 and H by ~1e-9 relative: bars 1e-8 (fields) and 1e-8 relative (H).  A gauge-only
trajectory has no solve: 1e-11.
"""
import numpy as np
import pytest

import odwf_synth as syn
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, from_dev, make_case, to_dev, torch_cuda
from oracle import hmc

pytestmark = pytest.mark.gpu

BETA = 6.2


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("dims,eps", [((4, 4, 4, 4), 0.5), ((2, 4, 6, 8), 0.9), ((8, 2, 2, 2), 0.2)])
def test_gauge_force_matches_oracle(torch, dims, eps):
    U, w = make_case(dims, 4, 0.1, eps=eps, seed=21)
    h = odwf.Handle(dims, 4, M0, 0.1, w)
    F = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    S = h.gauge_force(to_dev(torch, U), BETA, F)
    Pi_ref = hmc.gauge_force(U, BETA)
    S_ref = hmc.gauge_action(U, BETA)
    got = from_dev(F)
    scale = np.abs(Pi_ref).max()
    assert abs(S - S_ref) <= 1e-12 * abs(S_ref), (S, S_ref)
    assert np.abs(got - Pi_ref).max() <= 1e-12 * scale, (np.abs(got - Pi_ref).max(), scale)
    # host pointers in and out; the action alone
    Fh = np.zeros(U.shape, dtype=np.complex128)
    assert h.gauge_force(U, BETA, Fh) == S
    assert np.array_equal(Fh, got)
    assert h.gauge_force(U, BETA, None) == S
    h.close()


def test_gauge_action_of_the_unit_field_is_zero(torch):
    dims = (4, 4, 2, 6)
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, dims[3], dims[2], dims[1], dims[0], 3, 3)).copy()
    w = np.full(4, 1.0)
    h = odwf.Handle(dims, 4, M0, 0.1, w)
    F = torch.ones(U.shape, dtype=torch.complex128, device="cuda")
    assert h.gauge_force(to_dev(torch, U), BETA, F) == 0.0
    assert float(F.abs().max()) == 0.0
    h.close()


def _terms(dims, ns, w):
    return [(syn.gaussian_spinor_even(ns, dims, 11), 0.1, 0.5),
            (syn.gaussian_spinor_even(ns, dims, 12), 0.5, 2 * M0)]


def _oracle_terms(terms, w):
    return [(phi, M0, m1, m2, w) for phi, m1, m2 in terms]


@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
def test_md_trajectory_matches_oracle(torch, integrator):
    dims, ns = (2, 2, 2, 4), 4
    U, w = make_case(dims, ns, 0.1, eps=0.5, seed=8)
    P = syn.gaussian_momenta(dims, 9)
    terms = _terms(dims, ns, w)
    step = hmc.md_leapfrog if integrator == "leapfrog" else hmc.md_omelyan
    U_ref, P_ref = step(U, P, 0.05, 3, _oracle_terms(terms, w), BETA)
    H0_ref = hmc.hamiltonian(U, P, _oracle_terms(terms, w), BETA)
    H1_ref = hmc.hamiltonian(U_ref, P_ref, _oracle_terms(terms, w), BETA)
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    Ud, Pd = to_dev(torch, U), to_dev(torch, P)
    H0, H1, st = h.md_trajectory(Ud, Pd, [(to_dev(torch, t[0]), t[1], t[2]) for t in terms], BETA, 0.15, 3,
                                 integrator, tol=1e-12, prec="f64")
    assert st["status"] == 0 and st["true_resid"] <= 1e-12
    # 2 terms x (start + force evaluations + end); leapfrog 1 + 3, Omelyan 1 + 6 force evaluations
    assert st["iters"] > 2 * (5 if integrator == "leapfrog" else 8)
    assert abs(H0 - H0_ref) <= 1e-8 * abs(H0_ref), (H0, H0_ref)
    assert abs(H1 - H1_ref) <= 1e-8 * abs(H1_ref), (H1, H1_ref)
    assert np.abs(from_dev(Ud) - U_ref).max() <= 1e-8
    assert np.abs(from_dev(Pd) - P_ref).max() <= 1e-8 * np.abs(P_ref).max()
    h.close()


@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
def test_nested_trajectory_matches_oracle(torch, integrator):
    """Sexton-Weingarten: the gauge force on an inner scale of 3 steps per outer drift."""
    dims, ns = (2, 2, 2, 4), 4
    U, w = make_case(dims, ns, 0.1, eps=0.5, seed=8)
    P = syn.gaussian_momenta(dims, 9)
    terms = _terms(dims, ns, w)
    U_ref, P_ref = hmc.md_nested(U, P, 0.05, 2, _oracle_terms(terms, w), BETA, 3, integrator)
    H1_ref = hmc.hamiltonian(U_ref, P_ref, _oracle_terms(terms, w), BETA)
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    Ud, Pd = to_dev(torch, U), to_dev(torch, P)
    _, H1, st = h.md_trajectory(Ud, Pd, [(to_dev(torch, t[0]), t[1], t[2]) for t in terms], BETA, 0.1, 2,
                                integrator, n_inner=3, tol=1e-12, prec="f64")
    assert st["status"] == 0
    assert abs(H1 - H1_ref) <= 1e-8 * abs(H1_ref), (H1, H1_ref)
    assert np.abs(from_dev(Ud) - U_ref).max() <= 1e-8
    assert np.abs(from_dev(Pd) - P_ref).max() <= 1e-8 * np.abs(P_ref).max()
    # without pseudofermion terms the nested trajectory is 2 x 3 plain gauge steps per outer step
    U1, P1 = to_dev(torch, U), to_dev(torch, P)
    U2, P2 = to_dev(torch, U), to_dev(torch, P)
    k = 1 if integrator == "leapfrog" else 2
    h.md_trajectory(U1, P1, [], BETA, 0.1, 2, integrator, n_inner=3)
    h.md_trajectory(U2, P2, [], BETA, 0.1, 2 * k * 3, integrator)
    assert (U1 - U2).abs().max().item() < 1e-13 and (P1 - P2).abs().max().item() < 1e-12
    h.close()


def test_gauge_only_trajectory_matches_oracle(torch):
    """No pseudofermion term: every step is FP64 arithmetic without a solve (ragged 5D-free case
    on a lattice that spans several blocks)."""
    dims = (4, 4, 6, 8)
    U, w = make_case(dims, 4, 0.1, eps=0.4, seed=31)
    P = syn.gaussian_momenta(dims, 32)
    U_ref, P_ref = hmc.md_omelyan(U, P, 0.1, 4, [], BETA)
    h = odwf.Handle(dims, 4, M0, 0.1, w)
    Ud, Pd = to_dev(torch, U), to_dev(torch, P)
    H0, H1, st = h.md_trajectory(Ud, Pd, [], BETA, 0.4, 4, "omelyan")
    assert st["iters"] == 0
    assert abs(H0 - hmc.hamiltonian(U, P, [], BETA)) <= 1e-11 * abs(H0)
    assert abs(H1 - hmc.hamiltonian(U_ref, P_ref, [], BETA)) <= 1e-11 * abs(H1)
    assert np.abs(from_dev(Ud) - U_ref).max() <= 1e-11
    assert np.abs(from_dev(Pd) - P_ref).max() <= 1e-11 * np.abs(P_ref).max()
    # links stay unitary
    Ug = from_dev(Ud)
    eye = np.einsum("...ab,...cb->...ac", Ug, np.conj(Ug))
    assert np.abs(eye - np.eye(3)).max() < 1e-12
    # zero steps: H at the start twice, fields untouched
    U2, P2 = to_dev(torch, U), to_dev(torch, P)
    H0b, H1b, _ = h.md_trajectory(U2, P2, [], BETA, 0.4, 0, "omelyan")
    assert H0b == H1b == H0
    assert np.array_equal(from_dev(U2), U) and np.array_equal(from_dev(P2), P)
    h.close()


def test_md_trajectory_is_reversible_and_second_order(torch):
    dims, ns = (2, 2, 2, 4), 4
    U, w = make_case(dims, ns, 0.1, eps=0.3, seed=10)
    P = syn.gaussian_momenta(dims, 13)
    terms = _terms(dims, ns, w)
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    tdev = [(to_dev(torch, t[0]), t[1], t[2]) for t in terms]
    Ud, Pd = to_dev(torch, U), to_dev(torch, P)
    H0, H1, _ = h.md_trajectory(Ud, Pd, tdev, BETA, 0.15, 3, "omelyan", tol=1e-12, prec="f64")
    assert np.abs(from_dev(Ud) - U).max() > 1e-2
    Pd.neg_()
    H1b, H2, _ = h.md_trajectory(Ud, Pd, tdev, BETA, 0.15, 3, "omelyan", tol=1e-12, prec="f64")
    assert abs(H1b - H1) <= 1e-10 * abs(H1)
    assert np.abs(from_dev(Ud) - U).max() < 1e-8 and np.abs(from_dev(Pd) + P).max() < 1e-8
    assert abs(H2 - H0) <= 1e-8 * abs(H0)
    # |dH| falls by ~4 when the step halves
    dH = []
    for n in (16, 32):
        Ud, Pd = to_dev(torch, U), to_dev(torch, P)
        a, b, _ = h.md_trajectory(Ud, Pd, tdev, BETA, 0.2, n, "omelyan", tol=1e-12, prec="f64")
        dH.append(abs(b - a))
    assert 3.0 < dH[0] / dH[1] < 5.5, dH
    h.close()


def test_md_trajectory_rejects_bad_arguments(torch):
    dims = (2, 2, 2, 4)
    U, w = make_case(dims, 4, 0.1, seed=1)
    P = syn.gaussian_momenta(dims, 2)
    h = odwf.Handle(dims, 4, M0, 0.1, w)
    Ud, Pd = to_dev(torch, U), to_dev(torch, P)
    with pytest.raises(odwf.OdwfError):
        h.md_trajectory(U, Pd, [], BETA, 0.1, 1)  # host U
    with pytest.raises(odwf.OdwfError):
        h.md_trajectory(Ud, Pd, [], BETA, 0.1, -1)
    with pytest.raises(odwf.OdwfError):
        h.md_trajectory(Ud, Pd, [], float("nan"), 0.1, 1)
    with pytest.raises(odwf.OdwfError):
        h.md_trajectory(Ud, Pd, [], BETA, 0.1, 1, n_inner=-1)
    assert np.array_equal(from_dev(Ud), U)
    h.close()


def test_pf_heatbath_matches_oracle(torch):
    """phi = S2^-1 S1^+ eta against the oracle's heat bath; S_pf(phi) = |eta|^2 on the GPU."""
    dims, ns = (4, 2, 2, 4), 4
    U, w = make_case(dims, ns, 0.1, eps=0.4, seed=7)
    eta = syn.gaussian_spinor_even(ns, dims, 8)
    phi_ref = hmc.heatbath_phi(U, eta, M0, 0.02, 0.2, w)
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    h.set_gauge(to_dev(torch, U))
    phi = torch.zeros(phi_ref.shape, dtype=torch.complex128, device="cuda")
    st = h.pf_heatbath(to_dev(torch, eta), 0.02, 0.2, phi, tol=1e-12, prec="f64")
    assert st["status"] == 0
    got = from_dev(phi)
    assert np.linalg.norm(got - phi_ref) <= 1e-8 * np.linalg.norm(phi_ref)
    act, _ = h.pf_force(phi, 0.02, 0.2, None, tol=1e-12, prec="f64")
    assert abs(act - np.vdot(eta, eta).real) <= 1e-9 * act
    # host buffers in and out, mixed-precision solve
    phih = np.zeros_like(phi_ref)
    h.pf_heatbath(eta, 0.02, 0.2, phih, tol=1e-10, prec="f16")
    assert np.linalg.norm(phih - phi_ref) <= 1e-6 * np.linalg.norm(phi_ref)
    h.close()


def test_hmc_trajectory_matches_oracle(torch):
    """Heat bath, Omelyan molecular dynamics and the Metropolis test against the oracle's pieces."""
    dims, ns = (2, 2, 2, 4), 4
    U, w = make_case(dims, ns, 0.1, eps=0.4, seed=17)
    P = syn.gaussian_momenta(dims, 18)
    masses = [(0.1, 0.5), (0.5, 2 * M0)]
    etas = [syn.gaussian_spinor_even(ns, dims, 19 + k) for k in range(2)]
    phis = [hmc.heatbath_phi(U, e, M0, m1, m2, w) for e, (m1, m2) in zip(etas, masses)]
    terms = [(phi, M0, m1, m2, w) for phi, (m1, m2) in zip(phis, masses)]
    U1_ref, P1_ref = hmc.md_omelyan(U, P, 0.05, 2, terms, BETA)
    dH_ref = hmc.hamiltonian(U1_ref, P1_ref, terms, BETA) - hmc.hamiltonian(U, P, terms, BETA)
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    for u in (0.0, 1.0):  # u = 0 always accepts; u = 1 accepts only dH < 0
        Ud, Pd = to_dev(torch, U), to_dev(torch, P)
        acc, dH = h.hmc_trajectory(Ud, Pd, [to_dev(torch, e) for e in etas], masses, BETA, 0.1, 2, u,
                                   tol=1e-12, prec="f64")
        assert abs(dH - dH_ref) <= 1e-8 * abs(hmc.hamiltonian(U, P, terms, BETA)), (dH, dH_ref)
        assert acc == (dH_ref <= 0 or u < np.exp(-dH_ref))
        assert np.abs(from_dev(Ud) - (U1_ref if acc else U)).max() <= 1e-8
    h.close()
