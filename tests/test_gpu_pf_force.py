"""GPU parity of the two-flavour pseudofermion action and force (odwf_pf_force, Sec. 2's HMC
two-flavour parts with mass preconditioning) against the FP64 oracle (oracle/hmc.py), through the
C ABI.  The oracle's force is pinned to finite differences of its action (test_oracle_hmc.py).

Tolerances: with the inner solve in FP64 to 1e-12 the solution X differs from the oracle's
(solved to 1e-13) by at most kappa * 1e-12 relative; the action and every component of the force
inherit that: bars 1e-9 relative (action) and 2e-8 of the largest force component.  With a
mixed-precision solve to 1e-10: 1e-7 and 2e-6.
"""
import numpy as np
import pytest

import odwf_synth as syn
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, from_dev, make_case, to_dev, torch_cuda
from oracle import hmc

pytestmark = pytest.mark.gpu

CASES = [
    ((4, 4, 4, 4), 8, 0.1, 2 * M0, True),   # the plain two-flavour term, m2 = m_PV
    ((2, 4, 2, 4), 4, 0.05, 0.5, False),     # a mass-preconditioning ratio, periodic time
    ((6, 4, 2, 10), 8, 0.01, 0.1, True),     # the paper's m_H1 / m_H2 pair, ragged last block
]


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("dims,ns,m1,m2,tbc", CASES)
def test_pf_force_matches_oracle(torch, dims, ns, m1, m2, tbc):
    U, w = make_case(dims, ns, 0.1, eps=0.5, seed=3)
    h = odwf.Handle(dims, ns, M0, 0.1, w, t_antiperiodic=tbc)
    h.set_gauge(to_dev(torch, U))
    phi = syn.gaussian_spinor_even(ns, dims, 5)
    Pi_ref, S_ref = hmc.pf_force(U, phi, M0, m1, m2, w, tbc)
    F = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    act, st = h.pf_force(to_dev(torch, phi), m1, m2, F, tol=1e-12, max_iter=100000, prec="f64")
    got = from_dev(F)
    scale = np.abs(Pi_ref).max()
    assert abs(act - S_ref) < 1e-9 * S_ref, (act, S_ref)
    assert np.abs(got - Pi_ref).max() < 2e-8 * scale, (np.abs(got - Pi_ref).max(), scale)
    # traceless anti-Hermitian
    assert np.abs(got + np.conj(np.swapaxes(got, -1, -2))).max() < 1e-12 * scale
    assert np.abs(np.trace(got, axis1=-2, axis2=-1)).max() < 1e-12 * scale
    assert st["status"] == 0 and st["true_resid"] <= 1e-12
    # mixed-precision inner solve; host pointers in and out; the action alone
    Fh = np.zeros(U.shape, dtype=np.complex128)
    act2, st2 = h.pf_force(phi, m1, m2, Fh, tol=1e-10, prec="f16")
    assert abs(act2 - S_ref) < 1e-7 * S_ref
    assert np.abs(Fh - Pi_ref).max() < 2e-6 * scale
    act3, _ = h.pf_force(to_dev(torch, phi), m1, m2, None, tol=1e-12, prec="f64")
    assert abs(act3 - act) < 1e-12 * act
    h.close()


def test_pf_force_heatbath_action(torch):
    """phi from the oracle's heat bath has S_pf = |eta|^2 on the GPU too."""
    dims, ns = (4, 4, 2, 4), 4
    U, w = make_case(dims, ns, 0.1, eps=0.4, seed=7)
    eta = syn.gaussian_spinor_even(ns, dims, 8)
    phi = hmc.heatbath_phi(U, eta, M0, 0.02, 0.2, w)
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    h.set_gauge(to_dev(torch, U))
    act, _ = h.pf_force(to_dev(torch, phi), 0.02, 0.2, None, tol=1e-12, prec="f64")
    assert abs(act - np.vdot(eta, eta).real) < 1e-9 * act
    h.close()
