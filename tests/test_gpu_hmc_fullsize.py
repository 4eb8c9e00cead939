"""The HMC pieces at the size and in the launch configuration of `bench.py --workload hmc`
(16^3 x 32, Ns = 16, m0 = 1.3, shifted Zolotarev weights on [0.05, 6.2], a field of the bench's
recipe exp(0.25 i H), beta = 6.2, f16 solves).

* Gauge action and force: against the oracle at every link (numpy, seconds at this size).
  Bar 1e-12 of the largest component / relative, as on the small lattices.
* Pseudofermion action and force: the oracle's solve at this size takes hours, so a property that
  holds at any size is checked instead, gauge covariance. Under U_mu(x) -> W(x) U_mu(x)
  W(x+mu)^+ and phi(x) -> W(x) phi(x) (W a random SU(3) field) the action is unchanged and the
  force becomes W(x) Pi_mu(x) W(x)^+. Every link and site enters, so a wrong neighbour, link
  orientation, parity or boundary sign at this size breaks it. Solves to 1e-12 (condition number
  ~5e3 at m = 0.01): bars 1e-9 relative (action) and 1e-7 of the largest force component.
* One Omelyan step with Sexton-Weingarten nesting, run forward and back with P -> -P, returns to
  the starting links to 1e-8 (the reversibility the integrator has at any size).
"""
import numpy as np
import pytest

import odwf_synth as syn
import oracle
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, from_dev, to_dev, torch_cuda
from oracle import hmc, zolotarev

pytestmark = pytest.mark.gpu

DIMS, NS, BETA = (16, 16, 16, 32), 16, 6.2
AX = {0: 3, 1: 2, 2: 1, 3: 0}  # array axis of direction mu in a [t][z][y][x] site field


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def case():
    U = syn.gauge_field(DIMS, 0.25, 21)
    w, _ = zolotarev.omega(NS, 0.05, 6.2, True)
    return U, w


def test_gauge_force_full_size_matches_oracle(torch, case):
    U, w = case
    h = odwf.Handle(DIMS, NS, M0, 0.01, w)
    F = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    S = h.gauge_force(to_dev(torch, U), BETA, F)
    Pi_ref = hmc.gauge_force(U, BETA)
    S_ref = hmc.gauge_action(U, BETA)
    assert abs(S - S_ref) <= 1e-12 * abs(S_ref), (S, S_ref)
    err = np.abs(from_dev(F) - Pi_ref).max()
    assert err <= 1e-12 * np.abs(Pi_ref).max(), err
    h.close()


def _transform(U, phi, W):
    """U_mu(x) -> W(x) U_mu(x) W(x+mu)^+, phi(x) -> W(x) phi(x) (phi on the even sites)."""
    Wd = np.conj(np.swapaxes(W, -1, -2))
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = W @ U[mu] @ np.roll(Wd, -1, axis=AX[mu])
    full = oracle.from_parity(phi, DIMS, 0)
    full = np.einsum("tzyxab,stzyxib->stzyxia", W, full)
    return Ug, oracle.to_parity(full, DIMS, 0)


def test_pf_force_full_size_gauge_covariant(torch, case):
    U, w = case
    W = syn.gauge_field(DIMS, 1.0, 77)[0]  # a random SU(3) matrix per site
    phi = syn.gaussian_spinor_even(NS, DIMS, 24)
    Ug, phig = _transform(U, phi, W)
    h = odwf.Handle(DIMS, NS, M0, 0.01, w)
    F = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    h.set_gauge(to_dev(torch, U))
    S1, st1 = h.pf_force(to_dev(torch, phi), 0.01, 0.1, F, tol=1e-12, prec="f16")
    F1 = from_dev(F)
    h.set_gauge(to_dev(torch, Ug))
    S2, st2 = h.pf_force(to_dev(torch, phig), 0.01, 0.1, F, tol=1e-12, prec="f16")
    F2 = from_dev(F)
    assert st1["status"] == 0 and st2["status"] == 0
    assert abs(S2 - S1) <= 1e-9 * abs(S1), (S1, S2)
    expect = W[None] @ F1 @ np.conj(np.swapaxes(W, -1, -2))[None]
    scale = np.abs(F1).max()
    assert np.abs(F2 - expect).max() <= 1e-7 * scale, (np.abs(F2 - expect).max(), scale)
    # the force is not trivially covariant: it differs from the untransformed one
    assert np.abs(F2 - F1).max() > 1e-2 * scale
    h.close()


def test_md_full_size_is_reversible(torch, case):
    U, w = case
    P = syn.gaussian_momenta(DIMS, 22)
    phi = to_dev(torch, syn.gaussian_spinor_even(NS, DIMS, 25))
    h = odwf.Handle(DIMS, NS, M0, 0.1, w)
    Ud, Pd = to_dev(torch, U), to_dev(torch, P)
    H0, H1, st = h.md_trajectory(Ud, Pd, [(phi, 0.1, 2 * M0)], BETA, 0.05, 1, "omelyan", n_inner=4, tol=1e-12,
                                 prec="f16")
    assert st["status"] == 0
    assert np.abs(from_dev(Ud) - U).max() > 1e-3
    Pd.neg_()
    H1b, H2, _ = h.md_trajectory(Ud, Pd, [(phi, 0.1, 2 * M0)], BETA, 0.05, 1, "omelyan", n_inner=4, tol=1e-12,
                                 prec="f16")
    assert abs(H1b - H1) <= 1e-9 * abs(H1)
    assert np.abs(from_dev(Ud) - U).max() <= 1e-8
    assert np.abs(from_dev(Pd) + P).max() <= 1e-8 * np.abs(P).max()
    assert abs(H2 - H0) <= 1e-9 * abs(H0)
    h.close()
