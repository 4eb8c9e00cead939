"""Pins of the oracle's gradient flow and flow observables (Sec. 2 scale condition, Sec. 3
admissibility and clover charge) against facts fixed outside the oracle:

* the flow force is minus the Lie-algebra gradient of the Wilson action (finite differences);
* an abelian wave flows exactly by a scalar ODE, integrated here by scipy's DOP853 (independent
  of the Runge-Kutta scheme), and its small-amplitude limit decays as exp(-k^2 t) with the
  lattice momentum k^2 = 4 sin^2(p/2);
* the flow integrator converges at third order;
* constant-flux abelian fields: closed forms of both energy densities, the clover charge, the
  plaquette minimum, and zero force;
* pure gauges have zero force, energy and charge; the flow is gauge covariant and the
  observables gauge invariant; the action decreases monotonically and the links stay in SU(3);
* a noisy flux-2 field flows to an admissible field whose clover charge is within 1% of 2.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.linalg import expm

import odwf_synth as syn
from oracle import flow as fl

AX = {0: 3, 1: 2, 2: 1, 3: 0}  # mu -> site axis of a (t, z, y, x) field


def _gauge_transform(U, Om):
    """U^Omega_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^+."""
    out = np.empty_like(U)
    for mu in range(4):
        Om_fwd = np.roll(Om, -1, axis=AX[mu])
        out[mu] = np.einsum("...ab,...bc,...dc->...ad", Om, U[mu], Om_fwd.conj())
    return out


def _unit_field(dims):
    lx, ly, lz, lt = dims
    U = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def test_force_is_minus_the_gradient_of_the_wilson_action():
    """d/ds S(exp(s T_a) U_mu(x)) at s = 0 equals 2 tr(T_a Z_mu(x)), T_a = i lambda_a / 2, with
    S = g0^2 S_W = 2 sum_p Re tr(1 - P) computed from the plaquettes (central differences)."""
    dims = (3, 2, 2, 3)
    U = syn.gauge_field(dims, 0.8, 21)
    T = 1j * syn.gell_mann() / 2
    rng = np.random.default_rng(3)
    sites = [tuple(int(rng.integers(0, L)) for L in dims) for _ in range(3)]
    c = np.array(sites, dtype=np.int64)
    Z = fl.force(U, c)
    h = 1e-5
    worst = 0.0
    for i, (x, y, z, t) in enumerate(sites):
        for mu in range(4):
            for a in range(8):
                Up, Um = U.copy(), U.copy()
                Up[mu, t, z, y, x] = expm(h * T[a]) @ U[mu, t, z, y, x]
                Um[mu, t, z, y, x] = expm(-h * T[a]) @ U[mu, t, z, y, x]
                fd = (fl.wilson_action(Up) - fl.wilson_action(Um)) / (2 * h)
                want = 2.0 * np.trace(T[a] @ Z[mu, i]).real
                worst = max(worst, abs(fd - want))
    assert worst < 1e-7, worst
    # and the force is large enough for the check to mean something
    assert np.abs(Z).max() > 0.1


def _wave_rhs(t, th):
    # d theta(y)/dt = -sin(theta(y) - theta(y+1)) + sin(theta(y-1) - theta(y))
    fwd = np.roll(th, -1)
    bwd = np.roll(th, 1)
    return -np.sin(th - fwd) + np.sin(bwd - th)


@pytest.mark.parametrize("mu,nu,amp,n", [(0, 1, 0.8, 1), (3, 2, 1.2, 2), (1, 3, 0.5, 3)])
def test_abelian_wave_flows_by_its_exact_ode(mu, nu, amp, n):
    """With U_mu = diag(e^{i th}, e^{-i th}, 1), th depending on x_nu only, and all other links
    1, the flow stays in this form and th(x_nu) obeys the scalar ODE above (derived from the
    plaquettes of the (mu, nu) plane); the other links stay 1."""
    dims = (4, 6, 4, 8)
    L = dims[nu]
    U = syn.abelian_wave_field(dims, mu, nu, amp, n)
    t_end = 0.4
    th0 = amp * np.cos(2 * np.pi * n * np.arange(L) / L)
    sol = solve_ivp(_wave_rhs, (0.0, t_end), th0, method="DOP853", rtol=1e-12, atol=1e-13)
    th_want = sol.y[:, -1]
    errs = []
    for steps in (40, 80):
        V, _ = fl.flow(U, t_end / steps, steps)
        idx = [0, 0, 0, 0]
        got = []
        for k in range(L):
            idx[3 - nu] = k  # site axes are (t, z, y, x)
            got.append(np.angle(V[(mu,) + tuple(idx)][0, 0]))
        errs.append(np.abs(np.array(got) - th_want).max())
        for m in range(4):
            if m != mu:
                assert np.abs(V[m] - np.eye(3)).max() < 1e-12
    # what is left is the integration error: small, and shrinking fast with the step (the order
    # itself is pinned below)
    assert errs[1] < 5e-8 and errs[0] / errs[1] > 4.0, errs
    # the field is not static: it moved by much more than the tolerance
    assert np.abs(th_want - th0).max() > 1e-2


def test_small_abelian_wave_decays_as_the_lattice_heat_kernel():
    dims = (4, 8, 4, 4)
    amp, n, eps, steps = 1e-4, 1, 0.01, 50
    U = syn.abelian_wave_field(dims, 0, 1, amp, n)
    V, _ = fl.flow(U, eps, steps)
    y = np.arange(dims[1])
    k2 = 4 * np.sin(np.pi * n / dims[1]) ** 2
    want = amp * np.exp(-k2 * eps * steps) * np.cos(2 * np.pi * n * y / dims[1])
    got = np.angle(V[0, 0, 0, :, 0, 0, 0])
    assert np.abs(got - want).max() < 1e-6 * amp


def test_flow_integrator_is_third_order():
    dims = (2, 2, 2, 4)
    U = syn.gauge_field(dims, 0.5, 31)
    t_end = 0.4
    ref, _ = fl.flow(U, t_end / 512, 512)
    errs = []
    for steps in (8, 16, 32):
        V, _ = fl.flow(U, t_end / steps, steps)
        errs.append(np.abs(V - ref).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.0 < r1 < 9.5 and 7.0 < r2 < 9.0, (errs, r1, r2)


FLUXES = {(0, 1): 1, (0, 2): 2, (0, 3): -1, (1, 2): 1, (1, 3): 3, (2, 3): 1}


@pytest.mark.parametrize("charges", [(1, -1, 0), (2, -1, -1)])
def test_constant_flux_closed_forms(charges):
    dims = (4, 4, 6, 6)
    U = syn.flux_field(dims, FLUXES, charges)
    V = syn.volume(dims)
    q = np.array(charges, dtype=np.float64)
    th = {p: 2 * np.pi * FLUXES[p] / (dims[p[0]] * dims[p[1]]) for p in fl.PLANES}
    # every plaquette of plane p is diag(exp(i q_k th_p)); the clover field is its sine, traceless
    f = {}
    for p in fl.PLANES:
        d = np.sin(q * th[p])
        f[p] = d - d.sum() / 3
    e_clov = sum(f[p] @ f[p] for p in fl.PLANES)
    e_plaq = 2 * sum(3 - np.cos(q * th[p]).sum() for p in fl.PLANES)
    qdens = (f[(0, 1)] @ f[(2, 3)] - f[(0, 2)] @ f[(1, 3)] + f[(0, 3)] @ f[(1, 2)]) / (4 * np.pi ** 2)
    pmin = min(np.cos(q * th[p]).sum() / 3 for p in fl.PLANES)
    s = fl.site_observables(U)
    assert np.abs(s["e_clover"] - e_clov).max() < 1e-13
    assert np.abs(s["e_plaq"] - e_plaq).max() < 1e-12
    assert np.abs(s["q"] - qdens).max() < 1e-15
    assert abs(s["plaq_min"].min() - pmin) < 1e-14
    o = fl.observables(U)
    assert abs(o["q"] - V * qdens) < 1e-11
    # a constant field strength is a stationary point of the flow
    assert np.abs(fl.force(U)).max() < 1e-13


def test_flux_charge_approaches_the_integer():
    """n_{xy} = n_{zt} = 1 with charges (1, -1, 0) carries Q = 2 n_{xy} n_{zt} in the continuum;
    the clover value is V sin(th_xy) sin(th_zt) / (2 pi^2) on the lattice."""
    for L in (8, 16):
        dims = (L, L, L, L)
        U = syn.flux_field(dims, {(0, 1): 1, (2, 3): 1})
        th = 2 * np.pi / L ** 2
        want = L ** 4 * np.sin(th) ** 2 / (2 * np.pi ** 2)
        c = fl.all_sites(dims)[:: max(1, L ** 4 // 512)]  # the density is constant: sample it
        qd = fl.site_observables(U, c)["q"]
        assert np.abs(qd * L ** 4 - want).max() < 1e-9
        assert abs(want - 2) < 0.01 * (8 / L) ** 4


def test_pure_gauge_has_no_force_energy_or_charge():
    dims = (4, 2, 4, 2)
    Om = syn.gauge_field(dims, 2.0, 41)[0]
    U = _gauge_transform(_unit_field(dims), Om)
    assert np.abs(fl.force(U)).max() < 1e-13
    o = fl.observables(U)
    assert abs(o["e_plaq"]) < 1e-13 and abs(o["e_clover"]) < 1e-13 and abs(o["q"]) < 1e-13
    assert abs(o["plaq_min"] - 1.0) < 1e-14


def test_flow_is_gauge_covariant_and_observables_invariant():
    dims = (4, 2, 2, 4)
    U = syn.gauge_field(dims, 0.7, 51)
    Om = syn.gauge_field(dims, 2.0, 52)[0]
    Ug = _gauge_transform(U, Om)
    V1 = fl.rk3_step(U, 0.05)
    V2 = fl.rk3_step(Ug, 0.05)
    assert np.abs(_gauge_transform(V1, Om) - V2).max() < 1e-13
    o1, o2 = fl.observables(V1), fl.observables(V2)
    for k in ("e_plaq", "e_clover", "q", "plaq_min"):
        assert abs(o1[k] - o2[k]) < 1e-12
    # the force itself transforms covariantly: Z[U^Omega](x) = Omega(x) Z[U](x) Omega(x)^+
    Z, Zg = fl.force(U), fl.force(Ug)
    Omf = Om.reshape(-1, 3, 3)
    assert np.abs(np.einsum("nab,mnbc,ndc->mnad", Omf, Z, Omf.conj()) - Zg).max() < 1e-13


def test_action_decreases_and_links_stay_special_unitary():
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, 1.0, 61)
    S = [fl.wilson_action(U)]
    V = U
    for _ in range(10):
        V = fl.rk3_step(V, 0.02)
        S.append(fl.wilson_action(V))
    assert all(b < a for a, b in zip(S, S[1:])), S
    assert S[-1] < 0.8 * S[0]
    W = V.reshape(-1, 3, 3)
    assert np.abs(W @ fl.dag(W) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(W) - 1).max() < 1e-13


@pytest.mark.slow
def test_noisy_flux_flows_to_an_admissible_field_of_integer_charge():
    """Sec. 3: once every plaquette satisfies Re tr P / 3 > 44/45 the clover charge sits near an
    integer.  A flux-2 field (8^4, Q_clover = 1.99 clean) with random noise is not admissible;
    after flow it is, and its charge is back near 2."""
    dims = (8, 8, 8, 8)
    clean = syn.flux_field(dims, {(0, 1): 1, (2, 3): 1})
    noise = syn.gauge_field(dims, 0.35, 71)
    U = noise @ clean
    o0 = fl.observables(U)
    assert o0["plaq_min"] < fl.ADMISSIBLE
    V, obs = fl.flow(U, 0.02, 50, measure_every=25)
    o = obs[-1]
    assert o["plaq_min"] > fl.ADMISSIBLE, o
    assert abs(o["q"] - 2.0) < 0.02, (o0["q"], o["q"])
    assert o["e_clover"] < 0.05 * o0["e_clover"]


def test_t0_scale_interpolates_the_crossing():
    ts = np.arange(0, 1.01, 0.1)
    t1 = 0.37
    es = np.where(ts > 0, 0.3 * ts / t1 / np.maximum(ts, 1e-30) ** 2, 0.0)  # t^2 E = 0.3 t / t1
    assert abs(fl.t0_scale(ts, es) - t1) < 1e-12
    assert fl.t0_scale(ts, es * 0.1) is None
