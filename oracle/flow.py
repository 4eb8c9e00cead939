"""Gradient (Wilson) flow of the gauge field and the observables measured on it (Sec. 2, Sec. 3).

TEST INFRASTRUCTURE ONLY: the test suite, `__graft_entry__.smoke()` and the benchmark's
CPU-baseline leg are the only users; the CUDA library shares nothing with this file.

Plain numpy in fp64.  Sites are held as integer coordinate arrays (n, 4) = (x, y, z, t),
wrapped periodically, so the same functions serve a whole small lattice and a sample of
sites of a large one.  Gauge layout as in odwf_synth: U[mu][t][z][y][x][a][b], mu = 0..3
<-> x, y, z, t, lattice spacing a = 1.

Definitions written out below:
  plaquette       P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
  projection      ta(X) = (X - X^+)/2 - tr(X - X^+)/6, the traceless anti-Hermitian part
  flow force      Z_mu(x) = -ta(U_mu(x) S_mu(x)), S_mu(x) the sum over nu != mu of the
                  upper and lower staples, so that U_mu(x) S_mu(x) is the sum of the six
                  plaquette loops through the link; Z = -g0^2 d S_W for the Wilson action
                  S_W = beta sum_p (1 - Re tr P / 3), beta = 6 / g0^2
  flow            dV/dt = Z(V) V (Sec. 2, the flow of the scale condition), integrated with
                  the third-order Runge-Kutta scheme for this equation given by Luscher
                  (JHEP 2010, appendix C); the paper names the flow and the step 0.01 but
                  not the integrator
  field strength  F_{mu nu}(x) = (Q - Q^+)/(8i) made traceless, Q the sum of the four
                  plaquette loops in the (mu, nu) plane that start and end at x (Sec. 3)
  energy density  E(x) = sum_{mu<nu} tr F_{mu nu}(x)^2 (clover), or
                  E(x) = 2 sum_{mu<nu} Re tr(1 - P_{mu nu}(x)) (plaquette); both tend to
                  -tr G_{mu nu} G_{mu nu} / 2 of the continuum field
  charge          Q = sum_x eps_{mu nu rho sigma} tr[F_{mu nu} F_{rho sigma}] / (32 pi^2)
                  (Sec. 3), eps_{xyzt} = +1
  admissibility   min over all plaquettes of Re tr P / 3, compared with 44/45 (Sec. 3)
  scale           t0 where t^2 <E(t)> = 0.3 (Sec. 2), linear interpolation between the
                  measured flow times
Parity status: pinned by tests/test_oracle_flow.py (finite-difference gradient of the
Wilson action, the exact flow of abelian waves against an independent ODE integration,
third-order convergence, closed forms of constant-flux fields, pure gauges, gauge
covariance, monotone action, near-integer charge after flow).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

EYE4 = np.eye(4, dtype=np.int64)
ADMISSIBLE = 44.0 / 45.0
T0_TARGET = 0.3


def dims_of(U):
    lt, lz, ly, lx = U.shape[1:5]
    return (lx, ly, lz, lt)


def all_sites(dims) -> np.ndarray:
    """Coordinates (x, y, z, t) of every site, x fastest (the lexicographic site order)."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1).astype(np.int64)


def link(U, mu, c):
    """U_mu at the (wrapped) sites c, shape (n, 3, 3)."""
    lx, ly, lz, lt = dims_of(U)
    return U[mu, c[:, 3] % lt, c[:, 2] % lz, c[:, 1] % ly, c[:, 0] % lx]


def dag(A):
    return np.conj(np.swapaxes(A, -1, -2))


def ta(X):
    """Traceless anti-Hermitian part of X."""
    A = 0.5 * (X - dag(X))
    tr = np.trace(A, axis1=-2, axis2=-1)
    return A - (tr / 3.0)[..., None, None] * np.eye(3)


def plaquette(U, mu, nu, c):
    e_mu, e_nu = EYE4[mu], EYE4[nu]
    return link(U, mu, c) @ link(U, nu, c + e_mu) @ dag(link(U, mu, c + e_nu)) @ dag(link(U, nu, c))


def staple_sum(U, mu, c):
    """S_mu(x): for each nu != mu the staple above (through x+nu) and below (through x-nu)."""
    e_mu = EYE4[mu]
    S = np.zeros((len(c), 3, 3), dtype=np.complex128)
    for nu in range(4):
        if nu == mu:
            continue
        e_nu = EYE4[nu]
        S += link(U, nu, c + e_mu) @ dag(link(U, mu, c + e_nu)) @ dag(link(U, nu, c))
        S += dag(link(U, nu, c + e_mu - e_nu)) @ dag(link(U, mu, c - e_nu)) @ link(U, nu, c - e_nu)
    return S


def force(U, c=None) -> np.ndarray:
    """Z_mu(x) for mu = 0..3 at the sites c (all sites, lexicographic, if None): (4, n, 3, 3)."""
    if c is None:
        c = all_sites(dims_of(U))
    return np.stack([-ta(link(U, mu, c) @ staple_sum(U, mu, c)) for mu in range(4)])


def _as_field(Z, U):
    return Z.reshape(U.shape)


def rk3_step(U, eps: float) -> np.ndarray:
    """One flow step V_t -> V_{t+eps}: three force evaluations, each stage a left
    multiplication by the exponential of a combination of eps Z_0, eps Z_1, eps Z_2."""
    Z0 = eps * _as_field(force(U), U)
    W1 = expm(Z0 / 4.0) @ U
    Z1 = eps * _as_field(force(W1), U)
    W2 = expm(8.0 / 9.0 * Z1 - 17.0 / 36.0 * Z0) @ W1
    Z2 = eps * _as_field(force(W2), U)
    return expm(3.0 / 4.0 * Z2 - 8.0 / 9.0 * Z1 + 17.0 / 36.0 * Z0) @ W2


def clover(U, mu, nu, c):
    """Hermitian traceless F_{mu nu} at the sites c from the four plaquette loops around x."""
    e_mu, e_nu = EYE4[mu], EYE4[nu]
    l1 = plaquette(U, mu, nu, c)
    l2 = link(U, nu, c) @ dag(link(U, mu, c - e_mu + e_nu)) @ dag(link(U, nu, c - e_mu)) @ link(U, mu, c - e_mu)
    l3 = (dag(link(U, mu, c - e_mu)) @ dag(link(U, nu, c - e_mu - e_nu)) @ link(U, mu, c - e_mu - e_nu)
          @ link(U, nu, c - e_nu))
    l4 = dag(link(U, nu, c - e_nu)) @ link(U, mu, c - e_nu) @ link(U, nu, c + e_mu - e_nu) @ dag(link(U, mu, c))
    Q = l1 + l2 + l3 + l4
    F = (Q - dag(Q)) / 8j
    tr = np.trace(F, axis1=-2, axis2=-1)
    return F - (tr / 3.0)[..., None, None] * np.eye(3)


PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def _trace_prod(A, B):
    return np.einsum("nab,nba->n", A, B)


def site_observables(U, c=None):
    """Per site: clover and plaquette energy densities, charge density, and the smallest
    Re tr P / 3 of the six plaquettes based at the site."""
    if c is None:
        c = all_sites(dims_of(U))
    F = {p: clover(U, *p, c) for p in PLANES}
    e_clover = sum(_trace_prod(F[p], F[p]).real for p in PLANES)
    q = (_trace_prod(F[(0, 1)], F[(2, 3)]) - _trace_prod(F[(0, 2)], F[(1, 3)])
         + _trace_prod(F[(0, 3)], F[(1, 2)])).real / (4.0 * np.pi ** 2)
    retr = np.stack([np.trace(plaquette(U, *p, c), axis1=-2, axis2=-1).real for p in PLANES])
    e_plaq = 2.0 * (3.0 - retr).sum(axis=0)
    return {"e_clover": e_clover, "e_plaq": e_plaq, "q": q, "plaq_min": retr.min(axis=0) / 3.0,
            "plaq_sum": retr.sum(axis=0) / 3.0}


def observables(U, t: float = 0.0) -> dict:
    """Lattice averages of the energy densities and of Re tr P / 3, the total charge and the
    admissibility minimum (Sec. 3)."""
    s = site_observables(U)
    V = len(s["q"])
    return {"t": t, "e_plaq": s["e_plaq"].mean(), "e_clover": s["e_clover"].mean(), "q": s["q"].sum(),
            "plaq_min": s["plaq_min"].min(), "plaq_mean": s["plaq_sum"].sum() / (6 * V)}


def wilson_action(U) -> float:
    """g0^2 S_W = 2 sum_x sum_{mu<nu} Re tr(1 - P_{mu nu}(x)) = sum_x E_plaq(x)."""
    c = all_sites(dims_of(U))
    return float(sum((3.0 - np.trace(plaquette(U, *p, c), axis1=-2, axis2=-1).real).sum() for p in PLANES) * 2.0)


def flow(U, eps: float, nsteps: int, measure_every: int = 0):
    """Integrate nsteps steps of size eps.  With measure_every > 0 the observables are taken at
    t = 0 and after every measure_every steps (t = k eps)."""
    obs = []
    V = np.array(U, dtype=np.complex128, copy=True)
    for k in range(nsteps):
        if measure_every and k % measure_every == 0:
            obs.append(observables(V, k * eps))
        V = rk3_step(V, eps)
    if measure_every and nsteps % measure_every == 0:
        obs.append(observables(V, nsteps * eps))
    return V, obs


def t0_scale(ts, es, target: float = T0_TARGET):
    """First flow time where t^2 E(t) reaches target (linear interpolation in t between the
    two bracketing measurements), or None if it is not reached."""
    f = np.asarray(ts, dtype=np.float64) ** 2 * np.asarray(es, dtype=np.float64) - target
    for i in range(1, len(f)):
        if f[i - 1] < 0.0 <= f[i]:
            return ts[i - 1] + (ts[i] - ts[i - 1]) * (-f[i - 1]) / (f[i] - f[i - 1])
    return None
