"""Pins of the oracle's 4D Wilson operator D_w against facts fixed outside the oracle:
the Clifford algebra, the free-field momentum-space closed form (with the
antiperiodic time boundary), gamma_5-hermiticity and gauge covariance."""
import numpy as np
import pytest

import odwf_synth as syn
import oracle
from oracle import dense

M0 = 1.3


def test_gamma_algebra(oracle_lib):
    g = oracle.gammas()
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * (a == b) * np.eye(4), atol=1e-15)
    # chiral basis: gamma_5 = g1 g2 g3 g4 is diagonal (+1, +1, -1, -1)
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]), atol=1e-15)


@pytest.mark.parametrize("tbc", [True, False])
def test_free_field_closed_form(oracle_lib, tbc):
    """U = 1 and psi(x) = exp(i p.x) chi:  D_w psi = [(4 - m0) - sum cos p + i sum gamma sin p] psi."""
    dims = (4, 6, 4, 8)
    lx, ly, lz, lt = dims
    U = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    g = oracle.gammas()
    rng = np.random.default_rng(5)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    for n in [(0, 0, 0, 0), (1, 2, 3, 1), (3, 5, 1, 6), (2, 3, 2, 4)]:
        p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
             (2 * np.pi * n[3] + (np.pi if tbc else 0.0)) / lt]
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * chi
        got = oracle.dw(U, psi, M0, tbc)
        Dp = (4 - M0 - sum(np.cos(pm) for pm in p)) * np.eye(4) + 1j * sum(g[m] * np.sin(p[m]) for m in range(4))
        want = phase[..., None, None] * (Dp @ chi)
        assert np.abs(got - want).max() < 1e-13


def test_gamma5_hermiticity_dense(oracle_lib):
    dims = (2, 2, 2, 2)
    U = syn.gauge_field(dims, 0.7, 3)
    Dw = dense.dense_dw(U, M0)
    Dwd = dense.dense_dw(U, M0, dagger=True)
    g5 = dense.gamma5_4d(16)
    assert np.abs(Dwd - Dw.conj().T).max() < 1e-14
    assert np.abs(g5 @ Dw @ g5 - Dw.conj().T).max() < 1e-14
    H = g5 @ Dw
    assert np.abs(H - H.conj().T).max() < 1e-14


def test_gauge_covariance(oracle_lib):
    """D_w[U^Omega] (Omega psi) = Omega D_w[U] psi with U^Omega_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^dag."""
    dims = (4, 4, 2, 6)
    lx, ly, lz, lt = dims
    U = syn.gauge_field(dims, 0.9, 7)
    Om = syn.gauge_field(dims, 2.0, 8)[0]  # one random SU(3) matrix per site, (Lt, Lz, Ly, Lx, 3, 3)
    psi = syn.gaussian_spinor(1, dims, 9)[0]
    Ug = np.empty_like(U)
    for mu in range(4):
        ax = {0: 3, 1: 2, 2: 1, 3: 0}[mu]  # site axes are (t, z, y, x)
        Om_fwd = np.roll(Om, -1, axis=ax)
        Ug[mu] = np.einsum("...ab,...bc,...dc->...ad", Om, U[mu], Om_fwd.conj())
    lhs = oracle.dw(Ug, np.einsum("...ab,...sb->...sa", Om, psi), M0, True)
    rhs = np.einsum("...ab,...sb->...sa", Om, oracle.dw(U, psi, M0, True))
    assert np.abs(lhs - rhs).max() < 1e-13
    # the check has teeth: an operator that used U^T in place of U (a transposed index) is
    # not covariant, i.e. D_w[(U^Omega)^T](Omega psi) != Omega D_w[U^T] psi
    tr = lambda A: np.swapaxes(A, -1, -2).copy()
    bad_lhs = oracle.dw(tr(Ug), np.einsum("...ab,...sb->...sa", Om, psi), M0, True)
    bad_rhs = np.einsum("...ab,...sb->...sa", Om, oracle.dw(tr(U), psi, M0, True))
    assert np.abs(bad_lhs - bad_rhs).max() > 1e-3


def test_antiperiodic_sign(oracle_lib):
    """Flipping the sign of every t-link on the last time slice reproduces the antiperiodic operator."""
    dims = (2, 2, 2, 4)
    U = syn.gauge_field(dims, 0.5, 11)
    psi = syn.gaussian_spinor(1, dims, 12)[0]
    Uf = U.copy()
    Uf[3, -1] *= -1
    assert np.abs(oracle.dw(U, psi, M0, True) - oracle.dw(Uf, psi, M0, False)).max() < 1e-14
