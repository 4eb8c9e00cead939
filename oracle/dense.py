"""Dense-matrix builds from the FP64 oracle, for the identities the paper states (Sec. 2).

Test infrastructure only.  Matrices are built column by column by applying the
oracle to unit vectors, in the flattened external layouts:
  4D:  index = (site * 4 + spin) * 3 + colour
  5D:  index = ((s * V + site) * 4 + spin) * 3 + colour      (s-major)
"""
from __future__ import annotations

import numpy as np

from . import d5, dw, gammas, schur, zolotarev


def _dims_of(U):
    lt, lz, ly, lx = U.shape[1:5]
    return (lx, ly, lz, lt)


def dense_dw(U, m0, tbc=True, dagger=False):
    lx, ly, lz, lt = _dims_of(U)
    n = 12 * lx * ly * lz * lt
    out = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        out[:, j] = dw(U, e.reshape(lt, lz, ly, lx, 4, 3), m0, tbc, dagger).reshape(-1)
    return out


def dense_d5(U, ns, m0, mq, omega, tbc=True, dagger=False):
    lx, ly, lz, lt = _dims_of(U)
    n = 12 * ns * lx * ly * lz * lt
    out = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        out[:, j] = d5(U, e.reshape(ns, lt, lz, ly, lx, 4, 3), m0, mq, omega, tbc, dagger).reshape(-1)
    return out


def dense_schur(U, ns, m0, mq, omega, tbc=True, dagger=False):
    lx, ly, lz, lt = _dims_of(U)
    vh = lx * ly * lz * lt // 2
    n = 12 * ns * vh
    out = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        out[:, j] = schur(U, e.reshape(ns, vh, 4, 3), m0, mq, omega, tbc, dagger).reshape(-1)
    return out


def gamma5_4d(V):
    g5 = gammas()[4]
    return np.kron(np.eye(V), np.kron(g5, np.eye(3)))


def chiral_perm(ns, V):
    """P_{s,s'} = P_- delta_{s,s'} + P_+ delta_{s+1,s'} (s+1 taken cyclically), 5D dense."""
    g5 = gammas()[4]
    pp = 0.5 * (np.eye(4) + g5)
    pm = 0.5 * (np.eye(4) - g5)
    blk_m = np.kron(np.eye(V), np.kron(pm, np.eye(3)))
    blk_p = np.kron(np.eye(V), np.kron(pp, np.eye(3)))
    n4 = 12 * V
    P = np.zeros((ns * n4, ns * n4), dtype=np.complex128)
    for s in range(ns):
        P[s * n4:(s + 1) * n4, s * n4:(s + 1) * n4] += blk_m
        s2 = (s + 1) % ns
        P[s * n4:(s + 1) * n4, s2 * n4:(s2 + 1) * n4] += blk_p
    return P


def effective_from_5d(U, ns, m0, mq, omega, tbc=True):
    """(P^-1 D(m_PV)^-1 D(m_q) P)_{11}, the 4D effective operator of the 5D theory, m_PV = 2 m0."""
    lx, ly, lz, lt = _dims_of(U)
    V = lx * ly * lz * lt
    D = dense_d5(U, ns, m0, mq, omega, tbc)
    Dpv = dense_d5(U, ns, m0, 2.0 * m0, omega, tbc)
    P = chiral_perm(ns, V)
    X = np.linalg.solve(P, np.linalg.solve(Dpv, D @ P))
    n4 = 12 * V
    return X[:n4, :n4], D, Dpv


def effective_zolotarev(U, ns, m0, mq, lmin, lmax, shifted=True, tbc=True):
    """(1 + r)/2 + (1 - r)/2 gamma_5 S(H_w), r = m_q/(2 m0), S the (shifted) Zolotarev sign
    approximation applied to H_w = gamma_5 D_w by eigendecomposition."""
    lx, ly, lz, lt = _dims_of(U)
    V = lx * ly * lz * lt
    g5 = gamma5_4d(V)
    Hw = g5 @ dense_dw(U, m0, tbc)
    Hw = 0.5 * (Hw + Hw.conj().T)
    lam, vec = np.linalg.eigh(Hw)
    S = (vec * zolotarev.sign_approx(lam, ns, lmin, lmax, shifted)) @ vec.conj().T
    r = mq / (2.0 * m0)
    return 0.5 * (1 + r) * np.eye(12 * V) + 0.5 * (1 - r) * g5 @ S, lam


def effective_dense(U, ns, m0, mq, lmin, lmax, shifted=True, tbc=True, exact_sign=False):
    """D_eff(m_q) of Sec. 2 as a dense 4D matrix: (1 + r)/2 + (1 - r)/2 gamma_5 S(H_w) with
    S the (shifted) Zolotarev sign approximation, or the exact sign function when exact_sign."""
    if not exact_sign:
        return effective_zolotarev(U, ns, m0, mq, lmin, lmax, shifted, tbc)[0]
    lx, ly, lz, lt = _dims_of(U)
    V = lx * ly * lz * lt
    g5 = gamma5_4d(V)
    Hw = g5 @ dense_dw(U, m0, tbc)
    Hw = 0.5 * (Hw + Hw.conj().T)
    lam, vec = np.linalg.eigh(Hw)
    S = (vec * np.sign(lam)) @ vec.conj().T
    r = mq / (2.0 * m0)
    return 0.5 * (1 + r) * np.eye(12 * V) + 0.5 * (1 - r) * g5 @ S


def effective_propagator(Deff, b4):
    """x = D_eff^-1 b for a 4D field b of shape (Lt, Lz, Ly, Lx, 4, 3) (dense LU solve)."""
    return np.linalg.solve(Deff, np.asarray(b4).reshape(-1)).reshape(np.shape(b4))


def residual_mass(Deff, m0, mq, site_index):
    """Residual mass read off the 4D effective operator at one source site.

    With D(m_q) = 2 m0 D_eff = m_q + (1 - m_q/(2 m0)) D, the valence propagator of the chirally
    symmetric operator D_c = D (1 - D/(2 m0))^-1 is G = (D_c + m_q)^-1 = (D_eff^-1 - 1)/(2 m0 - m_q).
    m_res = tr G_00 / sum_x tr (G_x0^dag G_x0) - m_q (the second sum equals
    tr [gamma_5 (D_c + m_q) gamma_5 (D_c + m_q)]^-1_00 by gamma_5-hermiticity); it vanishes when
    S^2 = 1.  Returns (m_res, numerator, denominator, per_site) with per_site[x] =
    tr (G_x0^dag G_x0) for every site x (lexicographic)."""
    n = Deff.shape[0]
    V = n // 12
    cols = slice(12 * site_index, 12 * site_index + 12)
    rhs = np.zeros((n, 12), dtype=np.complex128)
    rhs[cols, :] = np.eye(12)
    G = (np.linalg.solve(Deff, rhs) - rhs) / (2.0 * m0 - mq)  # columns G_{x0}, x over all sites
    num = np.trace(G[cols, :]).real
    per_site = (np.abs(G) ** 2).reshape(V, 12, 12).sum(axis=(1, 2))
    den = per_site.sum()
    return num / den - mq, num, den, per_site
