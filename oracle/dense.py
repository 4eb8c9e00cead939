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
