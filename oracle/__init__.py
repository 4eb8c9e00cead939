"""FP64 CPU oracle for the ODWF operator and its even-odd normal-equation solves.

TEST INFRASTRUCTURE ONLY: the test suite, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg are the only users.  The CUDA library never imports,
links or calls anything here, and this package imports nothing from it.

`odwf_oracle.c` holds the operator (naive loops, definitions written out, see its
header); `zolotarev.py` the optimal weights; `dense.py` dense-matrix builds for the
identities of Sec. 2; `flow.py` the gradient flow of the gauge field and the flow
observables (energy density, clover charge, admissibility) of Sec. 2-3; `hmc.py` the
two-flavour pseudofermion action and force, the Wilson gauge force and the molecular-dynamics
integrators of the paper's HMC (Sec. 2).  Parity status: every function here is pinned by tests under
`tests/test_oracle_*.py` (free-field closed form, gamma_5-hermiticity, gauge
covariance, dense adjoint, the effective-operator / shifted-Zolotarev identity of
Sec. 2, the determinant-ratio identity of Eq. (1)-(2), dense Schur complement, dense
LU solves, Zolotarev equioscillation and the bound 0 <= 1 - S <= 2 d_Z).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "odwf_oracle.c")
_LIB = os.path.join(_HERE, "libodwf_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain C11 + OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.oracle_dw.argtypes = [P, P, I, D, P, P, I]
            lib.oracle_d5.argtypes = [P, P, I, I, D, D, P, P, P, P, I]
            lib.oracle_m5.argtypes = [I, D, D, P, P, ctypes.c_long, P, P, I]
            lib.oracle_m5.restype = I
            lib.oracle_b5.argtypes = [I, D, D, P, P, ctypes.c_long, P, P, I]
            lib.oracle_schur.argtypes = [P, P, I, I, D, D, P, P, P, P, I]
            lib.oracle_cg.argtypes = [I, P, P, I, I, D, D, P, P, P, P, D, I, I, ctypes.POINTER(D), P]
            lib.oracle_cg.restype = I
            lib.oracle_num_threads.restype = I
            lib.oracle_gammas.argtypes = [P]
            _lib = lib
    return _lib


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(U):
    # U has shape (4, Lt, Lz, Ly, Lx, 3, 3)
    lt, lz, ly, lx = U.shape[1:5]
    return np.array([lx, ly, lz, lt], dtype=np.int32)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def gammas() -> np.ndarray:
    """gamma_1..gamma_4 and gamma_5 (= g1 g2 g3 g4) as used by the oracle, shape (5, 4, 4)."""
    out = np.zeros((5, 4, 4), dtype=np.complex128)
    _load().oracle_gammas(_p(out))
    return out


def dw(U, psi, m0: float, tbc: bool = True, dagger: bool = False) -> np.ndarray:
    """4D Wilson operator D_w (or its adjoint) on a 4D field of shape (Lt, Lz, Ly, Lx, 4, 3)."""
    U = _c(U)
    psi = _c(psi)
    out = np.empty_like(psi)
    dims = _dims(U)
    _load().oracle_dw(_p(U), _p(dims), int(tbc), float(m0), _p(psi), _p(out), int(dagger))
    return out


def _rs(ns, omega, rho, sigma):
    if rho is None:
        rho = omega
    if sigma is None:
        sigma = omega
    rho = _c(rho, np.float64)
    sigma = _c(sigma, np.float64)
    assert rho.shape == (ns,) and sigma.shape == (ns,)
    return rho, sigma


def d5(U, psi, m0: float, mq: float, omega=None, tbc: bool = True, dagger: bool = False,
       rho=None, sigma=None) -> np.ndarray:
    """5D ODWF operator D(m_q) (or D^dag) on a full field of shape (Ns, Lt, Lz, Ly, Lx, 4, 3).

    rho_s = c omega_s + d, sigma_s = c omega_s - d; with the paper's c = 1, d = 0 both
    equal omega (pass rho / sigma explicitly for other choices)."""
    U = _c(U)
    psi = _c(psi)
    ns = psi.shape[0]
    rho, sigma = _rs(ns, omega, rho, sigma)
    out = np.empty_like(psi)
    _load().oracle_d5(_p(U), _p(_dims(U)), int(tbc), ns, float(m0), float(mq), _p(rho), _p(sigma),
                      _p(psi), _p(out), int(dagger))
    return out


M, MDAG, MINV, MINVDAG = 0, 1, 2, 3


def m5(psi, m0: float, mq: float, omega=None, op: int = M, rho=None, sigma=None) -> np.ndarray:
    """Site-local part M of D (op 0), M^dag (1), M^-1 (2) or M^-dag (3) on any 5D field
    whose first axis is s and whose last two axes are (spin, colour)."""
    psi = _c(psi)
    ns = psi.shape[0]
    rho, sigma = _rs(ns, omega, rho, sigma)
    nsite = psi.size // (12 * ns)
    out = np.empty_like(psi)
    rc = _load().oracle_m5(ns, float(m0), float(mq), _p(rho), _p(sigma), nsite, _p(psi), _p(out), int(op))
    if rc != 0:
        raise ArithmeticError("singular site-local matrix M")
    return out


def b5(psi, m0: float, mq: float, omega=None, dagger: bool = False, rho=None, sigma=None) -> np.ndarray:
    """The chiral shift B = rho + sigma L of D = D_w B + 1 - L (or B^dag = rho + L^dag sigma) on
    any 5D field whose first axis is s and whose last two axes are (spin, colour)."""
    psi = _c(psi)
    ns = psi.shape[0]
    rho, sigma = _rs(ns, omega, rho, sigma)
    nsite = psi.size // (12 * ns)
    out = np.empty_like(psi)
    _load().oracle_b5(ns, float(m0), float(mq), _p(rho), _p(sigma), nsite, _p(psi), _p(out), int(dagger))
    return out


def hop_w(U, half, parity_in: int, m0: float, tbc: bool = True, dagger: bool = False) -> np.ndarray:
    """-1/2 W psi (or -1/2 W^dag psi) on a half field (Ns, V/2, 4, 3) of parity `parity_in`,
    returned on the other parity: the hopping part of D_w = (4 - m0) - W/2, taken from the
    Wilson operator applied slice by slice to the parity-embedded field (its diagonal term
    stays on the input parity and drops out)."""
    lt, lz, ly, lx = U.shape[1:5]
    dims = (lx, ly, lz, lt)
    full = from_parity(_c(half), dims, parity_in)
    out = np.empty_like(full)
    for s in range(full.shape[0]):
        out[s] = dw(U, full[s], m0, tbc, dagger)
    return to_parity(out, dims, 1 - parity_in)


def schur(U, psi_e, m0: float, mq: float, omega=None, tbc: bool = True, dagger: bool = False,
          rho=None, sigma=None) -> np.ndarray:
    """Even-odd Schur operator S = 1 - M^-1 H_eo M^-1 H_oe (or S^dag) on an even-site field
    of shape (Ns, V/2, 4, 3)."""
    U = _c(U)
    psi_e = _c(psi_e)
    ns = psi_e.shape[0]
    rho, sigma = _rs(ns, omega, rho, sigma)
    out = np.empty_like(psi_e)
    _load().oracle_schur(_p(U), _p(_dims(U)), int(tbc), ns, float(m0), float(mq), _p(rho), _p(sigma),
                         _p(psi_e), _p(out), int(dagger))
    return out


SCHUR_NORMAL, FULL_NORMAL = 0, 1


def cg(U, b, m0: float, mq: float, omega=None, tbc: bool = True, system: int = SCHUR_NORMAL,
       tol: float = 1e-12, max_iter: int = 100000, x0=None, rho=None, sigma=None, coefs=None):
    """CG on S^dag S x = b (even-site b) or D^dag D x = b (full b).

    Returns (x, iterations, true relative residual); iterations = -1 if not converged.
    coefs: optional float64 array of 2 * max_iter entries that receives alpha_k, beta_k of
    every iteration (the Lanczos coefficients: see lanczos_extremes)."""
    U = _c(U)
    b = _c(b)
    ns = b.shape[0]
    rho, sigma = _rs(ns, omega, rho, sigma)
    x = np.zeros_like(b) if x0 is None else _c(x0).copy()
    res = ctypes.c_double(0.0)
    it = _load().oracle_cg(int(system), _p(U), _p(_dims(U)), int(tbc), ns, float(m0), float(mq),
                           _p(rho), _p(sigma), _p(b), _p(x), float(tol), int(max_iter),
                           int(x0 is not None), ctypes.byref(res),
                           None if coefs is None else _p(coefs))
    return x, int(it), float(res.value)


def lanczos_extremes(coefs, iters):
    """Smallest and largest eigenvalue estimates of the normal operator from `iters` CG
    iterations' alpha_k, beta_k (CG is the Lanczos process: its tridiagonal matrix has
    T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_{k,k+1} = sqrt(beta_k)/alpha_k, and the extreme
    eigenvalues of T converge to those of the operator from inside the spectrum)."""
    a = np.asarray(coefs[0:2 * iters:2], dtype=np.float64)
    bt = np.asarray(coefs[1:2 * iters:2], dtype=np.float64)
    n = len(a)
    diag = 1.0 / a
    diag[1:] += bt[:-1] / a[:-1]
    off = np.sqrt(bt[:-1]) / a[:-1]
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    ev = np.linalg.eigvalsh(T) if n else np.array([np.nan])
    return float(ev[0]), float(ev[-1])


def normal_op(U, psi, m0, mq, omega=None, tbc=True, system=SCHUR_NORMAL, rho=None, sigma=None):
    """A psi with A = S^dag S (even fields) or D^dag D (full fields)."""
    if system == SCHUR_NORMAL:
        t = schur(U, psi, m0, mq, omega, tbc, False, rho, sigma)
        return schur(U, t, m0, mq, omega, tbc, True, rho, sigma)
    t = d5(U, psi, m0, mq, omega, tbc, False, rho, sigma)
    return d5(U, t, m0, mq, omega, tbc, True, rho, sigma)


def to_even(full, dims):
    """Even-site part of a full 5D field: (Ns, Lt, Lz, Ly, Lx, 4, 3) -> (Ns, V/2, 4, 3)."""
    ns = full.shape[0]
    f = full.reshape(ns, -1, 4, 3)
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    ev = np.nonzero(((x + y + z + t) % 2).reshape(-1) == 0)[0]
    return np.ascontiguousarray(f[:, ev])


def from_parity(half, dims, parity):
    """Embed a half field (Ns, V/2, 4, 3) of the given parity into a full 5D field."""
    ns = half.shape[0]
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    idx = np.nonzero(((x + y + z + t) % 2).reshape(-1) == parity)[0]
    out = np.zeros((ns, lx * ly * lz * lt, 4, 3), dtype=np.complex128)
    out[:, idx] = half
    return out.reshape(ns, lt, lz, ly, lx, 4, 3)


def to_parity(full, dims, parity):
    ns = full.shape[0]
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    idx = np.nonzero(((x + y + z + t) % 2).reshape(-1) == parity)[0]
    return np.ascontiguousarray(full.reshape(ns, -1, 4, 3)[:, idx])
