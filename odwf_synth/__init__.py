"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module builds inputs only: gauge links, right-hand-side spinors and point
sources in the library's external layouts.  It holds none of the operator's
arithmetic, so the CPU oracle and the CUDA path can both draw their inputs from
it without sharing any of the computation they are compared on.

Layouts (complex128, C order, x fastest among sites):
  gauge   U[mu][t][z][y][x][a][b]        mu = 0..3 <-> x, y, z, t; row a, column b
  spinor  psi[s][t][z][y][x][spin][col]  s = 0..Ns-1
  even    psi_e[s][i_e][spin][col]       i_e = lexicographic site index // 2 over the
                                          even sites ((x+y+z+t) even), all dims even

Recipe (the paper's runs use 64^4 x 16 ensembles at beta = 6.20, which are not
available; these stand in for them):
  * links U = exp(i eps H) with H = sum_a h_a lambda_a / 2, h_a ~ N(0, 1), lambda_a
    the Gell-Mann matrices; eps = 0.3 / 0.25 / 0.2 for the small, medium and
    paper-scale workloads;
  * right-hand sides with independent unit-Gaussian real and imaginary parts;
  * point sources: a unit spin-colour delta at one seeded site, placed on the
    domain walls (its negative-chirality spins on s = 1, positive on s = Ns);
  * for the gradient flow: abelian fields diag(e^{i q_1 phi}, e^{i q_2 phi}, e^{i q_3 phi}),
    q_1 + q_2 + q_3 = 0, carrying n_{mu nu} units of constant flux through every
    (mu, nu) plane of the torus (optionally times the random links above as noise), and
    single abelian waves phi_mu(x) = a cos(2 pi n x_nu / L_nu).
The random stream is numpy's PCG64 `default_rng(seed)`; the large-lattice path uses
torch's generator on the target device with the same recipe.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann", "gauge_field", "gauge_field_torch", "gaussian_spinor",
    "gaussian_spinor_even", "point_source", "random_site", "random_even_site", "volume",
    "even_sites", "flux_field", "abelian_wave_field", "gaussian_momenta",
]


def volume(dims):
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0] = 1
    l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


def _expm_hermitian(h: np.ndarray, eps: float) -> np.ndarray:
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ab,...b,...cb->...ac", v, ph, v.conj())


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """SU(3) links U = exp(i eps H), H Gaussian traceless Hermitian; shape (4, Lt, Lz, Ly, Lx, 3, 3)."""
    lx, ly, lz, lt = dims
    n = 4 * volume(dims)
    rng = np.random.default_rng(seed)
    lam = gell_mann() / 2
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        h = rng.standard_normal((i1 - i0, 8))
        hm = np.einsum("na,aij->nij", h, lam)
        out[i0:i1] = _expm_hermitian(hm, eps)
    return out.reshape(4, lt, lz, ly, lx, 3, 3)


def gauge_field_torch(dims, eps: float, seed: int, device="cuda"):
    """Same distribution on a torch device (for lattices where the host path is slow)."""
    import torch

    lx, ly, lz, lt = dims
    n = 4 * volume(dims)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    lam = torch.as_tensor(gell_mann() / 2, device=device)
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    chunk = 1 << 22
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        h = torch.randn((i1 - i0, 8), generator=g, device=device, dtype=torch.float64)
        hm = torch.einsum("na,aij->nij", h.to(torch.complex128), lam)
        # matrix exponential by scaling and squaring (no batched eigensolver needed on the device)
        out[i0:i1] = torch.linalg.matrix_exp(1j * eps * hm)
    return out.reshape(4, lt, lz, ly, lx, 3, 3)


def gaussian_spinor(ns: int, dims, seed: int) -> np.ndarray:
    """Full 5D field with unit-Gaussian real and imaginary parts, shape (Ns, Lt, Lz, Ly, Lx, 4, 3)."""
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    shape = (ns, lt, lz, ly, lx, 4, 3)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def gaussian_spinor_even(ns: int, dims, seed: int) -> np.ndarray:
    """Even-site 5D field, shape (Ns, V/2, 4, 3)."""
    rng = np.random.default_rng(seed)
    shape = (ns, volume(dims) // 2, 4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def even_sites(dims) -> np.ndarray:
    """Lexicographic indices of the even sites, in increasing order."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    par = ((x + y + z + t) % 2).reshape(-1)
    return np.nonzero(par == 0)[0]


def random_site(dims, seed: int):
    rng = np.random.default_rng(seed)
    return tuple(int(rng.integers(0, L)) for L in dims)


def random_even_site(dims, seed: int):
    """A seeded site with x + y + z + t even, and its index among the even sites."""
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    while True:
        site = tuple(int(rng.integers(0, L)) for L in dims)
        if sum(site) % 2 == 0:
            x, y, z, t = site
            return site, (((t * lz + z) * ly + y) * lx + x) // 2


def point_source(ns: int, dims, site, spin: int, color: int) -> np.ndarray:
    """Unit spin-colour delta at `site` = (x, y, z, t) on the domain walls.

    In the chiral basis used by the library, spins 0, 1 have gamma_5 = +1 and spins
    2, 3 have gamma_5 = -1.  The negative-chirality part sits on s = 1 and the
    positive-chirality part on s = Ns (full 5D field, shape (Ns, Lt, Lz, Ly, Lx, 4, 3)).
    """
    lx, ly, lz, lt = dims
    x, y, z, t = site
    out = np.zeros((ns, lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    s = ns - 1 if spin < 2 else 0
    out[s, t, z, y, x, spin, color] = 1.0
    return out


def _abelian_links(phases, charges):
    """diag(exp(i q_k phi)) for phases (..., ) and integer charges summing to zero."""
    q = np.asarray(charges, dtype=np.float64)
    assert q.shape == (3,) and abs(q.sum()) < 1e-12
    out = np.zeros(phases.shape + (3, 3), dtype=np.complex128)
    for k in range(3):
        out[..., k, k] = np.exp(1j * q[k] * phases)
    return out


def flux_field(dims, fluxes, charges=(1, -1, 0)) -> np.ndarray:
    """Abelian links with n_{mu nu} = fluxes[(mu, nu)] (mu < nu) flux quanta through each
    (mu, nu) plane: every plaquette of that plane has the phase 2 pi n / (L_mu L_nu) (mod 2 pi).

    phi_mu(x) gets -2 pi n x_nu / (L_mu L_nu); phi_nu(x) gets 2 pi n x_mu / L_mu on the last
    slice x_nu = L_nu - 1, which closes the flux across the periodic boundary."""
    lx, ly, lz, lt = dims
    L = (lx, ly, lz, lt)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    X = (x, y, z, t)
    phi = np.zeros((4, lt, lz, ly, lx))
    for (mu, nu), n in fluxes.items():
        assert mu < nu
        phi[mu] += -2.0 * np.pi * n * X[nu] / (L[mu] * L[nu])
        phi[nu] += np.where(X[nu] == L[nu] - 1, 2.0 * np.pi * n * X[mu] / L[mu], 0.0)
    return _abelian_links(phi, charges)


def abelian_wave_field(dims, mu: int, nu: int, amp: float, n: int, charges=(1, -1, 0)) -> np.ndarray:
    """Links equal to 1 except U_mu(x) = diag(exp(i q_k phi(x_nu))), phi = amp cos(2 pi n x_nu / L_nu)."""
    lx, ly, lz, lt = dims
    L = (lx, ly, lz, lt)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    X = (x, y, z, t)
    phi = np.zeros((4, lt, lz, ly, lx))
    phi[mu] = amp * np.cos(2.0 * np.pi * n * X[nu] / L[nu])
    return _abelian_links(phi, charges)


def gaussian_momenta(dims, seed: int) -> np.ndarray:
    """Molecular-dynamics momenta P = sum_a p_a T_a with T_a = i lambda_a / 2 and p_a ~ N(0, 1)
    (traceless anti-Hermitian), shape (4, Lt, Lz, Ly, Lx, 3, 3) like the gauge field."""
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((4, lt, lz, ly, lx, 8))
    return np.einsum("...a,aij->...ij", p, 1j * gell_mann() / 2)
