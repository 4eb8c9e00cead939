"""Pins of the oracle's Zolotarev weights (Sec. 2): Chebyshev equioscillation of the
optimal approximation, the paper's bound 0 <= 1 - S <= 2 d_Z for the shifted form,
the R5 symmetry of its weights, a brute-force minimax for the lowest degree, and the
stored fixture written by tests/golden/make_golden.py."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import zolotarev

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "zolotarev_weights.json")


def _s_from_weights(lam, w):
    T = np.ones_like(lam)
    for ws in w:
        T = T * (1 - ws * lam) / (1 + ws * lam)
    return (1 - T) / (1 + T)


@pytest.mark.parametrize("ns,lmin,lmax", [(4, 0.05, 6.0), (8, 0.05, 6.0), (16, 0.05, 6.2), (12, 0.1, 3.0)])
def test_equioscillation(ns, lmin, lmax):
    """1 - sqrt(x) R_Z(x) alternates 2n + 1 times between +d_Z and -d_Z on [1, b]."""
    n = ns // 2
    b = (lmax / lmin) ** 2
    _, _, _, dz = zolotarev.zolotarev_coeffs(n, b)
    y = np.geomspace(1, np.sqrt(b), 400001)
    e = 1 - zolotarev.t_of_y(y, n, b)
    assert np.abs(e).max() <= dz * (1 + 1e-9)
    # count sign-alternating near-extremal points
    ext = []
    for i in range(len(y)):
        if abs(abs(e[i]) - dz) < 1e-6 * dz + 1e-15:
            sgn = np.sign(e[i])
            if not ext or ext[-1] != sgn:
                ext.append(sgn)
    assert len(ext) == 2 * n + 1


@pytest.mark.parametrize("ns,lmin,lmax", [(4, 0.05, 6.0), (8, 0.05, 6.0), (16, 0.05, 6.2)])
def test_shifted_bound_and_r5(ns, lmin, lmax):
    """Sec. 2: with the R5-symmetric weights, 0 <= 1 - S(lambda) <= 2 d_Z on [lambda_min, lambda_max],
    S computed from the weights by the product formula."""
    w, dz = zolotarev.omega(ns, lmin, lmax, shifted=True)
    assert np.allclose(w, w[::-1], rtol=0, atol=0)  # omega_s = omega_{Ns+1-s}
    assert np.all(w > 1 / lmax) and np.all(w < 1 / lmin)
    lam = np.geomspace(lmin, lmax, 200001)
    one_minus_s = 1 - _s_from_weights(lam, w)
    assert one_minus_s.min() >= -1e-12
    assert one_minus_s.max() <= 2 * dz
    assert one_minus_s.max() >= 2 * dz / (1 + dz) * (1 - 1e-6)  # the bound is attained


@pytest.mark.parametrize("ns,lmin,lmax", [(4, 0.05, 6.0), (8, 0.05, 6.0), (16, 0.05, 6.0)])
def test_plain_weights_reproduce_zolotarev(ns, lmin, lmax):
    w, dz = zolotarev.omega(ns, lmin, lmax, shifted=False)
    assert len(np.unique(np.round(w, 12))) == ns
    lam = np.geomspace(lmin, lmax, 20001)
    s = _s_from_weights(lam, w)
    t = zolotarev.sign_approx(lam, ns, lmin, lmax, shifted=False)
    assert np.abs(s - t).max() < 1e-12
    assert np.abs(1 - s).max() <= dz * (1 + 1e-9)


def test_lowest_degree_is_minimax():
    """n = 1: R(x) = d0/(x + c) on [1, b]; a brute-force minimax over (d0, c) finds the same error."""
    b = (6.0 / 0.5) ** 2
    _, c_odd, _, dz = zolotarev.zolotarev_coeffs(1, b)
    x = np.geomspace(1, b, 20001)

    def err(p):
        d0, c = np.exp(p)
        return np.abs(1 - np.sqrt(x) * d0 / (x + c)).max()

    best = min((minimize(err, x0, method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-14,
                                                                   "maxiter": 20000})
                for x0 in ([np.log(2 * np.sqrt(b) ** 0.5), np.log(np.sqrt(b))], [0.0, 1.0], [2.0, 3.0])),
               key=lambda r: r.fun)
    assert abs(best.fun - dz) < 1e-6 * dz
    assert abs(np.exp(best.x[1]) - c_odd[0]) < 1e-3 * c_odd[0]


def test_golden_weights():
    with open(GOLDEN) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        w, dz = zolotarev.omega(case["Ns"], case["lmin"], case["lmax"], case["shifted"])
        assert np.allclose(w, case["omega"], rtol=1e-12, atol=0)
        assert abs(dz - case["d_Z"]) < 1e-12 * case["d_Z"]
