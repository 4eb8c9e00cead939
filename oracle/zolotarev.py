"""Zolotarev optimal weights for ODWF (oracle side; test infrastructure only).

Sec. 2: with c = 1, d = 0 the 4D effective operator of ODWF is
  D_eff = (1 + r)/2 + (1 - r)/2 gamma_5 S(H_w),
  S(H) = (1 - prod_s T_s) / (1 + prod_s T_s),  T_s = (1 - omega_s H) / (1 + omega_s H),
and the optimal weights make S the Zolotarev optimal rational approximation of
sign(H) for lambda in [lambda_min, lambda_max].  R_Z(x) is the optimal rational
approximation of degree (n-1, n) to 1/sqrt(x) on [1, b], b = (lambda_max/lambda_min)^2,
N_s = 2n, and d_Z = max |1 - sqrt(x) R_Z(x)|.  The paper uses the "shifted" form
whose weights carry the R5 symmetry and satisfy 0 <= 1 - S <= 2 d_Z.

Writing A(lambda) = prod_s (1 + omega_s lambda), S = (odd part of A)/(even part of A).
With t(y) = y R_Z(y^2) = y P(y^2)/Q(y^2) (y = lambda/lambda_min):
  * plain weights:   S = t        <=> 1/(omega_s lambda_min) are the 2n roots of Q(y^2) - y P(y^2),
                                      i.e. the 2n points y > 0 where t(y) = 1;
  * shifted weights: S = t/(1+d_Z) <=> roots of (1+d_Z) Q(y^2) - y P(y^2), which are the n
                                      interior maxima of t (t = 1 + d_Z there), each double;
                                      the 2n weights therefore come in equal pairs (R5 symmetry).
Both are found here numerically from those definitions (grid bracketing + brentq on
1 - t, or on d log t / dy for the maxima); the coefficients of R_Z are Zolotarev's elliptic-function
formula, with d_0 fixed by symmetric equioscillation measured on the function itself.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq, minimize_scalar
from scipy.special import ellipj, ellipk
from functools import lru_cache


@lru_cache(maxsize=64)
def zolotarev_coeffs(n: int, b: float):
    """Coefficients of R_Z(x) = d0 prod_{l=1}^{n-1} (x + c_{2l}) / prod_{l=1}^{n} (x + c_{2l-1}).

    c_l = sn^2(l K'/(2n); k') / (1 - sn^2(l K'/(2n); k')), k'^2 = 1 - 1/b, K' = K(k').
    d0 makes 1 - sqrt(x) R_Z(x) equioscillate symmetrically about 0.
    Returns (d0, c_odd[n], c_even[n-1], d_Z)."""
    m = 1.0 - 1.0 / b  # parameter k'^2 (scipy's ellipj / ellipk take m = k^2)
    K = ellipk(m)
    l = np.arange(1, 2 * n)
    sn, _, _, _ = ellipj(l * K / (2 * n), m)
    c = sn ** 2 / (1.0 - sn ** 2)
    c_odd = c[0::2].copy()
    c_even = c[1::2].copy()

    def f(x):
        x = np.asarray(x, dtype=np.float64)
        num = np.ones_like(x)
        for ce in c_even:
            num = num * (x + ce)
        den = np.ones_like(x)
        for co in c_odd:
            den = den * (x + co)
        return np.sqrt(x) * num / den

    fmin, fmax = _extrema(f, 1.0, b)
    d0 = 2.0 / (fmin + fmax)
    dz = (fmax - fmin) / (fmax + fmin)
    return d0, c_odd, c_even, dz


def _extrema(f, a, b, ngrid=20001):
    """Global min and max of f on [a, b]: log grid, then local refinement around each grid extremum."""
    x = np.geomspace(a, b, ngrid)
    y = f(x)
    vals = [y[0], y[-1]]
    for i in range(1, ngrid - 1):
        if (y[i] - y[i - 1]) * (y[i + 1] - y[i]) <= 0:
            lo, hi = x[i - 1], x[i + 1]
            sgn = -1.0 if y[i] >= y[i - 1] else 1.0
            res = minimize_scalar(lambda u: sgn * float(f(np.array([u]))[0]), bounds=(lo, hi),
                                  method="bounded", options={"xatol": 1e-14 * hi})
            vals.append(sgn * res.fun)
    return float(np.min(vals)), float(np.max(vals))


def t_of_y(y, n: int, b: float):
    """t(y) = y R_Z(y^2): the plain Zolotarev approximation of sign(y) for y in [1, sqrt(b)]."""
    d0, c_odd, c_even, _ = zolotarev_coeffs(n, b)
    y = np.asarray(y, dtype=np.float64)
    x = y * y
    num = d0 * np.ones_like(x)
    for ce in c_even:
        num = num * (x + ce)
    den = np.ones_like(x)
    for co in c_odd:
        den = den * (x + co)
    return y * num / den


def sign_approx(lam, ns: int, lmin: float, lmax: float, shifted: bool = True):
    """S(lambda) of the ODWF effective operator: t(lambda/lmin), divided by (1 + d_Z) when shifted."""
    n = ns // 2
    b = (lmax / lmin) ** 2
    _, _, _, dz = zolotarev_coeffs(n, b)
    t = t_of_y(np.asarray(lam) / lmin, n, b)
    return t / (1.0 + dz) if shifted else t


def omega(ns: int, lmin: float, lmax: float, shifted: bool = True):
    """Optimal weights omega_s, s = 1..Ns (Ns even).

    shifted=True (the paper's R5-symmetric choice): the n distinct weights in increasing
    order, mirrored, so omega_s = omega_{Ns+1-s} and the smallest weights sit on the walls.
    shifted=False: the 2n distinct plain-Zolotarev weights in increasing order.
    Returns (omega[Ns], d_Z)."""
    if ns < 2 or ns % 2:
        raise ValueError("Ns must be even and >= 2")
    n = ns // 2
    b = (lmax / lmin) ** 2
    _, _, _, dz = zolotarev_coeffs(n, b)
    ymax = np.sqrt(b)
    g = lambda y: float(t_of_y(np.array([y]), n, b)[0])
    ys = np.geomspace(1.0, ymax, 40001)
    ts = t_of_y(ys, n, b)
    if not shifted:
        e = 1.0 - ts
        roots = []
        for i in range(len(ys) - 1):
            if e[i] == 0.0:
                roots.append(ys[i])
            elif e[i] * e[i + 1] < 0:
                roots.append(brentq(lambda y: 1.0 - g(y), ys[i], ys[i + 1], xtol=1e-15, rtol=1e-15))
        if len(roots) != 2 * n:
            raise ArithmeticError("expected %d crossings of t = 1, found %d" % (2 * n, len(roots)))
        w = np.sort(1.0 / (lmin * np.array(roots)))
        return w, dz
    _, c_odd, c_even, _ = zolotarev_coeffs(n, b)

    def dlogt(y):
        # d/dy log t(y): zero at each interior extremum of t
        return 1.0 / y + sum(2 * y / (y * y + ce) for ce in c_even) - sum(2 * y / (y * y + co) for co in c_odd)

    h = np.array([dlogt(y) for y in ys])
    peaks = []
    for i in range(len(ys) - 1):
        if h[i] > 0 and h[i + 1] <= 0:  # t rises then falls: a maximum
            peaks.append(brentq(dlogt, ys[i], ys[i + 1], xtol=1e-15, rtol=1e-15))
    if len(peaks) != n:
        raise ArithmeticError("expected %d interior maxima of t, found %d" % (n, len(peaks)))
    w = np.sort(1.0 / (lmin * np.array(peaks)))
    return np.concatenate([w, w[::-1]]), dz
