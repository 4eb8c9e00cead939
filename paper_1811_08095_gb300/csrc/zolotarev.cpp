// Optimal ODWF weights from Zolotarev's optimal rational approximation (host, FP64).
//
// R_Z(x) = d0 prod_{l=1}^{n-1} (x + c_{2l}) / prod_{l=1}^{n} (x + c_{2l-1}) on x in [1, b],
// b = (lmax/lmin)^2, Ns = 2n, c_l = sn^2(u_l; k') / cn^2(u_l; k'), u_l = l K'/(2n),
// k'^2 = 1 - 1/b, K' = K(k').  The error 1 - sqrt(x) R_Z(x) equioscillates; its 2n+1
// extrema sit at x_l = 1/dn^2(u_l; k'), l = 0..2n, which fixes d0 and d_Z.
// With t(y) = y R_Z(y^2) and A(lambda) = prod_s (1 + omega_s lambda), the 4D effective
// sign function of ODWF is S = (odd part of A)/(even part of A) (Sec. 2):
//   shifted (R5-symmetric) weights: S = t/(1 + d_Z); the roots of (1+d_Z) Q - y P are the
//     interior maxima y = 1/dn(u_l), l odd, each double, so omega = dn(u_{2k-1}; k')/lmin twice;
//   plain weights: S = t; omega = 1/(lmin y) at the 2n crossings t(y) = 1, one between each
//     pair of neighbouring extrema (found by bisection).
// Elliptic functions: K by the arithmetic-geometric mean; sn, cn, dn by the descending
// Landen (AGM) recursion of Abramowitz & Stegun 16.4.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/odwf.h"

namespace odwf {

int fail(int code, const std::string& msg);

namespace {

const double kPi = 3.14159265358979323846;

// complete elliptic integral of the first kind, modulus k (0 <= k < 1)
double ellip_K(double k) {
    double a = 1.0, b = std::sqrt(1.0 - k * k);
    for (int i = 0; i < 60 && std::fabs(a - b) > 1e-16 * a; ++i) {
        const double an = 0.5 * (a + b);
        b = std::sqrt(a * b);
        a = an;
    }
    return kPi / (2.0 * a);
}

// Jacobi sn, cn, dn of argument u and modulus k (A&S 16.4.3)
void ellip_sncndn(double u, double k, double* sn, double* cn, double* dn) {
    const int NMAX = 40;
    double a[NMAX + 1], c[NMAX + 1];
    a[0] = 1.0;
    double b = std::sqrt(1.0 - k * k);
    c[0] = k;
    int n = 0;
    while (n < NMAX && std::fabs(c[n]) > 1e-17) {
        const double an = 0.5 * (a[n] + b);
        const double cn1 = 0.5 * (a[n] - b);
        b = std::sqrt(a[n] * b);
        ++n;
        a[n] = an;
        c[n] = cn1;
    }
    double phi = std::ldexp(1.0, n) * a[n] * u;
    double phi_next = phi;
    for (int i = n; i >= 1; --i) {
        phi_next = phi;
        phi = 0.5 * (phi + std::asin(c[i] * std::sin(phi) / a[i]));
    }
    *sn = std::sin(phi);
    *cn = std::cos(phi);
    *dn = (n >= 1) ? std::cos(phi) / std::cos(phi_next - phi) : 1.0;
}

struct Zolo {
    int n;
    double b;
    std::vector<double> c_odd, c_even;  // n and n-1 coefficients
    std::vector<double> y_ext;          // extremal points y_l = 1/dn(u_l), l = 0..2n
    double d0, dz;

    double f(double x) const {  // sqrt(x) prod (x + c_even) / prod (x + c_odd), without d0
        double num = 1.0, den = 1.0;
        for (double ce : c_even) num *= (x + ce);
        for (double co : c_odd) den *= (x + co);
        return std::sqrt(x) * num / den;
    }
    double t(double y) const { return d0 * f(y * y); }
};

Zolo make_zolo(int n, double b) {
    Zolo z;
    z.n = n;
    z.b = b;
    const double kp = std::sqrt(1.0 - 1.0 / b);
    const double Kp = ellip_K(kp);
    for (int l = 1; l <= 2 * n - 1; ++l) {
        double sn, cn, dn;
        ellip_sncndn(l * Kp / (2.0 * n), kp, &sn, &cn, &dn);
        const double cl = (sn * sn) / (cn * cn);
        if (l & 1) z.c_odd.push_back(cl); else z.c_even.push_back(cl);
    }
    double fmin = 1e300, fmax = -1e300;
    for (int l = 0; l <= 2 * n; ++l) {
        double sn, cn, dn;
        ellip_sncndn(l * Kp / (2.0 * n), kp, &sn, &cn, &dn);
        double y = 1.0 / dn;
        if (l == 0) y = 1.0;
        if (l == 2 * n) y = std::sqrt(b);
        z.y_ext.push_back(y);
        const double fv = z.f(y * y);
        fmin = std::min(fmin, fv);
        fmax = std::max(fmax, fv);
    }
    z.d0 = 2.0 / (fmin + fmax);
    z.dz = (fmax - fmin) / (fmax + fmin);
    return z;
}

}  // namespace

int zolotarev_omega(int Ns, double lmin, double lmax, int variant, double* omega, double* dz_out) {
    if (!omega) return fail(ODWF_EINVAL, "odwf_zolotarev_omega: null output");
    if (Ns < 2 || Ns > 64 || (Ns & 1)) return fail(ODWF_EINVAL, "odwf_zolotarev_omega: Ns must be even, 2..64");
    if (!(lmin > 0.0) || !(lmax > lmin) || !std::isfinite(lmax))
        return fail(ODWF_EINVAL, "odwf_zolotarev_omega: need 0 < lmin < lmax");
    if (variant != ODWF_OMEGA_SHIFTED_R5 && variant != ODWF_OMEGA_PLAIN)
        return fail(ODWF_EINVAL, "odwf_zolotarev_omega: unknown variant");
    const int n = Ns / 2;
    const double b = (lmax / lmin) * (lmax / lmin);
    const Zolo z = make_zolo(n, b);
    std::vector<double> w;
    if (variant == ODWF_OMEGA_SHIFTED_R5) {
        const double kp = std::sqrt(1.0 - 1.0 / b);
        const double Kp = ellip_K(kp);
        for (int k = 1; k <= n; ++k) {
            double sn, cn, dn;
            ellip_sncndn((2 * k - 1) * Kp / (2.0 * n), kp, &sn, &cn, &dn);
            w.push_back(dn / lmin);
        }
        std::sort(w.begin(), w.end());
        for (int k = 0; k < n; ++k) omega[k] = w[k];
        for (int k = 0; k < n; ++k) omega[Ns - 1 - k] = w[k];
    } else {
        for (int l = 0; l < 2 * n; ++l) {
            double lo = z.y_ext[l], hi = z.y_ext[l + 1];
            double glo = 1.0 - z.t(lo);
            for (int it = 0; it < 200 && hi - lo > 1e-16 * hi; ++it) {
                const double mid = 0.5 * (lo + hi);
                const double gm = 1.0 - z.t(mid);
                if ((gm < 0) == (glo < 0)) {
                    lo = mid;
                    glo = gm;
                } else {
                    hi = mid;
                }
            }
            w.push_back(1.0 / (lmin * 0.5 * (lo + hi)));
        }
        std::sort(w.begin(), w.end());
        for (int k = 0; k < Ns; ++k) omega[k] = w[k];
    }
    if (dz_out) *dz_out = z.dz;
    return ODWF_OK;
}

}  // namespace odwf
