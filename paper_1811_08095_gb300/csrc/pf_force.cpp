// Two-flavour pseudofermion action and force of the ODWF operator (Sec. 2: the two-flavour parts
// of the HMC, with mass preconditioning), on the handle's gauge field.
//
// Reading (the action's formula is cited, not printed): det D(m) = det(M(m))^2 det S(m) for the
// even-odd split and M has no links, so the ratio det[D(m1)^+ D(m1)] / det[D(m2)^+ D(m2)] is, up
// to a constant, det[S1^+ S1] / det[S2^+ S2] (S_i the Schur operator at m_i), represented by
//     S_pf = phi^+ S2^+ (S1^+ S1)^-1 S2 phi = |S1 X|^2,   X = (S1^+ S1)^-1 S2 phi.
// Its derivative along U_mu(x) -> exp(eps T) U_mu(x) is
//     dS = 2 Re<X, dS2 phi> - 2 Re<Y, dS1 X>,   Y = S1 X,
//     <A, dS psi> = 1/2 <L1, dW (B R1)> + 1/2 <L2, dW (B psi)>,
//     L1 = M^-+ A (even), R1 = M^-1 H_oe psi (odd), L2 = M^-+ H_eo^+ M^-+ A (odd),
// with H = -1/2 W B, and each <L, dW R> is the link contraction of kernels_force.cu.
#include <cmath>

#include "engine.h"
#include "profile.h"

namespace odwf {

namespace {
// a device input passes through; host data is copied into a workspace
int stage_phi(Engine* E, const void* in, size_t bytes, cudaStream_t st, const double2** out) {
    if (is_device_ptr(in)) {
        *out = (const double2*)in;
        return ODWF_OK;
    }
    int rc = 0;
    void* d = E->get_ws("pf.in", bytes, &rc);
    if (rc) return rc;
    ODWF_CK(cudaMemcpyAsync(d, in, bytes, cudaMemcpyHostToDevice, st));
    *out = (const double2*)d;
    return ODWF_OK;
}

// the four fields of one <A, dS(m) psi> term: Le = L1, Lo = L2, Re = B psi, Ro = B R1
int term_fields(Engine* E, const HalfField& A, const HalfField& psi, const double* r, HalfField& Le, HalfField& Lo,
                HalfField& Re, HalfField& Ro, HalfField& T, cudaStream_t st) {
    const size_t vh = E->vh();
    const int ns = E->ns;
    ODWF_CK(launch_m5_f64(A.ref_sys(0), Le.ref_sys(0), vh, ns, r, 0, 1, 3, E->cf64, st));  // L1 = M^-+ A
    auto P = E->hop_params<double>(1, r);
    P.in = psi.ref_sys(0);
    P.out = T.ref_sys(0);
    ODWF_CK(launch_hop_f64(P, Epi::PLAIN, 1, st));                                           // H_oe psi
    ODWF_CK(launch_m5_f64(T.ref_sys(0), Ro.ref_sys(0), vh, ns, r, 0, 1, 2, E->cf64, st));  // R1 = M^-1 H_oe psi
    ODWF_CK(launch_m5_f64(Ro.ref_sys(0), T.ref_sys(0), vh, ns, r, 0, 1, 4, E->cf64, st));  // B R1
    ODWF_CK(cudaMemcpyAsync(Ro.data, T.data, Ro.stride, cudaMemcpyDeviceToDevice, st));
    P = E->hop_params<double>(1, r);
    P.in = Le.ref_sys(0);
    P.out = T.ref_sys(0);
    ODWF_CK(launch_hop_f64(P, Epi::D_PLAIN, 1, st));                                         // H_eo^+ L1
    ODWF_CK(launch_m5_f64(T.ref_sys(0), Lo.ref_sys(0), vh, ns, r, 0, 1, 3, E->cf64, st));  // L2
    ODWF_CK(launch_m5_f64(psi.ref_sys(0), Re.ref_sys(0), vh, ns, r, 0, 1, 4, E->cf64, st));  // B psi
    return ODWF_OK;
}
}  // namespace

int Engine::pf_force(const void* phi, double m1, double m2, const odwf_solve_params* prm, double* action, void* force,
                     odwf_solve_stats* stats, cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "odwf_pf_force: gauge field not set");
    if (!phi || !action) return fail(ODWF_EINVAL, "odwf_pf_force: null phi or action");
    if (!std::isfinite(m1) || !std::isfinite(m2)) return fail(ODWF_EINVAL, "odwf_pf_force: non-finite mass");
    int rc = check_params(prm);
    if (rc) return rc;
    const size_t eb = ext_bytes(ODWF_MODE_SCHUR_EVEN);
    const double2* dphi = nullptr;
    if ((rc = stage_phi(this, phi, eb, st, &dphi))) return rc;
    // r = m / (2 m0) of the two masses, on the device
    double* r = (double*)get_ws("pf.r", 2 * sizeof(double), &rc);
    if (rc) return rc;
    const double rv[2] = {m1 / (2.0 * m0), m2 / (2.0 * m0)};
    ODWF_CK(cudaMemcpyAsync(r, rv, sizeof(rv), cudaMemcpyHostToDevice, st));
    ODWF_CK(cudaStreamSynchronize(st));  // rv lives on this stack frame
    const double* r1 = r;
    const double* r2 = r + 1;
    HalfField Phi, Psi, X, Y, Le, Lo, Re, Ro, T;
    if ((rc = alloc_half("pf.phi", Sp::F64, 1, &Phi)) || (rc = alloc_half("pf.psi", Sp::F64, 1, &Psi)) ||
        (rc = alloc_half("pf.x", Sp::F64, 1, &X)) || (rc = alloc_half("pf.y", Sp::F64, 1, &Y)))
        return rc;
    ODWF_CK(launch_pack(Sp::F64, dphi, Phi.ref_sys(0), g, 0, ns, 1, st));
    if ((rc = apply_schur64(Phi, Psi, false, r2, st))) return rc;  // psi = S2 phi
    // X = (S1^+ S1)^-1 psi through the library's CG (external layout in and out)
    double2* bext = (double2*)get_ws("pf.bext", eb, &rc);
    if (rc) return rc;
    double2* xext = (double2*)get_ws("pf.xext", eb, &rc);
    if (rc) return rc;
    ODWF_CK(launch_unpack(Sp::F64, Psi.ref_sys(0), bext, g, 0, ns, 1, st));
    odwf_solve_params p1 = *prm;
    p1.system = ODWF_SYS_SCHUR_NORMAL;
    p1.mq = m1;
    void* xs[1] = {xext};
    const void* bs[1] = {bext};
    odwf_solve_stats st1{};
    rc = solve(1, xs, bs, &m1, &p1, &st1, st);
    if (stats) *stats = st1;
    if (rc) return rc;
    ODWF_CK(launch_pack(Sp::F64, xext, X.ref_sys(0), g, 0, ns, 1, st));
    if ((rc = apply_schur64(X, Y, false, r1, st))) return rc;  // Y = S1 X
    double* acts = (double*)get_ws("pf.sum", (sumsq_partials() + 1) * sizeof(double), &rc);
    if (rc) return rc;
    ODWF_CK(launch_sumsq((const double*)Y.data, Y.stride / sizeof(double), acts, acts + sumsq_partials(), st));
    ODWF_CK(cudaMemcpyAsync(action, acts + sumsq_partials(), sizeof(double), cudaMemcpyDeviceToHost, st));
    if (force) {
        if ((rc = check_ptr_device(force, device, "odwf_pf_force"))) return rc;
        if ((rc = alloc_half("pf.le", Sp::F64, 1, &Le)) || (rc = alloc_half("pf.lo", Sp::F64, 1, &Lo)) ||
            (rc = alloc_half("pf.re", Sp::F64, 1, &Re)) || (rc = alloc_half("pf.ro", Sp::F64, 1, &Ro)) ||
            (rc = alloc_half("pf.t", Sp::F64, 1, &T)))
            return rc;
        const size_t gb = (size_t)8 * vh() * 9 * sizeof(double2);
        double2* G = (double2*)get_ws("pf.G", gb, &rc);
        if (rc) return rc;
        // 2 Re<X, dS2 phi>: weight 2 x 1/2; then -2 Re<Y, dS1 X>
        // algorithmic bytes per link: four spinors per s, the link, G in and out
        const double cbytes = 8.0 * (double)vh() * (4.0 * ns * 192 + 144 + 2 * 144);
        if ((rc = term_fields(this, X, Phi, r2, Le, Lo, Re, Ro, T, st))) return rc;
        {
            ProfScope ps("pf.force_contract", cbytes, st);
            ODWF_CK(launch_force_contract(g, ns, links_d18, Le.ref_sys(0), Lo.ref_sys(0), Re.ref_sys(0), Ro.ref_sys(0),
                                          1.0, G, false, st));
        }
        if ((rc = term_fields(this, Y, X, r1, Le, Lo, Re, Ro, T, st))) return rc;
        {
            ProfScope ps("pf.force_contract", cbytes, st);
            ODWF_CK(launch_force_contract(g, ns, links_d18, Le.ref_sys(0), Lo.ref_sys(0), Re.ref_sys(0), Ro.ref_sys(0),
                                          -1.0, G, true, st));
        }
        const size_t fb = (size_t)8 * vh() * 9 * sizeof(double2);
        const bool fdev = is_device_ptr(force);
        double2* fout = fdev ? (double2*)force : (double2*)get_ws("pf.fext", fb, &rc);
        if (rc) return rc;
        ODWF_CK(launch_force_finalize(g, G, fout, st));
        if (!fdev) ODWF_CK(cudaMemcpyAsync(force, fout, fb, cudaMemcpyDeviceToHost, st));
    }
    ODWF_CK(cudaStreamSynchronize(st));
    return ODWF_OK;
}

// Heat bath of the two-flavour ratio: phi = S2^-1 S1^+ eta gives S_pf(phi) = |eta|^2 for a
// Gaussian eta, i.e. phi drawn from exp(-S_pf).  S2 phi = S1^+ eta is solved through the normal
// equations, phi = (S2^+ S2)^-1 S2^+ S1^+ eta, by the library's CG at m2.
int Engine::pf_heatbath(const void* eta, double m1, double m2, const odwf_solve_params* prm, void* phi,
                        odwf_solve_stats* stats, cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "odwf_pf_heatbath: gauge field not set");
    if (!eta || !phi) return fail(ODWF_EINVAL, "odwf_pf_heatbath: null eta or phi");
    if (!std::isfinite(m1) || !std::isfinite(m2)) return fail(ODWF_EINVAL, "odwf_pf_heatbath: non-finite mass");
    int rc = check_params(prm);
    if (rc) return rc;
    const size_t eb = ext_bytes(ODWF_MODE_SCHUR_EVEN);
    const double2* deta = nullptr;
    if ((rc = stage_phi(this, eta, eb, st, &deta))) return rc;
    double* r = (double*)get_ws("pf.r", 2 * sizeof(double), &rc);
    if (rc) return rc;
    const double rv[2] = {m1 / (2.0 * m0), m2 / (2.0 * m0)};
    ODWF_CK(cudaMemcpyAsync(r, rv, sizeof(rv), cudaMemcpyHostToDevice, st));
    ODWF_CK(cudaStreamSynchronize(st));  // rv lives on this stack frame
    HalfField E, T;
    if ((rc = alloc_half("pf.phi", Sp::F64, 1, &E)) || (rc = alloc_half("pf.psi", Sp::F64, 1, &T))) return rc;
    ODWF_CK(launch_pack(Sp::F64, deta, E.ref_sys(0), g, 0, ns, 1, st));
    if ((rc = apply_schur64(E, T, true, r, st))) return rc;      // S1^+ eta
    if ((rc = apply_schur64(T, E, true, r + 1, st))) return rc;  // S2^+ S1^+ eta
    double2* bext = (double2*)get_ws("pf.bext", eb, &rc);
    if (rc) return rc;
    ODWF_CK(launch_unpack(Sp::F64, E.ref_sys(0), bext, g, 0, ns, 1, st));
    odwf_solve_params p2 = *prm;
    p2.system = ODWF_SYS_SCHUR_NORMAL;
    p2.mq = m2;
    void* xs[1] = {phi};
    const void* bs[1] = {bext};
    odwf_solve_stats s2{};
    rc = solve(1, xs, bs, &m2, &p2, &s2, st);
    if (stats) *stats = s2;
    if (rc) return rc;
    ODWF_CK(cudaStreamSynchronize(st));
    return ODWF_OK;
}

}  // namespace odwf
