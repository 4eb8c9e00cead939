// The 4D effective operator of Sec. 2 through the 5D solve, and the residual mass read off it.
//
// With P_{s,s'} = P_- delta_{s,s'} + P_+ delta_{s+1,s'} (s + 1 cyclic) and m_PV = 2 m0, the
// (1,1) block of P^-1 D(m_PV)^-1 D(m_q) P is D_eff(m_q) = (1 + r)/2 + (1 - r)/2 gamma_5 S(H_w)
// (r = m_q / (2 m0), S the shifted Zolotarev sign approximation), and the matrix is block
// triangular with identity below, so
//   D_eff(m_q)^-1 b = [P^-1 D(m_q)^-1 D(m_PV) P (b (x) e_1)]_1.
// P (b (x) e_1) puts P_- b on s = 1 and P_+ b on s = Ns; [P^-1 y]_1 = P_- y_1 + P_+ y_Ns.  In the
// chiral basis P_+ keeps spins 0, 1 and P_- spins 2, 3, so both are strided copies of 6 of the
// 12 complex components of every site.
//
// Residual mass (the reading used here): with D(m_q) = 2 m0 D_eff = m_q + (1 - m_q/(2 m0)) D,
// the propagator of the chirally symmetric D_c = D (1 - D/(2 m0))^-1 is
//   G = (D_c + m_q)^-1 = (D_eff^-1 - 1) / (2 m0 - m_q),
// and m_res = tr G_00 / sum_x tr (G_x0^dag G_x0) - m_q for a point source at site 0 (zero when
// S^2 = 1).  The twelve spin-colour columns come from twelve effective solves.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "engine.h"
#include "profile.h"

namespace odwf {

namespace {

// copy spins [sp0, sp0 + 2) of every site between 4D field a and s-slice `s` of 5D field f
// (external layouts; 12 complex per site, 6 per spin pair)
cudaError_t spin_pair_copy(double2* dst, const double2* src, size_t V, int sp0, int s, bool to5d, cudaStream_t st) {
    const size_t pitch = 12 * sizeof(double2), width = 6 * sizeof(double2);
    const size_t off5 = ((size_t)s * V) * 12 + 3 * sp0, off4 = 3 * (size_t)sp0;
    if (to5d) return cudaMemcpy2DAsync(dst + off5, pitch, src + off4, pitch, width, V, cudaMemcpyDeviceToDevice, st);
    return cudaMemcpy2DAsync(dst + off4, pitch, src + off5, pitch, width, V, cudaMemcpyDeviceToDevice, st);
}

}  // namespace

int Engine::effective_solve(void* x, const void* b, const odwf_solve_params* prm, odwf_solve_stats* stats,
                            cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "odwf_effective_solve: gauge field not set");
    NvtxRange nv_("odwf.effective_solve");
    if (!x || !b || !prm) return fail(ODWF_EINVAL, "odwf_effective_solve: null argument");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t V = 2 * vh();
    const size_t b4 = V * 12 * sizeof(double2);
    const size_t e5 = ext_bytes(ODWF_MODE_FULL);
    int rc = 0;
    double2* B4 = (double2*)get_ws("eff.b4", b4, &rc);
    if (rc) return rc;
    double2* X4 = is_device_ptr(x) ? (double2*)x : (double2*)get_ws("eff.x4", b4, &rc);
    if (rc) return rc;
    double2* Eta = (double2*)get_ws("eff.eta", e5, &rc);
    if (rc) return rc;
    double2* Y = (double2*)get_ws("eff.y", e5, &rc);
    if (rc) return rc;
    ODWF_CK(cudaMemcpyAsync(B4, b, b4, cudaMemcpyDefault, st));
    // Y = P (b (x) e_1): P_- b (spins 2, 3) on s = 1, P_+ b (spins 0, 1) on s = Ns
    ODWF_CK(cudaMemsetAsync(Y, 0, e5, st));
    ODWF_CK(spin_pair_copy(Y, B4, V, 2, 0, true, st));
    ODWF_CK(spin_pair_copy(Y, B4, V, 0, ns - 1, true, st));
    // eta = D(m_PV) Y with m_PV = 2 m0 (r = 1), in FP64
    double* rpv = (double*)get_ws("eff.rpv", sizeof(double), &rc);
    if (rc) return rc;
    const double one = 1.0;
    ODWF_CK(cudaMemcpyAsync(rpv, &one, sizeof(double), cudaMemcpyHostToDevice, st));
    HalfField Xe, Xo, Ye, Yo;
    if ((rc = alloc_half("eff.Xe", Sp::F64, 1, &Xe)) || (rc = alloc_half("eff.Xo", Sp::F64, 1, &Xo)) ||
        (rc = alloc_half("eff.Ye", Sp::F64, 1, &Ye)) || (rc = alloc_half("eff.Yo", Sp::F64, 1, &Yo)))
        return rc;
    ODWF_CK(launch_pack(Sp::F64, Y, Xe.ref_sys(0), g, 0, ns, 0, st));
    ODWF_CK(launch_pack(Sp::F64, Y, Xo.ref_sys(0), g, 1, ns, 0, st));
    if ((rc = apply_full64(Xe, Xo, Ye, Yo, false, rpv, st))) return rc;
    ODWF_CK(launch_unpack(Sp::F64, Ye.ref_sys(0), Eta, g, 0, ns, 0, st));
    ODWF_CK(launch_unpack(Sp::F64, Yo.ref_sys(0), Eta, g, 1, ns, 0, st));
    // Y = D(m_q)^-1 eta
    odwf_solve_params p = *prm;
    p.system = ODWF_SYS_FULL_DIRAC;
    odwf_solve_stats s5;
    std::memset(&s5, 0, sizeof(s5));
    rc = solve_full(Y, Eta, &p, &s5, st);
    if (rc && rc != ODWF_ENOCONV && rc != ODWF_EBREAKDOWN) return rc;
    const int solve_rc = rc;
    // x = [P^-1 Y]_1 = P_- Y_1 + P_+ Y_Ns
    ODWF_CK(spin_pair_copy(X4, Y, V, 2, 0, false, st));
    ODWF_CK(spin_pair_copy(X4, Y, V, 0, ns - 1, false, st));
    if (X4 != x) ODWF_CK(cudaMemcpyAsync(x, X4, b4, cudaMemcpyDeviceToHost, st));
    ODWF_CK(cudaStreamSynchronize(st));
    if (stats) {
        *stats = s5;
        stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return solve_rc;
}

int Engine::residual_mass(const int32_t site[4], const odwf_solve_params* prm, double* mres, double* corr,
                          odwf_solve_stats* stats, cudaStream_t st) {
    if (!site || !prm || !mres) return fail(ODWF_EINVAL, "odwf_residual_mass: null argument");
    for (int i = 0; i < 4; ++i)
        if (site[i] < 0 || site[i] >= g.L[i]) return fail(ODWF_EINVAL, "odwf_residual_mass: site outside the lattice");
    const double mqv = std::isfinite(prm->mq) ? prm->mq : mq;
    if (!(2.0 * m0 - mqv != 0.0)) return fail(ODWF_EINVAL, "odwf_residual_mass: m_q = 2 m0");
    const size_t V = 2 * vh();
    const size_t lex = (size_t)site[0] + (size_t)g.L[0] * (site[1] + (size_t)g.L[1] * (site[2] + (size_t)g.L[2] * site[3]));
    const size_t v3 = V / g.L[3];
    std::vector<double2> bsrc(V * 12), col(V * 12);
    double num = 0.0, den = 0.0;
    std::vector<double> ct(g.L[3], 0.0);
    odwf_solve_params p = *prm;
    p.mq = mqv;
    int worst = ODWF_OK, iters = 0, nrel = 0;
    double resid = 0.0, ms = 0.0;
    for (int sc = 0; sc < 12; ++sc) {
        std::memset(bsrc.data(), 0, bsrc.size() * sizeof(double2));
        bsrc[lex * 12 + sc] = make_double2(1.0, 0.0);
        odwf_solve_stats s1;
        std::memset(&s1, 0, sizeof(s1));
        const int rc = effective_solve(col.data(), bsrc.data(), &p, &s1, st);
        if (rc && rc != ODWF_ENOCONV && rc != ODWF_EBREAKDOWN) return rc;
        if (rc && !worst) worst = rc;
        iters += s1.iters;
        nrel += s1.n_reliable;
        resid = std::max(resid, s1.true_resid);
        ms += s1.time_ms;
        // G column sc = (D_eff^-1 delta - delta) / (2 m0 - m_q)
        col[lex * 12 + sc].x -= 1.0;
        const double inv = 1.0 / (2.0 * m0 - mqv);
        num += col[lex * 12 + sc].x * inv;
        for (size_t i = 0; i < V; ++i) {
            double a = 0.0;
            for (int k = 0; k < 12; ++k) a += col[i * 12 + k].x * col[i * 12 + k].x + col[i * 12 + k].y * col[i * 12 + k].y;
            a *= inv * inv;
            den += a;
            ct[i / v3] += a;
        }
    }
    *mres = num / den - mqv;
    if (corr)
        for (int t = 0; t < g.L[3]; ++t) corr[t] = ct[(t + site[3]) % g.L[3]];  // relative to the source time
    if (stats) {
        stats->iters = iters;
        stats->n_reliable = nrel;
        stats->true_resid = resid;
        stats->time_ms = ms;
        stats->status = worst;
    }
    return worst;
}

}  // namespace odwf
