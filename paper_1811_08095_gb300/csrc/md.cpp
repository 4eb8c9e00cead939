// Wilson gauge action and force and the molecular-dynamics trajectory of the HMC (Sec. 2: the
// Wilson plaquette gauge action at beta = 6/g0^2, the two-flavour pseudofermion terms with mass
// preconditioning, the Omelyan integrator and Sexton-Weingarten multiple time scales).
//
// Conventions: momenta P_mu(x) traceless anti-Hermitian with kinetic energy K = -sum tr(P^2);
// every force Pi satisfies dS/deps = tr(T Pi) for U -> exp(eps T) U, so Hamilton's equations of
// H = K + S are dU/dt = P U and dP/dt = Pi / 2.  One leapfrog step: P += eps/4 Pi, U <- exp(eps P) U,
// P += eps/4 Pi.  One Omelyan (minimum-norm, second-order) step: P += lambda eps/2 Pi,
// U <- exp(eps/2 P) U, P += (1 - 2 lambda) eps/2 Pi, U <- exp(eps/2 P) U, P += lambda eps/2 Pi,
// lambda = 0.1931833275037836.  The force at the end of a step is the force at the start of the
// next (same links), so it is computed once.  With n_inner > 0 the outer steps kick with the
// pseudofermion forces alone and every drift of time h is n_inner steps of the same integrator
// over h under the gauge force (Sexton-Weingarten): the solves run on the outer scale only.
#include <algorithm>
#include <cmath>
#include <vector>

#include "engine.h"
#include "profile.h"

namespace odwf {

namespace {
constexpr double kOmelyanLambda = 0.1931833275037836;
}

int Engine::gauge_force(const double2* U, double beta, double* action, double2* F, cudaStream_t st) {
    int rc = 0;
    const size_t V = 2 * (size_t)vh();
    const size_t nb = gauge_force_blocks(V);
    double* part = (double*)get_ws("md.gpart", (nb + 1) * sizeof(double), &rc);
    if (rc) return rc;
    {
        ProfScope ps("md.gauge_force", (double)V * 4 * (144 + (F ? 144 : 0)), st);  // U in, F out
        ODWF_CK(launch_gauge_force(lat.dims, U, beta, F, part, part + nb, st));
    }
    if (action) {
        double retr = 0.0;
        ODWF_CK(cudaMemcpyAsync(&retr, part + nb, sizeof(double), cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
        *action = beta * (6.0 * (double)V - retr / 12.0);
    }
    return ODWF_OK;
}

int Engine::gauge_force_api(const void* U, double beta, double* action, void* force, cudaStream_t st) {
    if (!U || !action) return fail(ODWF_EINVAL, "odwf_gauge_force: null U or action");
    if (!std::isfinite(beta)) return fail(ODWF_EINVAL, "odwf_gauge_force: non-finite beta");
    int rc = 0;
    const size_t gbytes = (size_t)8 * vh() * 9 * sizeof(double2);  // 4 V links x 9 complex
    const double2* Ud = (const double2*)U;
    if (!is_device_ptr(U)) {
        void* d = get_ws("md.ustage", gbytes, &rc);
        if (rc) return rc;
        ODWF_CK(cudaMemcpyAsync(d, U, gbytes, cudaMemcpyHostToDevice, st));
        Ud = (const double2*)d;
    }
    double2* Fd = nullptr;
    const bool fdev = force && is_device_ptr(force);
    if (force) {
        Fd = fdev ? (double2*)force : (double2*)get_ws("md.fstage", gbytes, &rc);
        if (rc) return rc;
    }
    if ((rc = gauge_force(Ud, beta, action, Fd, st))) return rc;
    if (force && !fdev) ODWF_CK(cudaMemcpyAsync(force, Fd, gbytes, cudaMemcpyDeviceToHost, st));
    ODWF_CK(cudaStreamSynchronize(st));
    return ODWF_OK;
}

int Engine::md_trajectory(void* U, void* P, int nterms, const void* const* phi, const double* m1, const double* m2,
                          double beta, double tau, int nsteps, int integrator, int n_inner,
                          const odwf_solve_params* prm, double* energies, odwf_solve_stats* stats, cudaStream_t st) {
    if (stats) *stats = odwf_solve_stats{};
    if (!U || !P || !energies) return fail(ODWF_EINVAL, "odwf_md_trajectory: null U, P or energies");
    if (!is_device_ptr(U) || !is_device_ptr(P)) return fail(ODWF_EINVAL, "odwf_md_trajectory: U and P must be device memory");
    if (nterms < 0 || nterms > 16 || (nterms > 0 && (!phi || !m1 || !m2)))
        return fail(ODWF_EINVAL, "odwf_md_trajectory: 0 <= nterms <= 16 with phi, m1, m2");
    if (nsteps < 0 || !std::isfinite(tau) || !std::isfinite(beta))
        return fail(ODWF_EINVAL, "odwf_md_trajectory: bad nsteps, tau or beta");
    if (integrator != 0 && integrator != 1) return fail(ODWF_EINVAL, "odwf_md_trajectory: integrator 0 or 1");
    if (n_inner < 0 || n_inner > 1000) return fail(ODWF_EINVAL, "odwf_md_trajectory: 0 <= n_inner <= 1000");
    int rc = check_params(prm);
    if (rc) return rc;
    double2* Ud = (double2*)U;
    double2* Pd = (double2*)P;
    const size_t nl = (size_t)8 * vh();  // 4 V links
    const size_t n9 = nl * 9;
    double2* F = (double2*)get_ws("md.F", n9 * sizeof(double2), &rc);
    if (rc) return rc;
    double2* Ft = (double2*)get_ws("md.Ft", n9 * sizeof(double2), &rc);
    if (rc) return rc;
    double* ks = (double*)get_ws("md.ksum", (sumsq_partials() + 1) * sizeof(double), &rc);
    if (rc) return rc;
    const bool nested = n_inner > 0;
    double2* Fg = F;  // the gauge force: a share of F on one time scale, its own buffer on two
    if (nested) {
        Fg = (double2*)get_ws("md.Fg", n9 * sizeof(double2), &rc);
        if (rc) return rc;
    }
    const double lam = kOmelyanLambda;

    // H = K + S_g + sum S_pf at the current U, P; with_force also leaves the forces in F (all of
    // them on one time scale; the pseudofermion ones when nested, the gauge force then in Fg)
    auto evaluate = [&](bool with_force, double* H) -> int {
        int r = set_gauge(Ud, st);
        if (r) return r;
        double sg = 0.0;
        if ((r = gauge_force(Ud, beta, &sg, with_force ? Fg : nullptr, st))) return r;
        if (with_force && nested) ODWF_CK(cudaMemsetAsync(F, 0, n9 * sizeof(double2), st));
        double total = sg;
        for (int i = 0; i < nterms; ++i) {
            double spf = 0.0;
            odwf_solve_stats si{};
            r = pf_force(phi[i], m1[i], m2[i], prm, &spf, with_force ? (void*)Ft : nullptr, &si, st);
            if (stats) {  // sums over the trajectory's solves; the worst residual; the first failure
                stats->iters += si.iters;
                stats->n_reliable += si.n_reliable;
                stats->true_resid = std::max(stats->true_resid, si.true_resid);
                stats->time_ms += si.time_ms;
                if (stats->status == ODWF_OK) stats->status = si.status;
            }
            if (r) return r;
            if (with_force) ODWF_CK(launch_axpy(n9, F, Ft, 1.0, st));
            total += spf;
        }
        if (H) {
            ODWF_CK(launch_sumsq((const double*)Pd, 2 * n9, ks, ks + sumsq_partials(), st));
            double k = 0.0;
            ODWF_CK(cudaMemcpyAsync(&k, ks + sumsq_partials(), sizeof(double), cudaMemcpyDeviceToHost, st));
            ODWF_CK(cudaStreamSynchronize(st));
            *H = k + total;
        }
        return ODWF_OK;
    };
    auto force_only = [&]() -> int { return evaluate(true, nullptr); };
    auto kick = [&](const double2* Fk, double c) -> int {  // P += c Pi (Fk holds Pi at the current U)
        ODWF_CK(launch_axpy(n9, Pd, Fk, c, st));
        return ODWF_OK;
    };
    auto drift = [&](double a) -> int {  // U <- exp(a P) U
        ProfScope ps("md.link_update", (double)nl * 3 * 144, st);  // U in and out, P in
        ODWF_CK(launch_link_update(nl, Ud, Pd, a, st));
        return ODWF_OK;
    };
    auto gauge_only = [&]() -> int { return gauge_force(Ud, beta, nullptr, Fg, st); };
    // the outer drift over time h: plain, or n_inner integrator steps under the gauge force
    auto outer_drift = [&](double h) -> int {
        if (!nested) return drift(h);
        const double d = h / n_inner;
        int r = 0;
        for (int j = 0; j < n_inner && !r; ++j) {
            if (integrator == 0) {
                if (!r) r = kick(Fg, 0.25 * d);
                if (!r) r = drift(d);
                if (!r) r = gauge_only();
                if (!r) r = kick(Fg, 0.25 * d);
            } else {
                if (!r) r = kick(Fg, 0.5 * lam * d);
                if (!r) r = drift(0.5 * d);
                if (!r) r = gauge_only();
                if (!r) r = kick(Fg, 0.5 * (1.0 - 2.0 * lam) * d);
                if (!r) r = drift(0.5 * d);
                if (!r) r = gauge_only();
                if (!r) r = kick(Fg, 0.5 * lam * d);
            }
        }
        return r;
    };

    if ((rc = evaluate(true, &energies[0]))) return rc;  // H(0) and the force at the start
    const double eps = nsteps > 0 ? tau / nsteps : 0.0;
    for (int k = 0; k < nsteps && !rc; ++k) {
        if (integrator == 0) {
            if (!rc) rc = kick(F, 0.25 * eps);
            if (!rc) rc = outer_drift(eps);
            if (!rc) rc = force_only();
            if (!rc) rc = kick(F, 0.25 * eps);
        } else {
            if (!rc) rc = kick(F, 0.5 * lam * eps);
            if (!rc) rc = outer_drift(0.5 * eps);
            if (!rc) rc = force_only();
            if (!rc) rc = kick(F, 0.5 * (1.0 - 2.0 * lam) * eps);
            if (!rc) rc = outer_drift(0.5 * eps);
            if (!rc) rc = force_only();
            if (!rc) rc = kick(F, 0.5 * lam * eps);
        }
    }
    if (rc) return rc;
    return evaluate(false, &energies[1]);
}

}  // namespace odwf
