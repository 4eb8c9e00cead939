// extern "C" entry points declared in include/odwf.h.
#include <cmath>
#include <initializer_list>
#include <new>
#include <string>

#include "engine.h"

namespace odwf {
const char* last_error();
int zolotarev_omega(int Ns, double lmin, double lmax, int variant, double* omega, double* dz);
}  // namespace odwf

using odwf::fail;

#define GUARD_BEGIN try {
#define GUARD_END                                                   \
    }                                                               \
    catch (const std::bad_alloc&) {                                 \
        return fail(ODWF_ENOMEM, "host allocation failed");         \
    }                                                               \
    catch (...) {                                                   \
        return fail(ODWF_EINVAL, "unexpected exception");           \
    }

namespace {
// A handle's kernels run on the current device and use memory of the device it was created
// on: both must agree, and every device pointer argument must belong to that device.
int on_handle_device(odwf_handle* h, const char* fn, std::initializer_list<const void*> ptrs) {
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return odwf::cuda_fail(e, "cudaGetDevice");
    if (dev != h->e.device)
        return fail(ODWF_EINVAL, std::string(fn) + ": the handle belongs to GPU " + std::to_string(h->e.device) +
                                     ", but GPU " + std::to_string(dev) + " is current");
    for (const void* p : ptrs) {
        const int rc = odwf::check_ptr_device(p, dev, fn);
        if (rc) return rc;
    }
    return ODWF_OK;
}
}  // namespace

// the call's status, or the debug build's bounds-check error when the call itself succeeded
#define WITH_BOUNDS(h, call, stream)                                      \
    do {                                                                  \
        const int rc0_ = (call);                                          \
        const int rb_ = (h)->e.bounds_status((cudaStream_t)(stream));     \
        return rb_ ? rb_ : rc0_;                                          \
    } while (0)

#define ON_DEVICE(h, fn, ...)                                   \
    do {                                                        \
        const int rc_ = on_handle_device(h, fn, {__VA_ARGS__}); \
        if (rc_) return rc_;                                    \
    } while (0)

extern "C" {

const char* odwf_last_error(void) { return odwf::last_error(); }

#ifdef ODWF_BOUNDS_CHECK
const char* odwf_version(void) { return "odwf-gb300 0.2 (sm_103a, bounds-checked)"; }
#else
const char* odwf_version(void) { return "odwf-gb300 0.2 (sm_103a)"; }
#endif

int odwf_zolotarev_omega(int Ns, double lmin, double lmax, int variant, double* omega_out, double* dz_out) {
    GUARD_BEGIN
    return odwf::zolotarev_omega(Ns, lmin, lmax, variant, omega_out, dz_out);
    GUARD_END
}

int odwf_create(const odwf_lattice* lat, int Ns, double m0, double mq, const double* omega, odwf_handle** out) {
    GUARD_BEGIN
    if (!out) return fail(ODWF_EINVAL, "odwf_create: null out");
    *out = nullptr;
    odwf_handle* h = new odwf_handle();
    const int rc = h->e.init(lat, Ns, m0, mq, omega);
    if (rc) {
        delete h;
        return rc;
    }
    *out = h;
    return ODWF_OK;
    GUARD_END
}

int odwf_destroy(odwf_handle* h) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_destroy: null handle");
    delete h;
    return ODWF_OK;
    GUARD_END
}

int odwf_set_gauge(odwf_handle* h, const void* U, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_set_gauge: null handle");
    ON_DEVICE(h, "odwf_set_gauge", U);
    return h->e.set_gauge(U, (cudaStream_t)stream);
    GUARD_END
}

int odwf_apply(odwf_handle* h, void* out, const void* in, int mode, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply: null handle");
    ON_DEVICE(h, "odwf_apply", out, in);
    WITH_BOUNDS(h, h->e.apply(out, in, mode, false, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_apply_dagger(odwf_handle* h, void* out, const void* in, int mode, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply_dagger: null handle");
    ON_DEVICE(h, "odwf_apply_dagger", out, in);
    WITH_BOUNDS(h, h->e.apply(out, in, mode, true, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_apply_normal(odwf_handle* h, void* out, const void* in, int system, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply_normal: null handle");
    ON_DEVICE(h, "odwf_apply_normal", out, in);
    WITH_BOUNDS(h, h->e.apply_normal(out, in, system, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_apply_normal_prec(odwf_handle* h, void* out, const void* in, int prec, int link_recon, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply_normal_prec: null handle");
    ON_DEVICE(h, "odwf_apply_normal_prec", out, in);
    WITH_BOUNDS(h, h->e.apply_low_normal(out, in, prec, link_recon, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_apply_m5(odwf_handle* h, void* out, const void* in, long n_sites, int op, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply_m5: null handle");
    ON_DEVICE(h, "odwf_apply_m5", out, in);
    return h->e.apply_m5(out, in, n_sites, op, (cudaStream_t)stream);
    GUARD_END
}

int odwf_mixed_cg_step(odwf_handle* h, int prec, int link_recon, int link_prec, double mq, const void* p_prev, const void* r,
                       const void* x, void* const* outs, odwf_cg_step_scalars* sc, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_mixed_cg_step: null handle");
    ON_DEVICE(h, "odwf_mixed_cg_step", p_prev, r, x);
    if (outs)
        for (int i = 0; i < 8; ++i) ON_DEVICE(h, "odwf_mixed_cg_step", outs[i]);
    WITH_BOUNDS(h, h->e.mixed_cg_step(prec, link_recon, link_prec, mq, p_prev, r, x, outs, sc, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_time_kernel(odwf_handle* h, int kind, int prec, int link_recon, int link_prec, int nsys, int reps,
                     const void* fill, odwf_kernel_prof* out, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_time_kernel: null handle");
    ON_DEVICE(h, "odwf_time_kernel", fill);
    return h->e.time_kernel(kind, prec, link_recon, link_prec, nsys, reps, fill, out, (cudaStream_t)stream);
    GUARD_END
}

int odwf_effective_solve(odwf_handle* h, void* x, const void* b, const odwf_solve_params* params,
                         odwf_solve_stats* stats, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_effective_solve: null handle");
    ON_DEVICE(h, "odwf_effective_solve", x, b);
    const int rc = odwf::check_params(params);
    if (rc) return rc;
    WITH_BOUNDS(h, h->e.effective_solve(x, b, params, stats, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_pf_force(odwf_handle* h, const void* phi, double m1, double m2, const odwf_solve_params* params,
                  double* action, void* force, odwf_solve_stats* stats, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_pf_force: null handle");
    ON_DEVICE(h, "odwf_pf_force", phi, force);
    WITH_BOUNDS(h, h->e.pf_force(phi, m1, m2, params, action, force, stats, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_pf_heatbath(odwf_handle* h, const void* eta, double m1, double m2, const odwf_solve_params* params,
                     void* phi, odwf_solve_stats* stats, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_pf_heatbath: null handle");
    ON_DEVICE(h, "odwf_pf_heatbath", eta, phi);
    WITH_BOUNDS(h, h->e.pf_heatbath(eta, m1, m2, params, phi, stats, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_gauge_force(odwf_handle* h, const void* U, double beta, double* action, void* force, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_gauge_force: null handle");
    ON_DEVICE(h, "odwf_gauge_force", U, force);
    WITH_BOUNDS(h, h->e.gauge_force_api(U, beta, action, force, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_md_trajectory(odwf_handle* h, void* U, void* P, int nterms, const void* const* phi, const double* m1,
                       const double* m2, double beta, double tau, int nsteps, int integrator, int n_inner,
                       const odwf_solve_params* params, double* energies, odwf_solve_stats* stats,
                       void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_md_trajectory: null handle");
    ON_DEVICE(h, "odwf_md_trajectory", U, P);
    for (int i = 0; phi && i < nterms && i < 16; ++i) ON_DEVICE(h, "odwf_md_trajectory", phi[i]);
    WITH_BOUNDS(h,
                h->e.md_trajectory(U, P, nterms, phi, m1, m2, beta, tau, nsteps, integrator, n_inner, params, energies,
                                   stats, (cudaStream_t)stream),
                stream);
    GUARD_END
}

int odwf_residual_mass(odwf_handle* h, const int32_t* site, const odwf_solve_params* params, double* mres,
                       double* corr, odwf_solve_stats* stats, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_residual_mass: null handle");
    ON_DEVICE(h, "odwf_residual_mass");
    const int rc = odwf::check_params(params);
    if (rc) return rc;
    WITH_BOUNDS(h, h->e.residual_mass(site, params, mres, corr, stats, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_cg_solve(odwf_handle* h, void* x, const void* b, const odwf_solve_params* params, odwf_solve_stats* stats,
                  void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_cg_solve: null handle");
    ON_DEVICE(h, "odwf_cg_solve", x, b);
    void* xs[1] = {x};
    const void* bs[1] = {b};
    WITH_BOUNDS(h, h->e.solve(1, xs, bs, nullptr, params, stats, (cudaStream_t)stream), stream);
    GUARD_END
}

int odwf_cg_solve_batched(odwf_handle* h, int nsys, void* const* x, const void* const* b, const double* mq,
                          const odwf_solve_params* params, odwf_solve_stats* stats, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_cg_solve_batched: null handle");
    if (x && b && nsys > 0)
        for (int i = 0; i < nsys; ++i) ON_DEVICE(h, "odwf_cg_solve_batched", x[i], b[i]);
    if (params && params->system != ODWF_SYS_SCHUR_NORMAL)
        return fail(ODWF_EINVAL, "odwf_cg_solve_batched: SCHUR_NORMAL only");
    WITH_BOUNDS(h, h->e.solve(nsys, x, b, mq, params, stats, (cudaStream_t)stream), stream);
    GUARD_END
}

}  // extern "C"
