// extern "C" entry points declared in include/odwf.h.
#include <cmath>
#include <new>

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

extern "C" {

const char* odwf_last_error(void) { return odwf::last_error(); }

const char* odwf_version(void) { return "odwf-gb300 0.1 (sm_103a)"; }

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
    return h->e.set_gauge(U, (cudaStream_t)stream);
    GUARD_END
}

int odwf_apply(odwf_handle* h, void* out, const void* in, int mode, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply: null handle");
    return h->e.apply(out, in, mode, false, (cudaStream_t)stream);
    GUARD_END
}

int odwf_apply_dagger(odwf_handle* h, void* out, const void* in, int mode, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply_dagger: null handle");
    return h->e.apply(out, in, mode, true, (cudaStream_t)stream);
    GUARD_END
}

int odwf_apply_normal(odwf_handle* h, void* out, const void* in, int system, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply_normal: null handle");
    return h->e.apply_normal(out, in, system, (cudaStream_t)stream);
    GUARD_END
}

int odwf_apply_normal_prec(odwf_handle* h, void* out, const void* in, int prec, int link_recon, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply_normal_prec: null handle");
    return h->e.apply_low_normal(out, in, prec, link_recon, (cudaStream_t)stream);
    GUARD_END
}

int odwf_apply_m5(odwf_handle* h, void* out, const void* in, long n_sites, int op, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_apply_m5: null handle");
    return h->e.apply_m5(out, in, n_sites, op, (cudaStream_t)stream);
    GUARD_END
}

int odwf_cg_solve(odwf_handle* h, void* x, const void* b, const odwf_solve_params* params, odwf_solve_stats* stats,
                  void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_cg_solve: null handle");
    void* xs[1] = {x};
    const void* bs[1] = {b};
    return h->e.solve(1, xs, bs, nullptr, params, stats, (cudaStream_t)stream);
    GUARD_END
}

int odwf_cg_solve_batched(odwf_handle* h, int nsys, void* const* x, const void* const* b, const double* mq,
                          const odwf_solve_params* params, odwf_solve_stats* stats, void* stream) {
    GUARD_BEGIN
    if (!h) return fail(ODWF_EINVAL, "odwf_cg_solve_batched: null handle");
    if (params && params->system != ODWF_SYS_SCHUR_NORMAL)
        return fail(ODWF_EINVAL, "odwf_cg_solve_batched: SCHUR_NORMAL only");
    return h->e.solve(nsys, x, b, mq, params, stats, (cudaStream_t)stream);
    GUARD_END
}

}  // extern "C"
