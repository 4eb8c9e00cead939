// Host side of the gradient flow (Sec. 2) and its observables (Sec. 3): the flow object, the
// stage loop and the extern "C" entry points declared in include/odwf_flow.h.
#include <cmath>
#include <initializer_list>
#include <new>
#include <string>

#include "../../include/odwf_flow.h"
#include "engine.h"
#include "flow.h"
#include "profile.h"

using odwf::cuda_fail;
using odwf::fail;
using odwf::flow::FlowGeom;
using odwf::flow::FlowObsDev;

struct odwf_flow {
    int device = 0;
    FlowGeom g{};
    float4* hi[2] = {nullptr, nullptr};  // first two rows of every link, [mu][3][V] float4 (hi + lo = the link)
    float4* lo[2] = {nullptr, nullptr};
    int cur = 0;
    float4* A = nullptr;  // six plaquette projections, [plane][2][V]
    float4* K = nullptr;  // Runge-Kutta carry, [mu][2][V]
    double* part_retr = nullptr;
    float* part_min = nullptr;
    double* part_e = nullptr;
    double* part_q = nullptr;
    FlowObsDev* obs_dev = nullptr;
    int obs_cap = 0;
    double2* stage = nullptr;  // host-pointer gauge copies: one direction at a time, kept until destroy
    bool gauge_set = false;
};

namespace {

#define FGUARD_BEGIN try {
#define FGUARD_END                                              \
    }                                                           \
    catch (const std::bad_alloc&) {                             \
        return fail(ODWF_ENOMEM, "host allocation failed");     \
    }                                                           \
    catch (...) {                                               \
        return fail(ODWF_EINVAL, "unexpected exception");       \
    }

#define FCK(call)                                               \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

int alloc(void** p, size_t bytes, const char* what) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ODWF_ENOMEM, std::string("odwf_flow_create: cannot allocate ") + what + " (" +
                                     std::to_string(bytes >> 20) + " MiB)");
    }
    return ODWF_OK;
}

void release(odwf_flow* f) {
    for (int b = 0; b < 2; ++b) {
        cudaFree(f->hi[b]);
        cudaFree(f->lo[b]);
    }
    cudaFree(f->A);
    cudaFree(f->K);
    cudaFree(f->part_retr);
    cudaFree(f->part_min);
    cudaFree(f->part_e);
    cudaFree(f->part_q);
    cudaFree(f->obs_dev);
    cudaFree(f->stage);
}

int on_device(const odwf_flow* f, const char* fn) {
    if (!f) return fail(ODWF_EINVAL, std::string(fn) + ": null flow object");
    int dev = -1;
    FCK(cudaGetDevice(&dev));
    if (dev != f->device)
        return fail(ODWF_EINVAL, std::string(fn) + ": the flow object belongs to GPU " + std::to_string(f->device) +
                                     ", but GPU " + std::to_string(dev) + " is current");
    return ODWF_OK;
}

int ensure_obs(odwf_flow* f, int n) {
    if (n <= f->obs_cap) return ODWF_OK;
    cudaFree(f->obs_dev);
    f->obs_dev = nullptr;
    f->obs_cap = 0;
    const int rc = alloc((void**)&f->obs_dev, sizeof(FlowObsDev) * (size_t)n, "observable records");
    if (rc) return rc;
    f->obs_cap = n;
    return ODWF_OK;
}

// Optional per-launch timing (odwf_profile_enable) with the kernel's algorithmic bytes per launch:
// each field read or written once (neighbour re-reads are not counted).
struct Timed {
    odwf::ProfSlot slot;
    cudaStream_t st;
    Timed(const char* name, double bytes, cudaStream_t s) : st(s) {
        const int cls = odwf::prof_enabled() ? odwf::prof_class(name, 0.0, bytes) : -1;
        slot = odwf::prof_begin(cls, s);
    }
    ~Timed() {
        odwf::prof_end(slot, st);
        odwf::note_launch();
    }
};

// bytes per site: links hi 192, lo 192 (two rows, per buffer), plaquette projections 192, carry 128
constexpr double kPlaqBytes = 192 + 192;
constexpr double kCloverBytes = 192 + 192;
double update_bytes(int stage) { return 192 + 2 * 192 + 2 * 192 + (stage > 0 ? 128 : 0) + (stage < 2 ? 128 : 0); }

int launch_plaq_t(odwf_flow* f, bool measure, cudaStream_t st) {
    Timed t(measure ? "flow.plaq_measure" : "flow.plaq", kPlaqBytes * f->g.V, st);
    FCK(odwf::flow::launch_plaq(f->g, f->hi[f->cur], f->A, f->part_retr, f->part_min, measure, st));
    return ODWF_OK;
}

// plaquettes (with the measurement reductions), clover densities and the record obs_dev[slot]
int measure_into(odwf_flow* f, double t, int slot, float* e_site, float* q_site, cudaStream_t st) {
    namespace fl = odwf::flow;
    odwf::NvtxRange r("flow measure");
    int rc = launch_plaq_t(f, true, st);
    if (rc) return rc;
    {
        Timed tm("flow.clover", kCloverBytes * f->g.V + (e_site ? 4.0 * f->g.V : 0) + (q_site ? 4.0 * f->g.V : 0), st);
        FCK(fl::launch_clover(f->g, f->hi[f->cur], f->A, f->part_e, f->part_q, e_site, q_site, st));
    }
    {
        Timed tm("flow.reduce", 12.0 * fl::plaq_blocks(f->g) + 16.0 * fl::clover_blocks(f->g), st);
        FCK(fl::launch_reduce(f->g, f->part_retr, f->part_min, f->part_e, f->part_q, t, f->obs_dev + slot, st));
    }
    return ODWF_OK;
}

int copy_obs(odwf_flow* f, odwf_flow_obs* obs, int n, cudaStream_t st) {
    static_assert(sizeof(odwf_flow_obs) == sizeof(FlowObsDev), "observable record layouts differ");
    FCK(cudaMemcpyAsync(obs, f->obs_dev, sizeof(FlowObsDev) * (size_t)n, cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    return ODWF_OK;
}

}  // namespace

extern "C" {

int odwf_flow_create(const int32_t dims[4], odwf_flow** out) {
    FGUARD_BEGIN
    if (!out || !dims) return fail(ODWF_EINVAL, "odwf_flow_create: null argument");
    *out = nullptr;
    size_t V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || dims[mu] > 4096)
            return fail(ODWF_EINVAL, "odwf_flow_create: every extent must be in [2, 4096]");
        V *= (size_t)dims[mu];
    }
    if (V > ((size_t)1 << 34)) return fail(ODWF_EINVAL, "odwf_flow_create: lattice too large");
    int device = 0;
    FCK(cudaGetDevice(&device));
    odwf_flow* f = new odwf_flow();
    f->device = device;
    FlowGeom& g = f->g;
    size_t stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.L[mu] = dims[mu];
        g.stride[mu] = stride;
        stride *= (size_t)dims[mu];
    }
    g.V = V;
    g.bt = dims[3] % 8 == 0 ? 8 : dims[3] % 4 == 0 ? 4 : dims[3] % 2 == 0 ? 2 : 1;
    const size_t nbp = odwf::flow::plaq_blocks(g), nbc = odwf::flow::clover_blocks(g);
    int rc = 0;
    for (int b = 0; b < 2 && !rc; ++b) {
        rc = alloc((void**)&f->hi[b], 12 * V * sizeof(float4), "links (hi)");
        if (!rc) rc = alloc((void**)&f->lo[b], 12 * V * sizeof(float4), "links (lo)");
    }
    if (!rc) rc = alloc((void**)&f->A, 12 * V * sizeof(float4), "plaquette projections");
    if (!rc) rc = alloc((void**)&f->K, 8 * V * sizeof(float4), "Runge-Kutta carry");
    if (!rc) rc = alloc((void**)&f->part_retr, nbp * sizeof(double), "partial sums");
    if (!rc) rc = alloc((void**)&f->part_min, nbp * sizeof(float), "partial minima");
    if (!rc) rc = alloc((void**)&f->part_e, nbc * sizeof(double), "partial sums");
    if (!rc) rc = alloc((void**)&f->part_q, nbc * sizeof(double), "partial sums");
    if (!rc) rc = ensure_obs(f, 64);
    if (rc) {
        release(f);
        delete f;
        return rc;
    }
    *out = f;
    return ODWF_OK;
    FGUARD_END
}

int odwf_flow_destroy(odwf_flow* f) {
    FGUARD_BEGIN
    if (!f) return ODWF_OK;
    release(f);
    delete f;
    return ODWF_OK;
    FGUARD_END
}

int odwf_flow_set_gauge(odwf_flow* f, const void* U, void* stream) {
    FGUARD_BEGIN
    int rc = on_device(f, "odwf_flow_set_gauge");
    if (rc) return rc;
    if (!U) return fail(ODWF_EINVAL, "odwf_flow_set_gauge: null U");
    rc = odwf::check_ptr_device(U, f->device, "odwf_flow_set_gauge");
    if (rc) return rc;
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t V = f->g.V;
    const size_t slab = 9 * V * sizeof(double2);  // one direction
    const bool dev = odwf::is_device_ptr(U);
    if (!dev && !f->stage) {
        rc = alloc((void**)&f->stage, slab, "gauge staging");
        if (rc) return rc;
    }
    double2* stage = dev ? nullptr : f->stage;
    for (int mu = 0; mu < 4 && !rc; ++mu) {
        const double2* src = (const double2*)U + (size_t)mu * 9 * V;
        if (!dev) {
            cudaError_t e = cudaMemcpyAsync(stage, src, slab, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync (gauge)");
            src = stage;
        }
        if (!rc) {
            cudaError_t e = odwf::flow::launch_split(src, f->hi[f->cur], f->lo[f->cur], V, mu, st);
            odwf::note_launch();
            if (e != cudaSuccess) rc = cuda_fail(e, "flow split kernel");
        }
    }
    if (stage) {  // the caller may reuse its host buffer on return
        const cudaError_t e = cudaStreamSynchronize(st);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (!rc) f->gauge_set = true;
    return rc;
    FGUARD_END
}

int odwf_flow_get_gauge(odwf_flow* f, void* U, void* stream) {
    FGUARD_BEGIN
    int rc = on_device(f, "odwf_flow_get_gauge");
    if (rc) return rc;
    if (!U) return fail(ODWF_EINVAL, "odwf_flow_get_gauge: null U");
    if (!f->gauge_set) return fail(ODWF_EINVAL, "odwf_flow_get_gauge: gauge field not set");
    rc = odwf::check_ptr_device(U, f->device, "odwf_flow_get_gauge");
    if (rc) return rc;
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t V = f->g.V;
    const size_t slab = 9 * V * sizeof(double2);
    const bool dev = odwf::is_device_ptr(U);
    if (!dev && !f->stage) {
        rc = alloc((void**)&f->stage, slab, "gauge staging");
        if (rc) return rc;
    }
    double2* stage = dev ? nullptr : f->stage;
    for (int mu = 0; mu < 4 && !rc; ++mu) {
        double2* dst = dev ? (double2*)U + (size_t)mu * 9 * V : stage;
        cudaError_t e = odwf::flow::launch_join(f->hi[f->cur], f->lo[f->cur], dst, V, mu, st);
        odwf::note_launch();
        if (e != cudaSuccess) rc = cuda_fail(e, "flow join kernel");
        if (!rc && !dev) {
            e = cudaMemcpyAsync((double2*)U + (size_t)mu * 9 * V, stage, slab, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync (gauge)");
        }
    }
    return rc;
    FGUARD_END
}

int odwf_flow_measure(odwf_flow* f, double t, odwf_flow_obs* obs, float* e_site, float* q_site, void* stream) {
    FGUARD_BEGIN
    int rc = on_device(f, "odwf_flow_measure");
    if (rc) return rc;
    if (!obs) return fail(ODWF_EINVAL, "odwf_flow_measure: null obs");
    if (!f->gauge_set) return fail(ODWF_EINVAL, "odwf_flow_measure: gauge field not set");
    for (const void* p : {(const void*)e_site, (const void*)q_site}) {
        rc = odwf::check_ptr_device(p, f->device, "odwf_flow_measure");
        if (rc) return rc;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t V = f->g.V;
    const bool host_e = e_site && !odwf::is_device_ptr(e_site);
    const bool host_q = q_site && !odwf::is_device_ptr(q_site);
    float* stage = nullptr;
    if (host_e || host_q) {
        rc = alloc((void**)&stage, 2 * V * sizeof(float), "density staging");
        if (rc) return rc;
    }
    float* ed = host_e ? stage : e_site;
    float* qd = host_q ? stage + V : q_site;
    rc = measure_into(f, t, 0, ed, qd, st);
    if (!rc && host_e) {
        const cudaError_t e = cudaMemcpyAsync(e_site, ed, V * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync (densities)");
    }
    if (!rc && host_q) {
        const cudaError_t e = cudaMemcpyAsync(q_site, qd, V * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync (densities)");
    }
    if (!rc) rc = copy_obs(f, obs, 1, st);
    if (stage) {
        cudaStreamSynchronize(st);
        cudaFree(stage);
    }
    return rc;
    FGUARD_END
}

int odwf_flow_run(odwf_flow* f, double eps, int nsteps, int measure_every, double t_start, odwf_flow_obs* obs,
                  int max_obs, int* n_obs, void* stream) {
    FGUARD_BEGIN
    namespace fl = odwf::flow;
    int rc = on_device(f, "odwf_flow_run");
    if (rc) return rc;
    if (n_obs) *n_obs = 0;
    if (!f->gauge_set) return fail(ODWF_EINVAL, "odwf_flow_run: gauge field not set");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(ODWF_EINVAL, "odwf_flow_run: eps must be finite and > 0");
    if (nsteps < 0 || measure_every < 0) return fail(ODWF_EINVAL, "odwf_flow_run: negative nsteps or measure_every");
    int need = 0;
    if (measure_every > 0) {
        need = nsteps > 0 ? (nsteps - 1) / measure_every + 1 : 0;
        if (nsteps % measure_every == 0) need += 1;
        if (!obs || !n_obs) return fail(ODWF_EINVAL, "odwf_flow_run: measuring needs obs and n_obs");
        if (need > max_obs)
            return fail(ODWF_EINVAL, "odwf_flow_run: " + std::to_string(need) + " measurements need more than max_obs = " +
                                         std::to_string(max_obs) + " records");
        rc = ensure_obs(f, need);
        if (rc) return rc;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const float fe = (float)eps;
    int m = 0;
    odwf::NvtxRange r("flow run");
    for (int k = 0; k < nsteps; ++k) {
        const bool meas = measure_every > 0 && k % measure_every == 0;
        for (int stage = 0; stage < 3; ++stage) {
            const int nxt = f->cur ^ 1;
            if (stage == 0 && meas) {
                rc = measure_into(f, t_start + k * eps, m++, nullptr, nullptr, st);  // also the stage's plaquettes
                if (rc) return rc;
            } else {
                rc = launch_plaq_t(f, false, st);
                if (rc) return rc;
            }
            {
                static const char* names[3] = {"flow.update_s0", "flow.update_s1", "flow.update_s2"};
                Timed tm(names[stage], update_bytes(stage) * f->g.V, st);
                FCK(fl::launch_update(f->g, stage, f->hi[f->cur], f->lo[f->cur], f->hi[nxt], f->lo[nxt], f->A, f->K,
                                      fe, st));
            }
            f->cur = nxt;
        }
    }
    if (measure_every > 0 && nsteps % measure_every == 0) {
        rc = measure_into(f, t_start + nsteps * eps, m++, nullptr, nullptr, st);
        if (rc) return rc;
    }
    if (m > 0) {
        rc = copy_obs(f, obs, m, st);
        if (rc) return rc;
        *n_obs = m;
    }
    return ODWF_OK;
    FGUARD_END
}

int odwf_flow_t0(const odwf_flow_obs* obs, int n, double target, double* t0) {
    FGUARD_BEGIN
    if (!obs || !t0 || n < 0) return fail(ODWF_EINVAL, "odwf_flow_t0: null argument");
    for (int i = 1; i < n; ++i) {
        const double f0 = obs[i - 1].t * obs[i - 1].t * obs[i - 1].e_clover - target;
        const double f1 = obs[i].t * obs[i].t * obs[i].e_clover - target;
        if (f0 < 0.0 && f1 >= 0.0) {
            *t0 = obs[i - 1].t + (obs[i].t - obs[i - 1].t) * (-f0) / (f1 - f0);
            return ODWF_OK;
        }
    }
    return fail(ODWF_ENOTFOUND, "odwf_flow_t0: t^2 E(t) does not reach the target");
    FGUARD_END
}

}  // extern "C"
