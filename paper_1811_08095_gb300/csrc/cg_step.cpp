// odwf_mixed_cg_step: one iteration of the mixed-precision inner CG, run through exactly the
// launches the batched solver replays every iteration (the p update P, then the hops K1..K4 of
// kernels_mixed2.cu), with every field the iteration stores returned in the external layout.
// It exists so that each stored field can be compared with the FP64 oracle element by element.
#include <climits>
#include <cmath>
#include <cstring>

#include "batch_cg.h"

namespace odwf {

namespace {

int stage_field(Engine* E, const void* in, size_t bytes, const char* name, cudaStream_t st, const double2** out) {
    if (is_device_ptr(in)) {
        *out = (const double2*)in;
        return ODWF_OK;
    }
    int rc = 0;
    void* d = E->get_ws(name, bytes, &rc);
    if (rc) return rc;
    ODWF_CK(cudaMemcpyAsync(d, in, bytes, cudaMemcpyHostToDevice, st));
    *out = (const double2*)d;
    return ODWF_OK;
}

// unpack one internal half field of parity p to `dst` (host or device, [s][h][12] complex128)
int emit(Engine* E, Sp sp, const FieldRef& f, int p, void* dst, cudaStream_t st) {
    if (!dst) return ODWF_OK;
    const size_t eb = E->ext_bytes(ODWF_MODE_SCHUR_EVEN);
    const bool dev = is_device_ptr(dst);
    int rc = 0;
    double2* d = dev ? (double2*)dst : (double2*)E->get_ws("step.out", eb, &rc);
    if (rc) return rc;
    ODWF_CK(launch_unpack(sp, f, d, E->g, p, E->ns, 1, st));
    if (!dev) {
        ODWF_CK(cudaMemcpyAsync(dst, d, eb, cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
    }
    return ODWF_OK;
}

}  // namespace

int Engine::mixed_cg_step(int prec, int recon, int link_prec, double mq_step, const void* p_prev, const void* r, const void* x,
                          void* const* outs, odwf_cg_step_scalars* sc, cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "odwf_mixed_cg_step: gauge field not set");
    if (!p_prev || !r || !x || !outs || !sc) return fail(ODWF_EINVAL, "odwf_mixed_cg_step: null argument");
    if (prec != ODWF_F32 && prec != ODWF_F16 && prec != ODWF_BF16)
        return fail(ODWF_EINVAL, "odwf_mixed_cg_step: prec must be F32, F16 or BF16");
    if (recon == 0) recon = 12;
    if (recon != 12 && recon != 18) return fail(ODWF_EINVAL, "odwf_mixed_cg_step: link_recon must be 12 or 18");
    if (link_prec != 0 && link_prec != ODWF_F32 && link_prec != ODWF_F16)
        return fail(ODWF_EINVAL, "odwf_mixed_cg_step: link_prec must be 0, ODWF_F32 or ODWF_F16");
    if (link_prec == ODWF_F16 && recon != 12)
        return fail(ODWF_EINVAL, "odwf_mixed_cg_step: FP16 links are stored with 12 reals");
    if (!std::isfinite(mq_step)) return fail(ODWF_EINVAL, "odwf_mixed_cg_step: non-finite m_q");
    if (!(sc->rr > 0.0) || !std::isfinite(sc->rr) || !std::isfinite(sc->beta))
        return fail(ODWF_EINVAL, "odwf_mixed_cg_step: rr must be positive and finite, beta finite");
    const Sp low = (Sp)prec;
    if (!hop2_supported(ns, low, vh()))
        return fail(ODWF_EINVAL, "odwf_mixed_cg_step: the production mixed kernels need Ns = 8 or 16");
    odwf_solve_params prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.tol = 1e-10;
    prm.max_iter = INT_MAX;
    prm.prec = prec;
    prm.delta = 0.01;
    prm.system = ODWF_SYS_SCHUR_NORMAL;
    prm.link_recon = recon;
    prm.link_prec = link_prec;
    prm.update_arith = ODWF_UPDATES_F64;  // no reliable update runs here
    BatchCG bc;
    int rc = bc.init(this, 1, prm, st, 0);
    if (rc) return rc;
    if (!bc.v2) return fail(ODWF_EINVAL, "odwf_mixed_cg_step: production mixed kernels unavailable");
    const size_t eb = ext_bytes(ODWF_MODE_SCHUR_EVEN);
    const double2 *pd = nullptr, *rd = nullptr, *xd = nullptr;
    if ((rc = stage_field(this, p_prev, eb, "step.p", st, &pd)) || (rc = stage_field(this, r, eb, "step.r", st, &rd)) ||
        (rc = stage_field(this, x, eb, "step.x", st, &xd)))
        return rc;
    ODWF_CK(launch_pack(low, pd, bc.Pl.ref_sys(0), g, 0, ns, 1, st));
    ODWF_CK(launch_pack(Sp::F32, rd, bc.Rin.ref_sys(0), g, 0, ns, 1, st));
    ODWF_CK(launch_pack(Sp::F32, xd, bc.Xin.ref_sys(0), g, 0, ns, 1, st));
    if ((rc = emit(this, low, bc.Pl.ref_sys(0), 0, outs[0], st))) return rc;
    // a running system that never parks: no stopping threshold, no reliable-update trigger
    SysState s0;
    std::memset(&s0, 0, sizeof(s0));
    s0.rr = sc->rr;
    s0.beta = sc->beta;
    s0.r_max = std::sqrt(sc->rr);
    s0.bb = 1.0;
    s0.rscale = 1.0;
    s0.status = kRunning;
    s0.max_iter = INT_MAX;
    s0.reliable = 1;
    if ((rc = bc.set_state(0, s0, mq_step / (2.0 * m0), st))) return rc;
    if ((rc = bc.launch_v2_pupdate(1, 0, 1, 1, kRunning, st))) return rc;
    if ((rc = bc.launch_v2_hops(0, 1, st))) return rc;
    if ((rc = emit(this, low, bc.Pl.ref_sys(0), 0, outs[1], st)) ||
        (rc = emit(this, low, bc.Chil.ref_sys(0), 0, outs[2], st)) ||
        (rc = emit(this, low, bc.Tl.ref_sys(0), 1, outs[3], st)) ||
        (rc = emit(this, low, bc.Al.ref_sys(0), 0, outs[4], st)) ||
        (rc = emit(this, low, bc.Cl.ref_sys(0), 1, outs[5], st)) ||
        (rc = emit(this, Sp::F32, bc.Rin.ref_sys(0), 0, outs[6], st)) ||
        (rc = emit(this, Sp::F32, bc.Xin.ref_sys(0), 0, outs[7], st)))
        return rc;
    ODWF_CK(cudaMemcpyAsync(bc.st_host, bc.st, sizeof(SysState), cudaMemcpyDeviceToHost, st));
    ODWF_CK(cudaStreamSynchronize(st));
    const SysState& S = bc.st_host[0];
    sc->pAp = S.pAp;
    sc->alpha = S.alpha;
    sc->rr_new = S.rr_new;
    sc->status = S.status == kBreakdown ? ODWF_EBREAKDOWN : ODWF_OK;
    return ODWF_OK;
}

int Engine::time_kernel(int kind, int prec, int recon, int link_prec, int nsys, int reps, const void* fill,
                        odwf_kernel_prof* out, cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "odwf_time_kernel: gauge field not set");
    if (!fill || !out) return fail(ODWF_EINVAL, "odwf_time_kernel: null argument");
    if (kind < 1 || kind > 5) return fail(ODWF_EINVAL, "odwf_time_kernel: kind must be 1..5");
    if (nsys < 1 || nsys > 64 || reps < 1) return fail(ODWF_EINVAL, "odwf_time_kernel: need 1 <= nsys <= 64, reps >= 1");
    if (prec != ODWF_F32 && prec != ODWF_F16 && prec != ODWF_BF16)
        return fail(ODWF_EINVAL, "odwf_time_kernel: prec must be F32, F16 or BF16");
    if (recon == 0) recon = 12;
    odwf_solve_params prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.tol = 1e-10;
    prm.max_iter = INT_MAX;
    prm.prec = prec;
    prm.delta = 0.01;
    prm.link_recon = recon;
    prm.link_prec = link_prec;
    prm.update_arith = ODWF_UPDATES_F64;  // no reliable update runs here
    BatchCG bc;
    int rc = bc.init(this, nsys, prm, st, 0);
    if (rc) return rc;
    if (!bc.v2) return fail(ODWF_EINVAL, "odwf_time_kernel: the production mixed kernels need Ns = 8 or 16");
    const double2* fd = nullptr;
    if ((rc = stage_field(this, fill, ext_bytes(ODWF_MODE_SCHUR_EVEN), "step.p", st, &fd))) return rc;
    const Sp low = (Sp)prec;
    SysState s0;
    std::memset(&s0, 0, sizeof(s0));
    s0.rr = 1.0;
    s0.beta = 0.5;
    s0.alpha = 0.1;
    s0.r_max = 1.0;
    s0.bb = 1.0;
    s0.rscale = 1.0;
    s0.status = kRunning;
    s0.max_iter = INT_MAX;
    s0.reliable = 1;
    for (int i = 0; i < nsys; ++i) {
        const HalfField* lows[5] = {&bc.Pl, &bc.Tl, &bc.Al, &bc.Cl, &bc.Chil};
        for (const HalfField* f : lows) ODWF_CK(launch_pack(low, fd, f->ref_sys(i), g, 0, ns, 1, st));
        ODWF_CK(launch_pack(Sp::F32, fd, bc.Rin.ref_sys(i), g, 0, ns, 1, st));
        ODWF_CK(launch_pack(Sp::F32, fd, bc.Xin.ref_sys(i), g, 0, ns, 1, st));
        if ((rc = bc.set_state(i, s0, mq / (2.0 * m0), st))) return rc;
    }
    if ((rc = bc.launch_v2_kernel(kind, 0, nsys, st))) return rc;  // warm-up launch
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ODWF_CK(cudaEventCreate(&e0));
    ODWF_CK(cudaEventCreate(&e1));
    float ms = 0.f;
    cudaError_t ce = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && ce == cudaSuccess && !rc; ++r) rc = bc.launch_v2_kernel(kind, 0, nsys, st);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (ce != cudaSuccess) return cuda_fail(ce, "odwf_time_kernel: events");
    std::memset(out, 0, sizeof(*out));
    std::strncpy(out->name, bc.kname[kind - 1].c_str(), sizeof(out->name) - 1);
    out->launches = reps;
    out->system_launches = (int64_t)reps * nsys;
    out->total_ms = ms;
    out->bytes_per_system = bc.kbytes_sys[kind - 1];
    out->bytes_per_launch = bc.kbytes_launch[kind - 1];
    return ODWF_OK;
}

}  // namespace odwf
