// Slot-based batched CG (see batch_cg.h).
#include "batch_cg.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace odwf {

Lk link_format(const odwf_solve_params& prm) {
    if (prm.link_prec == ODWF_F16) return Lk::H12;
    return prm.link_recon == 18 ? Lk::F18 : Lk::F12;
}

void BatchCG::drop_graphs() {
    for (auto& kv : graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
}

BatchCG::~BatchCG() {
    drop_graphs();
    if (s_rel) cudaStreamSynchronize(s_rel);
    for (cudaEvent_t e : ev_rel)
        if (e) cudaEventDestroy(e);
    if (s_rel) cudaStreamDestroy(s_rel);
    if (ev_sync) cudaEventDestroy(ev_sync);
    if (st_host) cudaFreeHost(st_host);
}

template <>
HopParams<double> BatchCG::params<double>(int p_out) const {
    auto P = E->hop_params<double>(p_out, r_dev);
    P.st = st;
    P.partials = partials;
    P.part_stride = nblk;
    P.counters = counters;
    return P;
}

template <>
HopParams<ff> BatchCG::params<ff>(int p_out) const {
    auto P = E->hop_params<ff>(p_out, r_dev);
    P.st = st;
    P.partials = partials;
    P.part_stride = nblk;
    P.counters = counters;
    return P;
}

template <>
HopParams<float> BatchCG::params<float>(int p_out) const {
    auto P = E->hop_params<float>(p_out, r_dev);
    P.links = v2 ? E->links_site[(int)lk] : E->links_of(lk);
    P.st = st;
    P.partials = partials;
    P.part_stride = nblk;
    P.counters = counters;
    return P;
}

int BatchCG::init(Engine* e, int capacity, const odwf_solve_params& prm, cudaStream_t s, int update_prio_drop) {
    E = e;
    cap = capacity;
    mixed = prm.prec != ODWF_F64;
    low = (Sp)prm.prec;
    // float-float updates unless FP64 is asked for: on this part the float-float hops take about
    // 1.0-1.3 ms per system on 16^3x32x16 against 2.7-4.2 ms for the FP64 ones, also in batches
    // where the FP64 updates would overlap the other systems' FP32-bound iterations
    const bool ffu = prm.update_arith != ODWF_UPDATES_F64;
    fsp = mixed && ffu ? Sp::FF : Sp::F64;
    lk = link_format(prm);
    delta = prm.delta > 0 ? prm.delta : 0.01;
    tol = prm.tol;
    max_iter = prm.max_iter;
    int rc = 0;
    const int nrb = mixed ? 1 : cap;  // mixed: R64 and B64 are shared by all systems
    if ((rc = E->alloc_half("cg.X64", fsp, cap, &X64)) || (rc = E->alloc_half("cg.R64", fsp, nrb, &R64)) ||
        (rc = E->alloc_half("cg.B64", fsp, nrb, &B64)))
        return rc;
    if (fsp == Sp::FF && (rc = E->ensure_links(Lk::FF18, s))) return rc;
    if (!mixed) {
        if ((rc = E->alloc_half("cg.P64", Sp::F64, cap, &P64)) || (rc = E->alloc_half("cg.T64", Sp::F64, cap, &T64)) ||
            (rc = E->alloc_half("cg.A64", Sp::F64, cap, &A64)) || (rc = E->alloc_half("cg.C64", Sp::F64, cap, &C64)))
            return rc;
    } else {
        const std::string tag = "cg.lo" + std::to_string((int)low);
        if ((rc = E->alloc_half("cg.Rin", Sp::F32, cap, &Rin)) || (rc = E->alloc_half("cg.Xin", Sp::F32, cap, &Xin)) ||
            (rc = E->alloc_half(tag + ".P", low, cap, &Pl)) || (rc = E->alloc_half(tag + ".T", low, cap, &Tl)) ||
            (rc = E->alloc_half(tag + ".A", low, cap, &Al)) || (rc = E->alloc_half(tag + ".C", low, cap, &Cl)) ||
            (rc = E->alloc_half("cg.A1", fsp, 1, &A1)) || (rc = E->alloc_half("cg.C1", fsp, 1, &C1)))
            return rc;
        if ((rc = E->ensure_links(lk, s))) return rc;
        v2 = hop2_supported(E->ns, low, E->vh());
        if (lk == Lk::H12 && !v2) return fail(ODWF_EINVAL, "solve: FP16 links need Ns = 8 or 16");
        if (v2 && (rc = E->alloc_half(tag + ".X", low, cap, &Chil))) return rc;
        if (v2 && (rc = E->ensure_site_links(lk, s))) return rc;
    }
    st = (SysState*)E->get_ws("cg.state", sizeof(SysState) * cap, &rc);
    if (rc) return rc;
    r_dev = (double*)E->get_ws("cg.r", sizeof(double) * cap, &rc);
    if (rc) return rc;
    // one partial per block of a reducing launch and system: sized for the smallest reducing
    // block (64 threads, one 5D site each), so every kernel's grid fits
    nblk = blocks_for(E->sites5(), kMinReduceBlock);
    partials = (double*)E->get_ws("cg.partials", sizeof(double) * (size_t)nblk * cap, &rc);
    if (rc) return rc;
    counters = (unsigned*)E->get_ws("cg.counters", sizeof(unsigned) * cap, &rc);
    if (rc) return rc;
    ODWF_CK(cudaMemsetAsync(counters, 0, sizeof(unsigned) * cap, s));
    // pinned: state mirror [cap], initial-state staging [cap], r staging [cap]
    if (cudaMallocHost(&st_host, 2 * sizeof(SysState) * cap + sizeof(double) * cap) != cudaSuccess) {
        cudaGetLastError();
        st_host = nullptr;
        return fail(ODWF_ENOMEM, "pinned host allocation failed");
    }
    std::memset(st_host, 0, sizeof(SysState) * cap);
    for (int i = 0; i < cap; ++i) st_host[i].status = kIdle;
    ODWF_CK(cudaMemcpyAsync(st, st_host, sizeof(SysState) * cap, cudaMemcpyHostToDevice, s));
    ODWF_CK(cudaStreamSynchronize(s));
    n_reliable.assign(cap, 0);
    upd.assign(cap, 0);
    int prio = 0, least = 0, greatest = 0;
    ODWF_CK(cudaStreamGetPriority(s, &prio));
    ODWF_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    ODWF_CK(cudaStreamCreateWithPriority(&s_rel, cudaStreamNonBlocking, std::min(least, prio + update_prio_drop)));
    ODWF_CK(cudaEventCreateWithFlags(&ev_sync, cudaEventDisableTiming));
    bsrc.assign(cap, nullptr);
    ev_rel.assign(cap, nullptr);
    for (int i = 0; i < cap; ++i) ODWF_CK(cudaEventCreateWithFlags(&ev_rel[i], cudaEventDisableTiming));
    active.assign(cap, 0);
    mq.assign(cap, 0.0);
    slot_tol.assign(cap, tol);
    // profiler classes with their algorithmic bytes (each field read or written once)
    const double n5 = (double)E->sites5();
    const double sp = !mixed ? 192.0 : (low == Sp::F32 ? 96.0 : 52.0);  // FP16/BF16: 48 + 4-byte scale
    const double acc = mixed ? 96.0 : 192.0;                              // r, x
    const double links = 8.0 * (double)E->vh() * (!mixed ? 144.0 : lk == Lk::F12 ? 48.0 : lk == Lk::H12 ? 24.0 : 72.0);
    const char* lowname[] = {"f64", "f32", "f16", "bf16"};
    const std::string pre = !mixed ? std::string("f64") :
        std::string("mixed.") + lowname[(int)low] + (lk == Lk::F12 ? ".l12" : lk == Lk::H12 ? ".lh12" : ".l18");
    if (v2) {
        const std::string p2 = pre + ".v2";
        const char* kn[5] = {".K1_chi_minv", ".K2_schur_norm_mdinv", ".K3_dag_minvdag", ".K4_normal_cg", ".P_update_chi"};
        const double ksys[5] = {n5 * 2 * sp, n5 * 3 * sp, n5 * 2 * sp, n5 * (3 * sp + 4 * acc), n5 * (acc + 3 * sp)};
        for (int k = 0; k < 5; ++k) {
            kname[k] = p2 + kn[k];
            kbytes_sys[k] = ksys[k];
            kbytes_launch[k] = k < 4 ? links : 0.0;
            pcls[k] = prof_class(kname[k], kbytes_sys[k], kbytes_launch[k]);
        }
    } else {
    pcls[0] = prof_class(pre + ".K1_minv", n5 * 2 * sp, links);
    pcls[1] = prof_class(pre + ".K2_schur_norm_mdinv", n5 * 3 * sp, links);
    pcls[2] = prof_class(pre + ".K3_dag_minvdag", n5 * 2 * sp, links);
    pcls[3] = prof_class(pre + ".K4_normal_cg", n5 * (3 * sp + 4 * acc), links);
    pcls[4] = prof_class(pre + ".P_update", n5 * (acc + 2 * sp), 0.0);
    }
    const double l64 = 8.0 * (double)E->vh() * 144.0;
    const std::string rn = fsp == Sp::FF ? "ff.reliable." : "f64.reliable.";
    pcls_rel[0] = prof_class(rn + "K1_minv", n5 * 2 * 192.0, l64);
    pcls_rel[1] = prof_class(rn + "K2_schur_mdinv", n5 * 3 * 192.0, l64);
    pcls_rel[2] = prof_class(rn + "K3_dag_minvdag", n5 * 2 * 192.0, l64);
    pcls_rel[3] = prof_class(rn + "K4_resid", n5 * 4 * 192.0, l64);
    return ODWF_OK;
}

int BatchCG::admit(int slot, const double2* b_ext, double mq_slot, cudaStream_t s, double tol_slot,
                   int max_iter_slot) {
    NvtxRange nv_("odwf.cg.admit");
    if (slot < 0 || slot >= cap) return fail(ODWF_EINVAL, "admit: bad slot");
    mq[slot] = mq_slot;
    const size_t eb = E->sites5() * 12 * sizeof(double2);
    const double2* bd = b_ext;
    if (!is_device_ptr(b_ext)) {
        // mixed: one copy per slot (read again at every update); FP64: packed at once, one buffer
        int rc = 0;
        bstage = (double2*)E->get_ws("cg.bstage", eb * (mixed ? cap : 1), &rc);
        if (rc) return rc;
        double2* dst = (double2*)((char*)bstage + eb * (mixed ? slot : 0));
        ODWF_CK(cudaMemcpyAsync(dst, b_ext, eb, cudaMemcpyHostToDevice, s));
        bd = dst;
    }
    if (!mixed) {
        ODWF_CK(launch_pack(Sp::F64, bd, B64.ref_sys(slot), E->g, 0, E->ns, 1, s));
        return admit_internal(slot, s, tol_slot, max_iter_slot);
    }
    bsrc[slot] = bd;
    int rc = order_after(s_rel, s);  // the shared FP64 buffers are free
    if (!rc) rc = load_b(slot, s);
    if (!rc) rc = admit_internal(slot, s, tol_slot, max_iter_slot);
    if (!rc) rc = order_after(s, s_rel);  // later updates start after this admission's reads
    return rc;
}

int BatchCG::order_after(cudaStream_t first, cudaStream_t then) {
    ODWF_CK(cudaEventRecord(ev_sync, first));
    ODWF_CK(cudaStreamWaitEvent(then, ev_sync, 0));
    return ODWF_OK;
}

int BatchCG::load_b(int slot, cudaStream_t s) {
    if (mixed && bsrc[slot]) ODWF_CK(launch_pack(fsp, bsrc[slot], B64.ref_sys(0), E->g, 0, E->ns, 1, s));
    return ODWF_OK;
}

int BatchCG::release(int slot) {
    if (slot < 0 || slot >= cap) return fail(ODWF_EINVAL, "release: bad slot");
    active[slot] = 0;
    if (!bsrc.empty()) bsrc[slot] = nullptr;
    st_host[slot].status = kIdle;
    return ODWF_OK;
}

int BatchCG::cancel(int slot, cudaStream_t s) {
    if (slot < 0 || slot >= cap) return fail(ODWF_EINVAL, "cancel: bad slot");
    if (upd[slot]) {
        ODWF_CK(cudaStreamWaitEvent(s, ev_rel[slot], 0));
        upd[slot] = 0;
    }
    ODWF_CK(launch_state(st + slot, 1, 3, 0.0, s));
    return release(slot);
}

int BatchCG::admit_internal(int slot, cudaStream_t s, double tol_slot, int max_iter_slot) {
    const double tl = tol_slot > 0 ? tol_slot : tol;
    slot_tol[slot] = tl;
    const size_t n5 = E->sites5();
    const int ns = E->ns;
    // per-slot scalars: r = m_q / (2 m0) and a fresh state (written through pinned memory)
    double* rpin = reinterpret_cast<double*>(st_host + 2 * cap) + slot;
    *rpin = mq[slot] / (2.0 * E->m0);
    ODWF_CK(cudaMemcpyAsync(r_dev + slot, rpin, sizeof(double), cudaMemcpyHostToDevice, s));
    SysState init;
    std::memset(&init, 0, sizeof(init));
    init.status = kIdle;
    init.max_iter = max_iter_slot > 0 ? max_iter_slot : max_iter;
    init.delta = delta;
    init.reliable = mixed ? 1 : 0;
    SysState* stage = st_host + cap + slot;  // a slot is re-admitted only after finalize() synchronized
    *stage = init;
    ODWF_CK(cudaMemcpyAsync(st + slot, stage, sizeof(SysState), cudaMemcpyHostToDevice, s));
    // ||b||^2 -> state, then rr = bb, status running
    const FieldRef B = Bref();
    ODWF_CK(launch_vec(fsp, fsp, B, B, n5, ns, 3, 0.0, st, 0, 0, partials, counters, slot, 1, s, nblk));
    ODWF_CK(launch_state(st + slot, 1, 0, tl * tl, s));
    ODWF_CK(launch_vec(fsp, fsp, X64.ref(), X64.ref(), n5, ns, 5, 0.0, st, 0, 0, nullptr, nullptr, slot, 1, s));
    if (!mixed) {
        ODWF_CK(launch_vec(Sp::F64, Sp::F64, B, R64.ref(), n5, ns, 0, 0.0, st, 0, 0, nullptr, nullptr, slot, 1, s));
        ODWF_CK(launch_vec(Sp::F64, Sp::F64, B, P64.ref(), n5, ns, 0, 0.0, st, 0, 0, nullptr, nullptr, slot, 1, s));
    } else {
        ODWF_CK(launch_vec(fsp, Sp::F32, B, Rin.ref(), n5, ns, 6, 0.0, st, 0, 0, nullptr, nullptr, slot, 1, s));
        ODWF_CK(launch_vec(Sp::F32, Sp::F32, Xin.ref(), Xin.ref(), n5, ns, 5, 0.0, st, 0, 0, nullptr, nullptr, slot, 1, s));
        if (v2) {
            ODWF_CK(launch_p_update2(low, ns, Rin.ref(), Pl.ref(), Chil.ref(), E->vh(), 0, E->cf32, r_dev, st, 0, 0,
                                     slot, 1, nullptr, s));
        } else {
            ODWF_CK(launch_vec(fsp, low, B, Pl.ref(), n5, ns, 6, 0.0, st, 0, 0, nullptr, nullptr, slot, 1, s));
        }
    }
    active[slot] = 1;
    n_reliable[slot] = 0;
    st_host[slot].status = kRunning;  // host view until the next poll
    return ODWF_OK;
}

int BatchCG::run_iterations(int k, cudaStream_t s) {
    NvtxRange nv_("odwf.cg.iterations");
    int lo = cap, hi = -1;
    for (int i = 0; i < cap; ++i)
        if (active[i] && slot_running(i)) {
            lo = std::min(lo, i);
            hi = std::max(hi, i);
        }
    if (hi < 0) return ODWF_OK;
    const int n = hi - lo + 1;
    // direct launches while profiling (per-launch events), on the default streams (not
    // capturable), or when ODWF_GRAPHS=0 is set in the environment
    static const bool graphs_on = [] {
        const char* v = std::getenv("ODWF_GRAPHS");
        return !(v && v[0] == '0');
    }();
    if (!graphs_on || prof_enabled() || s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
        return launch_iterations(k, lo, n, s);
    const unsigned long long key = ((unsigned long long)lo << 40) | ((unsigned long long)n << 20) | (unsigned)k;
    auto it = graphs.find(key);
    if (it == graphs.end()) {
        if (graphs.size() >= 32) drop_graphs();
        const long long c0 = launch_count();
        ODWF_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int rc = launch_iterations(k, lo, n, s);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        GraphEntry e;
        e.kernels = launch_count() - c0;
        note_launches(-e.kernels);  // captured, not launched
        if (rc || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : cuda_fail(ce, "cudaStreamEndCapture(CG iterations)");
        }
        const cudaError_t ie = cudaGraphInstantiate(&e.exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate(CG iterations)");
        it = graphs.emplace(key, e).first;
    }
    ODWF_CK(cudaGraphLaunch(it->second.exec, s));
    note_launches(it->second.kernels);
    return ODWF_OK;
}

int BatchCG::launch_iterations(int k, int lo, int n, cudaStream_t s) {
    const size_t n5 = E->sites5();
    for (int it = 0; it < k; ++it) {
        if (!mixed) {
            // as in the reliable update: the non-dagger hops read chi = B psi, shifted once per
            // site into C64 (free until the third hop writes it)
            ODWF_CK(launch_m5_f64(P64.ref(), C64.ref(), E->vh(), E->ns, r_dev, lo, n, 4, E->cf64, s, st, kRunning));
            auto P = params<double>(1);
            P.gate = 1;
            P.need_status = kRunning;
            P.sys_base = lo;
            P.preshifted = 1;
            P.in = C64.ref();
            P.out = T64.ref();
            { auto pb_ = prof_begin(pcls[0], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_f64(P, Epi::MINV, n, s)); prof_end(pb_, s); P.prof_count = nullptr; }
            ODWF_CK(launch_m5_f64(T64.ref(), C64.ref(), E->vh(), E->ns, r_dev, lo, n, 4, E->cf64, s, st, kRunning));
            P.p_out = 0;
            P.in = C64.ref();
            P.z = P64.ref();
            P.out = A64.ref();
            { auto pb_ = prof_begin(pcls[1], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_f64(P, Epi::SCHUR_NORM_MDINV, n, s)); prof_end(pb_, s); P.prof_count = nullptr; }
            P.preshifted = 0;
            P.p_out = 1;
            P.in = A64.ref();
            P.z = FieldRef{};
            P.out = C64.ref();
            { auto pb_ = prof_begin(pcls[2], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_f64(P, Epi::D_MINVDAG, n, s)); prof_end(pb_, s); P.prof_count = nullptr; }
            P.p_out = 0;
            P.in = C64.ref();
            P.z = A64.ref();
            P.out = FieldRef{};
            P.cg_r = R64.ref();
            P.cg_x = X64.ref();
            P.cg_p = P64.ref();
            { auto pb_ = prof_begin(pcls[3], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_f64(P, Epi::D_NORMAL_CG, n, s)); prof_end(pb_, s); P.prof_count = nullptr; }
            {
                auto pb_ = prof_begin(pcls[4], s);
                set_vec_prof(pb_.dev_count);
                cudaError_t e_ = launch_vec(Sp::F64, Sp::F64, R64.ref(), P64.ref(), n5, E->ns, 1, 0.0, st, 1, kRunning,
                                            nullptr, nullptr, lo, n, s);
                set_vec_prof(nullptr);
                prof_end(pb_, s);
                ODWF_CK(e_);
            }
        } else if (v2) {
            int rc = launch_v2_hops(lo, n, s);
            if (!rc) rc = launch_v2_pupdate(1, lo, n, 1, kRunning, s);
            if (rc) return rc;
        } else {
            auto P = params<float>(1);
            P.gate = 1;
            P.need_status = kRunning;
            P.sys_base = lo;
            P.in = Pl.ref();
            P.out = Tl.ref();
            { auto pb_ = prof_begin(pcls[0], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_mixed(P, Epi::MINV, low, lk, n, s)); prof_end(pb_, s); P.prof_count = nullptr; }
            P.p_out = 0;
            P.in = Tl.ref();
            P.z = Pl.ref();
            P.out = Al.ref();
            { auto pb_ = prof_begin(pcls[1], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_mixed(P, Epi::SCHUR_NORM_MDINV, low, lk, n, s)); prof_end(pb_, s); P.prof_count = nullptr; }
            P.p_out = 1;
            P.in = Al.ref();
            P.z = FieldRef{};
            P.out = Cl.ref();
            { auto pb_ = prof_begin(pcls[2], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_mixed(P, Epi::D_MINVDAG, low, lk, n, s)); prof_end(pb_, s); P.prof_count = nullptr; }
            P.p_out = 0;
            P.in = Cl.ref();
            P.z = Al.ref();
            P.out = FieldRef{};
            P.cg_r = Rin.ref();
            P.cg_x = Xin.ref();
            P.cg_p = Pl.ref();
            { auto pb_ = prof_begin(pcls[3], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_mixed(P, Epi::D_NORMAL_CG, low, lk, n, s)); prof_end(pb_, s); P.prof_count = nullptr; }
            {
                auto pb_ = prof_begin(pcls[4], s);
                set_vec_prof(pb_.dev_count);
                cudaError_t e_ = launch_vec(Sp::F32, low, Rin.ref(), Pl.ref(), n5, E->ns, 1, 0.0, st, 1, kRunning,
                                            nullptr, nullptr, lo, n, s);
                set_vec_prof(nullptr);
                prof_end(pb_, s);
                ODWF_CK(e_);
            }
        }
    }
    return ODWF_OK;
}

// The four hops K1..K4 of one second-generation mixed iteration over slots lo..lo+n-1 (the
// non-dagger hops read chi = B psi): the launches the solver replays every iteration.
int BatchCG::launch_v2_kernel(int kind, int lo, int n, cudaStream_t s) {
    if (kind == 5) return launch_v2_pupdate(1, lo, n, 1, kRunning, s);
    auto P = params<float>(1);
    P.gate = 1;
    P.need_status = kRunning;
    P.sys_base = lo;
    const FieldRef ins[4] = {Chil.ref(), Tl.ref(), Al.ref(), Cl.ref()};
    const FieldRef outs[4] = {Tl.ref(), Al.ref(), Cl.ref(), FieldRef{}};
    const FieldRef zs[4] = {FieldRef{}, Pl.ref(), FieldRef{}, Al.ref()};
    const int k = kind - 1;
    P.p_out = (k & 1) ? 0 : 1;
    P.in = ins[k];
    P.out = outs[k];
    P.z = zs[k];
    if (k == 3) {
        P.cg_r = Rin.ref();
        P.cg_x = Xin.ref();
        P.cg_p = Pl.ref();
    }
    ODWF_CK(launch_hop_prod(P, kind, low, lk, n, s));
    return ODWF_OK;
}

int BatchCG::launch_v2_hops(int lo, int n, cudaStream_t s) {
    auto P = params<float>(1);
    P.gate = 1;
    P.need_status = kRunning;
    P.sys_base = lo;
    const FieldRef ins[4] = {Chil.ref(), Tl.ref(), Al.ref(), Cl.ref()};
    const FieldRef outs[4] = {Tl.ref(), Al.ref(), Cl.ref(), FieldRef{}};
    const FieldRef zs[4] = {FieldRef{}, Pl.ref(), FieldRef{}, Al.ref()};
    for (int k = 0; k < 4; ++k) {
        P.p_out = (k & 1) ? 0 : 1;
        P.in = ins[k];
        P.out = outs[k];
        P.z = zs[k];
        if (k == 3) {
            P.cg_r = Rin.ref();
            P.cg_x = Xin.ref();
            P.cg_p = Pl.ref();
        }
        auto pb_ = prof_begin(pcls[k], s);
        P.prof_count = pb_.dev_count;
        const cudaError_t e_ = launch_hop_prod(P, k + 1, low, lk, n, s);
        prof_end(pb_, s);
        P.prof_count = nullptr;
        ODWF_CK(e_);
    }
    return ODWF_OK;
}

// p = r + beta p (mode 1) or p = r (mode 0), chi_p = B p, for the slots whose status is `need`.
int BatchCG::launch_v2_pupdate(int mode, int lo, int n, int gate, int need, cudaStream_t s) {
    auto pb_ = prof_begin(pcls[4], s);
    const cudaError_t e_ = launch_p_update2(low, E->ns, Rin.ref(), Pl.ref(), Chil.ref(), E->vh(), mode, E->cf32, r_dev,
                                            st, gate, need, lo, n, pb_.dev_count, s);
    prof_end(pb_, s);
    ODWF_CK(e_);
    return ODWF_OK;
}

int BatchCG::set_state(int slot, const SysState& init, double r, cudaStream_t s) {
    if (slot < 0 || slot >= cap) return fail(ODWF_EINVAL, "set_state: bad slot");
    double* rpin = reinterpret_cast<double*>(st_host + 2 * cap) + slot;
    *rpin = r;
    ODWF_CK(cudaMemcpyAsync(r_dev + slot, rpin, sizeof(double), cudaMemcpyHostToDevice, s));
    SysState* stage = st_host + cap + slot;
    *stage = init;
    ODWF_CK(cudaMemcpyAsync(st + slot, stage, sizeof(SysState), cudaMemcpyHostToDevice, s));
    ODWF_CK(cudaStreamSynchronize(s));
    return ODWF_OK;
}

int BatchCG::poll(cudaStream_t s) {
    ODWF_CK(cudaMemcpyAsync(st_host, st, sizeof(SysState) * cap, cudaMemcpyDeviceToHost, s));
    ODWF_CK(cudaStreamSynchronize(s));
    prof_collect();
    return ODWF_OK;
}

bool BatchCG::slot_running(int i) const {
    const int stt = st_host[i].status;
    return stt == kRunning || stt == kNeedUpdate;
}

bool BatchCG::slot_finished(int i) const {
    const int stt = st_host[i].status;
    return active[i] && (stt == kDone || stt == kBreakdown || stt == kMaxIter);
}

int BatchCG::any_running() const {
    for (int i = 0; i < cap; ++i)
        if (active[i] && (slot_running(i) || upd[i])) return 1;
    return 0;
}

int BatchCG::resume(cudaStream_t s, bool block) {
    bool any_iterating = false;
    for (int i = 0; i < cap; ++i)
        if (active[i] && !upd[i] && st_host[i].status == kRunning) any_iterating = true;
    for (int i = 0; i < cap; ++i) {
        if (!upd[i]) continue;
        cudaError_t q = cudaEventQuery(ev_rel[i]);
        if (q == cudaErrorNotReady && block && !any_iterating) {
            ODWF_CK(cudaEventSynchronize(ev_rel[i]));  // nothing else to do: wait for this update
            q = cudaSuccess;
        }
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return cuda_fail(q, "cudaEventQuery(reliable update)");
        // the iteration stream waits for the update, then the slot rejoins (kRestarting -> kRunning)
        ODWF_CK(cudaStreamWaitEvent(s, ev_rel[i], 0));
        ODWF_CK(launch_state(st + i, 1, 2, 0.0, s));
        upd[i] = 0;
        st_host[i].status = kRunning;  // host view until the next poll
        any_iterating = true;
    }
    return ODWF_OK;
}

// R[slot] = B[slot] - S^dag S X[slot] in FP64, |R|^2 -> st[slot].sum (mixed: R and B are the
// shared buffers, B loaded with the slot's right-hand side)
// The reliable update's r = b - S^dag S x in float-float arithmetic (fields, links and
// coefficients as FP32 pairs): the same launch sequence as the FP64 one below.
int BatchCG::ff_residual(int slot, cudaStream_t s) {
    const FieldRef t = Rref(), a = A1.ref_shared(), c = C1.ref_shared();
    const size_t vh = E->vh();
    ODWF_CK(launch_m5_ff(X64.ref(), c, vh, E->ns, r_dev, slot, 1, 4, E->cfff, s));
    auto P = params<ff>(1);
    P.sys_base = slot;
    P.preshifted = 1;
    P.in = c;
    P.out = t;
    { auto pb_ = prof_begin(pcls_rel[0], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_ff(P, Epi::MINV, 1, s)); prof_end(pb_, s); P.prof_count = nullptr; }
    ODWF_CK(launch_m5_ff(t, c, vh, E->ns, r_dev, slot, 1, 4, E->cfff, s));
    P.p_out = 0;
    P.in = c;
    P.z = X64.ref();
    P.out = a;
    { auto pb_ = prof_begin(pcls_rel[1], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_ff(P, Epi::SCHUR_MDINV, 1, s)); prof_end(pb_, s); P.prof_count = nullptr; }
    P.preshifted = 0;
    P.p_out = 1;
    P.in = a;
    P.z = FieldRef{};
    P.out = c;
    { auto pb_ = prof_begin(pcls_rel[2], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_ff(P, Epi::D_MINVDAG, 1, s)); prof_end(pb_, s); P.prof_count = nullptr; }
    P.p_out = 0;
    P.in = c;
    P.z = a;
    P.b = Bref();
    P.out = Rref();
    { auto pb_ = prof_begin(pcls_rel[3], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_ff(P, Epi::D_NORMAL_RESID, 1, s)); prof_end(pb_, s); P.prof_count = nullptr; }
    return ODWF_OK;
}

int BatchCG::fp64_residual(int slot, cudaStream_t s) {
    if (fsp == Sp::FF) return ff_residual(slot, s);
    const HalfField& X = X64;
    FieldRef t, a, c;
    if (mixed) {
        t = Rref();  // R is rewritten by the last hop; it holds t = M^-1 H_oe x until then
        a = A1.ref_shared();
        c = C1.ref_shared();
    } else {
        t = T64.ref();
        a = A64.ref();
        c = C64.ref();
    }
    // The non-dagger hops read chi = B psi, shifted once per site beforehand into c (free
    // until the third hop writes it) instead of once per neighbour inside the hop.
    const size_t vh = E->vh();
    ODWF_CK(launch_m5_f64(X.ref(), c, vh, E->ns, r_dev, slot, 1, 4, E->cf64, s));
    auto P = params<double>(1);
    P.sys_base = slot;
    P.preshifted = 1;
    P.in = c;
    P.out = t;
    { auto pb_ = prof_begin(pcls_rel[0], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_f64(P, Epi::MINV, 1, s)); prof_end(pb_, s); P.prof_count = nullptr; }
    ODWF_CK(launch_m5_f64(t, c, vh, E->ns, r_dev, slot, 1, 4, E->cf64, s));
    P.p_out = 0;
    P.in = c;
    P.z = X.ref();
    P.out = a;
    { auto pb_ = prof_begin(pcls_rel[1], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_f64(P, Epi::SCHUR_MDINV, 1, s)); prof_end(pb_, s); P.prof_count = nullptr; }
    P.preshifted = 0;
    P.p_out = 1;
    P.in = a;
    P.z = FieldRef{};
    P.out = c;
    { auto pb_ = prof_begin(pcls_rel[2], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_f64(P, Epi::D_MINVDAG, 1, s)); prof_end(pb_, s); P.prof_count = nullptr; }
    P.p_out = 0;
    P.in = c;
    P.z = a;
    P.b = Bref();
    P.out = Rref();
    { auto pb_ = prof_begin(pcls_rel[3], s); P.prof_count = pb_.dev_count; ODWF_CK(launch_hop_f64(P, Epi::D_NORMAL_RESID, 1, s)); prof_end(pb_, s); P.prof_count = nullptr; }
    return ODWF_OK;
}

int BatchCG::service(cudaStream_t s) {
    NvtxRange nv_("odwf.cg.reliable_updates");
    const size_t n5 = E->sites5();
    for (int i = 0; i < cap; ++i) {
        if (!active[i] || upd[i] || st_host[i].status != kNeedUpdate) continue;
        // the update stream starts after this slot's last iteration on s
        ODWF_CK(cudaEventRecord(ev_rel[i], s));
        ODWF_CK(cudaStreamWaitEvent(s_rel, ev_rel[i], 0));
        cudaStream_t r = s_rel;
        if (mixed)  // X64 += rscale x_in, x_in = 0
            ODWF_CK(launch_vec(Sp::F32, fsp, Xin.ref(), X64.ref(), n5, E->ns, 7, 0.0, st, 0, 0, nullptr, nullptr,
                               i, 1, r));
        int rc = load_b(i, r);
        if (!rc) rc = fp64_residual(i, r);
        if (rc) return rc;
        ODWF_CK(launch_state(st + i, 1, 1, tol * tol, r));  // done / max-iter / kRestarting
        if (mixed) {
            ODWF_CK(launch_vec(fsp, Sp::F32, Rref(), Rin.ref(), n5, E->ns, 6, 0.0, st, 1, kRestarting, nullptr,
                               nullptr, i, 1, r));
            if (v2) {
                ODWF_CK(launch_p_update2(low, E->ns, Rin.ref(), Pl.ref(), Chil.ref(), E->vh(), 1, E->cf32, r_dev, st,
                                         1, kRestarting, i, 1, nullptr, r));
            } else {
                ODWF_CK(launch_vec(Sp::F32, low, Rin.ref(), Pl.ref(), n5, E->ns, 1, 0.0, st, 1, kRestarting, nullptr,
                                   nullptr, i, 1, r));
            }
        } else {
            ODWF_CK(launch_vec(Sp::F64, Sp::F64, R64.ref(), P64.ref(), n5, E->ns, 1, 0.0, st, 1, kRestarting, nullptr,
                               nullptr, i, 1, r));
        }
        ODWF_CK(cudaEventRecord(ev_rel[i], r));
        upd[i] = 1;
        n_reliable[i] += 1;
        st_host[i].status = kRestarting;  // host view until the next poll
    }
    return ODWF_OK;
}

int BatchCG::finalize(int slot, double2* x_ext, cudaStream_t s, double* true_resid) {
    NvtxRange nv_("odwf.cg.finalize");
    if (upd[slot]) {
        ODWF_CK(cudaStreamWaitEvent(s, ev_rel[slot], 0));
        upd[slot] = 0;
    }
    ODWF_CK(cudaMemcpyAsync(st_host + slot, st + slot, sizeof(SysState), cudaMemcpyDeviceToHost, s));
    ODWF_CK(cudaStreamSynchronize(s));
    const int stt = st_host[slot].status;
    if (stt != kDone && stt != kMaxIter) {
        // breakdown (or an unfinished slot): fold and recompute the true residual
        int rc = ODWF_OK;
        if (mixed) {
            ODWF_CK(launch_vec(Sp::F32, fsp, Xin.ref(), X64.ref(), E->sites5(), E->ns, 7, 0.0, st, 0, 0, nullptr,
                               nullptr, slot, 1, s));
            rc = order_after(s_rel, s);  // the shared FP64 buffers are free
            if (!rc) rc = load_b(slot, s);
        }
        if (!rc) rc = fp64_residual(slot, s);
        if (!rc && mixed) rc = order_after(s, s_rel);
        if (rc) return rc;
    }
    if (x_ext) ODWF_CK(launch_unpack(fsp, X64.ref_sys(slot), x_ext, E->g, 0, E->ns, 1, s));
    ODWF_CK(cudaMemcpyAsync(st_host + slot, st + slot, sizeof(SysState), cudaMemcpyDeviceToHost, s));
    ODWF_CK(cudaStreamSynchronize(s));
    const SysState& S = st_host[slot];
    if (true_resid) *true_resid = S.bb > 0 ? std::sqrt(S.sum / S.bb) : 0.0;
    return ODWF_OK;
}

}  // namespace odwf
