// Host engine: handle set-up, gauge packing, FP64 operator applications and solves.
#include "engine.h"

#include <cmath>
#include <cstring>
#include <string>

#include "batch_cg.h"

namespace odwf {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
const char* last_error() { return g_err.c_str(); }
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ODWF_ENOMEM : ODWF_ECUDA;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_ptr_device(const void* p, int dev, const char* what) {
    if (!p) return ODWF_OK;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return ODWF_OK;  // not known to CUDA: host memory
    }
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return fail(ODWF_EINVAL, std::string(what) + ": pointer is device memory of GPU " + std::to_string(a.device) +
                                     ", but the call runs on GPU " + std::to_string(dev));
    return ODWF_OK;
}

Engine::~Engine() {
    for (auto& kv : ws)
        if (kv.second.p) cudaFree(kv.second.p);
    if (links_d18) cudaFree(links_d18);
    if (links_f18) cudaFree(links_f18);
    if (links_f12) cudaFree(links_f12);
    if (links_h12) cudaFree(links_h12);
    if (links_ff18) cudaFree(links_ff18);
    for (void* p : links_site)
        if (p) cudaFree(p);
    if (nbr) cudaFree(nbr);
    if (pinned) cudaFreeHost(pinned);
}

int Engine::init(const odwf_lattice* l, int Ns, double m0_, double mq_, const double* w) {
    if (!l || !w) return fail(ODWF_EINVAL, "odwf_create: null lattice or omega");
    for (int i = 0; i < 4; ++i)
        if (l->dims[i] < 2 || (l->dims[i] & 1))
            return fail(ODWF_EINVAL, "odwf_create: every lattice extent must be even and >= 2");
    if (Ns < 2 || Ns > kMaxNs || (Ns & (Ns - 1)))
        return fail(ODWF_EINVAL, "odwf_create: Ns must be 2, 4, 8, 16 or 32");
    const double V = (double)l->dims[0] * l->dims[1] * l->dims[2] * l->dims[3];
    if (V / 2 > 2147483647.0) return fail(ODWF_EINVAL, "odwf_create: lattice too large");
    if (!std::isfinite(m0_) || !std::isfinite(mq_)) return fail(ODWF_EINVAL, "odwf_create: non-finite mass");
    lat = *l;
    for (int i = 0; i < 4; ++i) g.L[i] = l->dims[i];
    g.Lxh = l->dims[0] / 2;
    g.Vh = (int)(V / 2);
    g.tbc = l->t_antiperiodic ? 1 : 0;
    ns = Ns;
    lg_ns = lg2(Ns);
    m0 = m0_;
    mq = mq_;
    omega.assign(w, w + Ns);
    const double a = 4.0 - m0;
    std::memset(&cf64, 0, sizeof(cf64));
    std::memset(&cf32, 0, sizeof(cf32));
    for (int s = 0; s < Ns; ++s) {
        if (!std::isfinite(w[s])) return fail(ODWF_EINVAL, "odwf_create: non-finite omega");
        const double rho = w[s], sig = w[s];  // c = 1, d = 0
        cf64.rho[s] = rho;
        cf64.sigma[s] = sig;
        cf64.d[s] = a * rho + 1.0;
        cf64.e[s] = a * sig - 1.0;
        if (cf64.d[s] == 0.0) return fail(ODWF_EINVAL, "odwf_create: singular diagonal (4-m0) omega_s + 1 = 0");
        cf64.inv_d[s] = 1.0 / cf64.d[s];
        cf32.rho[s] = (float)cf64.rho[s];
        cf32.sigma[s] = (float)cf64.sigma[s];
        cf32.d[s] = (float)cf64.d[s];
        cf32.e[s] = (float)cf64.e[s];
        cf32.inv_d[s] = (float)cf64.inv_d[s];
        cfff.rho[s] = ff(cf64.rho[s]);
        cfff.sigma[s] = ff(cf64.sigma[s]);
        cfff.d[s] = ff(cf64.d[s]);
        cfff.e[s] = ff(cf64.e[s]);
        cfff.inv_d[s] = ff(cf64.inv_d[s]);
    }
    ODWF_CK(cudaGetDevice(&device));
    int rc = 0;
    double* rd = (double*)get_ws("r_handle", sizeof(double), &rc);
    if (rc) return rc;
    const double r = mq / (2.0 * m0);
    ODWF_CK(cudaMemcpy(rd, &r, sizeof(double), cudaMemcpyHostToDevice));
    bounds_flag = (unsigned*)get_ws("bounds_flag", sizeof(unsigned), &rc);
    if (rc) return rc;
    ODWF_CK(cudaMemset(bounds_flag, 0, sizeof(unsigned)));
    return ODWF_OK;
}

int Engine::bounds_status(cudaStream_t st) {
#ifdef ODWF_BOUNDS_CHECK
    unsigned f = 0;
    ODWF_CK(cudaMemcpyAsync(&f, bounds_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    ODWF_CK(cudaStreamSynchronize(st));
    if (f)
        return fail(ODWF_ECUDA, std::string("bounds check: a kernel gathered an index outside its field (flags ") +
                                    std::to_string(f) + ")");
#else
    (void)st;
#endif
    return ODWF_OK;
}

size_t Engine::half_bytes(Sp sp) const {
    switch (sp) {
        case Sp::F64: return sites5() * 192;
        case Sp::FF: return sites5() * 192;
        case Sp::F32: return sites5() * 96;
        default: return sites5() * 48;
    }
}

void* Engine::get_ws(const std::string& name, size_t bytes, int* rc) {
    *rc = ODWF_OK;
    if (bytes == 0) bytes = 16;
    auto& b = ws[name];
    if (b.bytes >= bytes) return b.p;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        *rc = fail(ODWF_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes for '" + name + "' failed");
        return nullptr;
    }
    b.bytes = bytes;
    return b.p;
}

int Engine::alloc_half(const std::string& name, Sp sp, int nsys, HalfField* f) {
    int rc = 0;
    f->sp = sp;
    f->stride = half_bytes(sp);
    f->data = get_ws(name, f->stride * nsys, &rc);
    if (rc) return rc;
    if (sp == Sp::F16 || sp == Sp::BF16) {
        f->norm_stride = norm_count();
        f->norm = (float*)get_ws(name + ".n", f->norm_stride * sizeof(float) * nsys, &rc);
        if (rc) return rc;
    } else {
        f->norm = nullptr;
        f->norm_stride = 0;
    }
    return ODWF_OK;
}

void* Engine::host_stage(size_t bytes, int* rc) {
    *rc = ODWF_OK;
    if (pinned_bytes >= bytes) return pinned;
    if (pinned) cudaFreeHost(pinned);
    pinned = nullptr;
    pinned_bytes = 0;
    if (cudaMallocHost(&pinned, bytes) != cudaSuccess) {
        cudaGetLastError();
        *rc = fail(ODWF_ENOMEM, "pinned host allocation failed");
        return nullptr;
    }
    pinned_bytes = bytes;
    return pinned;
}

int Engine::set_gauge(const void* U, cudaStream_t st) {
    if (!U) return fail(ODWF_EINVAL, "odwf_set_gauge: null U");
    const size_t nb = (size_t)4 * 2 * vh() * 9 * sizeof(double2);
    const double2* Ud = (const double2*)U;
    int rc = 0;
    if (!is_device_ptr(U)) {
        void* tmp = get_ws("gauge_stage", nb, &rc);
        if (rc) return rc;
        ODWF_CK(cudaMemcpyAsync(tmp, U, nb, cudaMemcpyHostToDevice, st));
        Ud = (const double2*)tmp;
    }
    const size_t nl = 8 * vh();
    if (!links_d18) ODWF_CK(cudaMalloc(&links_d18, nl * 144));
    ODWF_CK(launch_pack_links(Ud, links_d18, nullptr, nullptr, g, st));
    // FP32 copies are derived from the FP64 ones on first use (ensure_links)
    have_f12 = have_f18 = have_h12 = have_ff18 = false;
    for (bool& b : have_site) b = false;
    if (!is_device_ptr(U)) {
        ODWF_CK(cudaStreamSynchronize(st));
        auto it = ws.find("gauge_stage");  // the staging copy is only needed during packing
        if (it != ws.end() && it->second.p) {
            cudaFree(it->second.p);
            ws.erase(it);
        }
    }
    gauge_set = true;
    return ODWF_OK;
}

int Engine::ensure_links(Lk lk, cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "gauge field not set");
    const size_t nl = 8 * vh();
    if (!nbr) {
        ODWF_CK(cudaMalloc(&nbr, 2 * nl * sizeof(int)));
        ODWF_CK(launch_build_neighbours(nbr, g, st));
    }
    if (lk == Lk::F12 && !have_f12) {
        if (!links_f12) ODWF_CK(cudaMalloc(&links_f12, nl * 48));
        ODWF_CK(launch_links_from_d18(links_d18, nullptr, links_f12, nl, st));
        have_f12 = true;
    } else if (lk == Lk::F18 && !have_f18) {
        if (!links_f18) ODWF_CK(cudaMalloc(&links_f18, nl * 80));
        ODWF_CK(launch_links_from_d18(links_d18, links_f18, nullptr, nl, st));
        have_f18 = true;
    } else if (lk == Lk::FF18 && !have_ff18) {
        if (!links_ff18) ODWF_CK(cudaMalloc(&links_ff18, nl * 144));
        ODWF_CK(launch_links_ff18_from_d18(links_d18, links_ff18, nl, st));
        have_ff18 = true;
    } else if (lk == Lk::H12 && !have_h12) {
        if (!links_h12) ODWF_CK(cudaMalloc(&links_h12, nl * 24));
        ODWF_CK(launch_links_h12_from_d18(links_d18, links_h12, nl, st));
        have_h12 = true;
    }
    return ODWF_OK;
}

int Engine::ensure_site_links(Lk lk, cudaStream_t st) {
    int rc = ensure_links(lk, st);
    if (rc) return rc;
    const int k = (int)lk;
    if (have_site[k]) return ODWF_OK;
    const int bytes = lk == Lk::F12 ? 48 : lk == Lk::F18 ? 80 : lk == Lk::H12 ? 24 : 144;
    if (!links_site[k]) ODWF_CK(cudaMalloc(&links_site[k], 16 * vh() * (size_t)bytes));
    ODWF_CK(launch_links_site_major(links_of(lk), links_site[k], bytes, nbr, g, st));
    have_site[k] = true;
    return ODWF_OK;
}

template <>
HopParams<double> Engine::hop_params<double>(int p_out, const double* r_dev) const {
    HopParams<double> P;
    std::memset(&P, 0, sizeof(P));
    P.g = g;
    P.ns = ns;
    P.lg_ns = lg_ns;
    P.p_out = p_out;
    P.links = links_d18;
    P.r_sys = r_dev;
    P.cf = cf64;
    P.bounds_flag = bounds_flag;
    return P;
}

template <>
HopParams<ff> Engine::hop_params<ff>(int p_out, const double* r_dev) const {
    HopParams<ff> P;
    std::memset(&P, 0, sizeof(P));
    P.g = g;
    P.ns = ns;
    P.lg_ns = lg_ns;
    P.p_out = p_out;
    P.links = links_ff18;
    P.r_sys = r_dev;
    P.cf = cfff;
    P.bounds_flag = bounds_flag;
    return P;
}

template <>
HopParams<float> Engine::hop_params<float>(int p_out, const double* r_dev) const {
    HopParams<float> P;
    std::memset(&P, 0, sizeof(P));
    P.g = g;
    P.ns = ns;
    P.lg_ns = lg_ns;
    P.p_out = p_out;
    P.links = links_f12;
    P.nbr = nbr;
    P.r_sys = r_dev;
    P.cf = cf32;
    P.bounds_flag = bounds_flag;
    return P;
}

int Engine::apply_schur64(const HalfField& in, const HalfField& out, bool dag, const double* r_dev, cudaStream_t st) {
    int rc = 0;
    HalfField T, A;
    if ((rc = alloc_half("op.T", Sp::F64, 1, &T)) || (rc = alloc_half("op.A", Sp::F64, 1, &A))) return rc;
    if (!dag) {
        auto P = hop_params<double>(1, r_dev);
        P.in = in.ref_sys(0);
        P.out = T.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::MINV, 1, st));
        P = hop_params<double>(0, r_dev);
        P.in = T.ref_sys(0);
        P.z = in.ref_sys(0);
        P.out = out.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::SCHUR, 1, st));
    } else {
        ODWF_CK(launch_m5_f64(in.ref_sys(0), A.ref_sys(0), vh(), ns, r_dev, 0, 1, 3, cf64, st));
        auto P = hop_params<double>(1, r_dev);
        P.in = A.ref_sys(0);
        P.out = T.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::D_MINVDAG, 1, st));
        P = hop_params<double>(0, r_dev);
        P.in = T.ref_sys(0);
        P.z = in.ref_sys(0);
        P.out = out.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::D_ZMINUS, 1, st));
    }
    return ODWF_OK;
}

int Engine::apply_full64(const HalfField& in_e, const HalfField& in_o, const HalfField& out_e,
                         const HalfField& out_o, bool dag, const double* r_dev, cudaStream_t st) {
    const Epi e = dag ? Epi::D_FULL : Epi::FULL;
    auto P = hop_params<double>(0, r_dev);
    P.in = in_o.ref_sys(0);
    P.z = in_e.ref_sys(0);
    P.out = out_e.ref_sys(0);
    ODWF_CK(launch_hop_f64(P, e, 1, st));
    P = hop_params<double>(1, r_dev);
    P.in = in_e.ref_sys(0);
    P.z = in_o.ref_sys(0);
    P.out = out_o.ref_sys(0);
    ODWF_CK(launch_hop_f64(P, e, 1, st));
    return ODWF_OK;
}

namespace {
// Resolve an external input: device pointers pass through, host data is staged.
int stage_in(Engine* E, const void* in, size_t bytes, const char* name, cudaStream_t st, const double2** out) {
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
}  // namespace

int Engine::apply(void* out, const void* in, int mode, bool dag, cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "apply: gauge field not set");
    if (!out || !in) return fail(ODWF_EINVAL, "apply: null field");
    if (mode != ODWF_MODE_FULL && mode != ODWF_MODE_SCHUR_EVEN) return fail(ODWF_EINVAL, "apply: bad mode");
    const size_t eb = ext_bytes(mode);
    int rc = 0;
    const double2* din = nullptr;
    if ((rc = stage_in(this, in, eb, "ext.in", st, &din))) return rc;
    const bool out_dev = is_device_ptr(out);
    double2* dout = out_dev ? (double2*)out : (double2*)get_ws("ext.out", eb, &rc);
    if (rc) return rc;
    const double* rd = (const double*)ws["r_handle"].p;
    HalfField Xe, Xo, Ye, Yo;
    if ((rc = alloc_half("io.Xe", Sp::F64, 1, &Xe)) || (rc = alloc_half("io.Ye", Sp::F64, 1, &Ye))) return rc;
    if (mode == ODWF_MODE_SCHUR_EVEN) {
        ODWF_CK(launch_pack(Sp::F64, din, Xe.ref_sys(0), g, 0, ns, 1, st));
        if ((rc = apply_schur64(Xe, Ye, dag, rd, st))) return rc;
        ODWF_CK(launch_unpack(Sp::F64, Ye.ref_sys(0), dout, g, 0, ns, 1, st));
    } else {
        if ((rc = alloc_half("io.Xo", Sp::F64, 1, &Xo)) || (rc = alloc_half("io.Yo", Sp::F64, 1, &Yo))) return rc;
        ODWF_CK(launch_pack(Sp::F64, din, Xe.ref_sys(0), g, 0, ns, 0, st));
        ODWF_CK(launch_pack(Sp::F64, din, Xo.ref_sys(0), g, 1, ns, 0, st));
        if ((rc = apply_full64(Xe, Xo, Ye, Yo, dag, rd, st))) return rc;
        ODWF_CK(launch_unpack(Sp::F64, Ye.ref_sys(0), dout, g, 0, ns, 0, st));
        ODWF_CK(launch_unpack(Sp::F64, Yo.ref_sys(0), dout, g, 1, ns, 0, st));
    }
    if (!out_dev) {
        ODWF_CK(cudaMemcpyAsync(out, dout, eb, cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
    }
    return ODWF_OK;
}

int Engine::apply_normal(void* out, const void* in, int system, cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "apply_normal: gauge field not set");
    if (!out || !in) return fail(ODWF_EINVAL, "apply_normal: null field");
    if (system != ODWF_SYS_SCHUR_NORMAL && system != ODWF_SYS_FULL_NORMAL)
        return fail(ODWF_EINVAL, "apply_normal: system must be SCHUR_NORMAL or FULL_NORMAL");
    const int mode = system == ODWF_SYS_SCHUR_NORMAL ? ODWF_MODE_SCHUR_EVEN : ODWF_MODE_FULL;
    const size_t eb = ext_bytes(mode);
    int rc = 0;
    const double2* din = nullptr;
    if ((rc = stage_in(this, in, eb, "ext.in", st, &din))) return rc;
    const bool out_dev = is_device_ptr(out);
    double2* dout = out_dev ? (double2*)out : (double2*)get_ws("ext.out", eb, &rc);
    if (rc) return rc;
    const double* rd = (const double*)ws["r_handle"].p;
    HalfField Xe, Ye, T, A, C;
    if ((rc = alloc_half("io.Xe", Sp::F64, 1, &Xe)) || (rc = alloc_half("io.Ye", Sp::F64, 1, &Ye))) return rc;
    if (system == ODWF_SYS_SCHUR_NORMAL) {
        if ((rc = alloc_half("op.T", Sp::F64, 1, &T)) || (rc = alloc_half("op.A", Sp::F64, 1, &A)) ||
            (rc = alloc_half("op.C", Sp::F64, 1, &C)))
            return rc;
        ODWF_CK(launch_pack(Sp::F64, din, Xe.ref_sys(0), g, 0, ns, 1, st));
        auto P = hop_params<double>(1, rd);
        P.in = Xe.ref_sys(0);
        P.out = T.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::MINV, 1, st));
        P = hop_params<double>(0, rd);
        P.in = T.ref_sys(0);
        P.z = Xe.ref_sys(0);
        P.out = A.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::SCHUR_MDINV, 1, st));
        P = hop_params<double>(1, rd);
        P.in = A.ref_sys(0);
        P.out = C.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::D_MINVDAG, 1, st));
        P = hop_params<double>(0, rd);
        P.in = C.ref_sys(0);
        P.z = A.ref_sys(0);
        P.out = Ye.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::D_NORMAL, 1, st));
        ODWF_CK(launch_unpack(Sp::F64, Ye.ref_sys(0), dout, g, 0, ns, 1, st));
    } else {
        HalfField Xo, Yo, Ze, Zo;
        if ((rc = alloc_half("io.Xo", Sp::F64, 1, &Xo)) || (rc = alloc_half("io.Yo", Sp::F64, 1, &Yo)) ||
            (rc = alloc_half("io.Ze", Sp::F64, 1, &Ze)) || (rc = alloc_half("io.Zo", Sp::F64, 1, &Zo)))
            return rc;
        ODWF_CK(launch_pack(Sp::F64, din, Xe.ref_sys(0), g, 0, ns, 0, st));
        ODWF_CK(launch_pack(Sp::F64, din, Xo.ref_sys(0), g, 1, ns, 0, st));
        if ((rc = apply_full64(Xe, Xo, Ze, Zo, false, rd, st))) return rc;
        if ((rc = apply_full64(Ze, Zo, Ye, Yo, true, rd, st))) return rc;
        ODWF_CK(launch_unpack(Sp::F64, Ye.ref_sys(0), dout, g, 0, ns, 0, st));
        ODWF_CK(launch_unpack(Sp::F64, Yo.ref_sys(0), dout, g, 1, ns, 0, st));
    }
    if (!out_dev) {
        ODWF_CK(cudaMemcpyAsync(out, dout, eb, cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
    }
    return ODWF_OK;
}

// S^dag S in float-float arithmetic with float-float fields and links: the operator of the
// mixed-precision CG's reliable updates.
int Engine::apply_ff_normal(void* out, const void* in, cudaStream_t st) {
    if (!out || !in) return fail(ODWF_EINVAL, "apply_normal_prec: null field");
    const size_t eb = ext_bytes(ODWF_MODE_SCHUR_EVEN);
    int rc = 0;
    const double2* din = nullptr;
    if ((rc = stage_in(this, in, eb, "ext.in", st, &din))) return rc;
    const bool out_dev = is_device_ptr(out);
    double2* dout = out_dev ? (double2*)out : (double2*)get_ws("ext.out", eb, &rc);
    if (rc) return rc;
    const double* rd = (const double*)ws["r_handle"].p;
    HalfField X, Y, T, A, C;
    if ((rc = alloc_half("ff.X", Sp::FF, 1, &X)) || (rc = alloc_half("ff.Y", Sp::FF, 1, &Y)) ||
        (rc = alloc_half("ff.T", Sp::FF, 1, &T)) || (rc = alloc_half("ff.A", Sp::FF, 1, &A)) ||
        (rc = alloc_half("ff.C", Sp::FF, 1, &C)))
        return rc;
    if ((rc = ensure_links(Lk::FF18, st))) return rc;
    ODWF_CK(launch_pack(Sp::FF, din, X.ref_sys(0), g, 0, ns, 1, st));
    auto P = hop_params<ff>(1, rd);
    P.in = X.ref_sys(0);
    P.out = T.ref_sys(0);
    ODWF_CK(launch_hop_ff(P, Epi::MINV, 1, st));
    P.p_out = 0;
    P.in = T.ref_sys(0);
    P.z = X.ref_sys(0);
    P.out = A.ref_sys(0);
    ODWF_CK(launch_hop_ff(P, Epi::SCHUR_MDINV, 1, st));
    P.p_out = 1;
    P.in = A.ref_sys(0);
    P.z = FieldRef{};
    P.out = C.ref_sys(0);
    ODWF_CK(launch_hop_ff(P, Epi::D_MINVDAG, 1, st));
    P.p_out = 0;
    P.in = C.ref_sys(0);
    P.z = A.ref_sys(0);
    P.out = Y.ref_sys(0);
    ODWF_CK(launch_hop_ff(P, Epi::D_NORMAL, 1, st));
    ODWF_CK(launch_unpack(Sp::FF, Y.ref_sys(0), dout, g, 0, ns, 1, st));
    if (!out_dev) {
        ODWF_CK(cudaMemcpyAsync(out, dout, eb, cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
    }
    return ODWF_OK;
}

int Engine::apply_low_normal(void* out, const void* in, int prec, int recon, cudaStream_t st) {
    if (!gauge_set) return fail(ODWF_EINVAL, "apply_normal_prec: gauge field not set");
    if (!out || !in) return fail(ODWF_EINVAL, "apply_normal_prec: null field");
    if (prec == ODWF_FF) return apply_ff_normal(out, in, st);
    if (prec != ODWF_F32 && prec != ODWF_F16 && prec != ODWF_BF16)
        return fail(ODWF_EINVAL, "apply_normal_prec: prec must be F32, F16, BF16 or FF");
    if (recon != 12 && recon != 18) return fail(ODWF_EINVAL, "apply_normal_prec: link_recon must be 12 or 18");
    const Sp low = (Sp)prec;
    const size_t eb = ext_bytes(ODWF_MODE_SCHUR_EVEN);
    int rc = 0;
    const double2* din = nullptr;
    if ((rc = stage_in(this, in, eb, "ext.in", st, &din))) return rc;
    const bool out_dev = is_device_ptr(out);
    double2* dout = out_dev ? (double2*)out : (double2*)get_ws("ext.out", eb, &rc);
    if (rc) return rc;
    const double* rd = (const double*)ws["r_handle"].p;
    HalfField X, Y, T, A, C;
    if ((rc = alloc_half("lo.X", low, 1, &X)) || (rc = alloc_half("lo.Y", low, 1, &Y)) ||
        (rc = alloc_half("lo.T", low, 1, &T)) || (rc = alloc_half("lo.A", low, 1, &A)) ||
        (rc = alloc_half("lo.C", low, 1, &C)))
        return rc;
    const Lk lk = recon == 12 ? Lk::F12 : Lk::F18;
    if ((rc = ensure_links(lk, st))) return rc;
    ODWF_CK(launch_pack(low, din, X.ref_sys(0), g, 0, ns, 1, st));
    auto P = hop_params<float>(1, rd);
    P.links = recon == 12 ? links_f12 : links_f18;
    P.in = X.ref_sys(0);
    P.out = T.ref_sys(0);
    ODWF_CK(launch_hop_mixed(P, Epi::MINV, low, lk, 1, st));
    P.p_out = 0;
    P.in = T.ref_sys(0);
    P.z = X.ref_sys(0);
    P.out = A.ref_sys(0);
    ODWF_CK(launch_hop_mixed(P, Epi::SCHUR_MDINV, low, lk, 1, st));
    P.p_out = 1;
    P.in = A.ref_sys(0);
    P.z = FieldRef{};
    P.out = C.ref_sys(0);
    ODWF_CK(launch_hop_mixed(P, Epi::D_MINVDAG, low, lk, 1, st));
    P.p_out = 0;
    P.in = C.ref_sys(0);
    P.z = A.ref_sys(0);
    P.out = Y.ref_sys(0);
    ODWF_CK(launch_hop_mixed(P, Epi::D_NORMAL, low, lk, 1, st));
    ODWF_CK(launch_unpack(low, Y.ref_sys(0), dout, g, 0, ns, 1, st));
    if (!out_dev) {
        ODWF_CK(cudaMemcpyAsync(out, dout, eb, cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
    }
    return ODWF_OK;
}

int Engine::apply_m5(void* out, const void* in, long n_sites, int op, cudaStream_t st) {
    if (!out || !in || n_sites <= 0) return fail(ODWF_EINVAL, "apply_m5: bad arguments");
    if (op < 0 || op > 3) return fail(ODWF_EINVAL, "apply_m5: op must be 0..3");
    if ((double)n_sites * ns > 4.0e9) return fail(ODWF_EINVAL, "apply_m5: too many sites");
    Geom gf = g;
    gf.Vh = (int)n_sites;  // a flat list of sites: ext_mode 1 uses h as the site index
    const size_t eb = (size_t)n_sites * ns * 192;
    int rc = 0;
    const double2* din = nullptr;
    if ((rc = stage_in(this, in, eb, "ext.in", st, &din))) return rc;
    const bool out_dev = is_device_ptr(out);
    double2* dout = out_dev ? (double2*)out : (double2*)get_ws("ext.out", eb, &rc);
    if (rc) return rc;
    HalfField X, Y;
    X.sp = Y.sp = Sp::F64;
    X.data = get_ws("m5.X", eb, &rc);
    if (rc) return rc;
    Y.data = get_ws("m5.Y", eb, &rc);
    if (rc) return rc;
    const double* rd = (const double*)ws["r_handle"].p;
    ODWF_CK(launch_pack(Sp::F64, din, X.ref_sys(0), gf, 0, ns, 1, st));
    ODWF_CK(launch_m5_f64(X.ref_sys(0), Y.ref_sys(0), (size_t)n_sites, ns, rd, 0, 1, op, cf64, st));
    ODWF_CK(launch_unpack(Sp::F64, Y.ref_sys(0), dout, gf, 0, ns, 1, st));
    if (!out_dev) {
        ODWF_CK(cudaMemcpyAsync(out, dout, eb, cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
    }
    return ODWF_OK;
}

int check_params(const odwf_solve_params* prm) {
    if (!prm) return fail(ODWF_EINVAL, "solve: null params");
    if (!(prm->tol > 0.0) || !std::isfinite(prm->tol)) return fail(ODWF_EINVAL, "solve: tol must be > 0");
    if (prm->max_iter <= 0) return fail(ODWF_EINVAL, "solve: max_iter must be > 0");
    if (prm->prec < ODWF_F64 || prm->prec > ODWF_BF16) return fail(ODWF_EINVAL, "solve: bad prec");
    if (prm->link_recon != 0 && prm->link_recon != 12 && prm->link_recon != 18)
        return fail(ODWF_EINVAL, "solve: link_recon must be 0, 12 or 18");
    if (prm->link_prec != 0 && prm->link_prec != ODWF_F32 && prm->link_prec != ODWF_F16)
        return fail(ODWF_EINVAL, "solve: link_prec must be 0, ODWF_F32 or ODWF_F16");
    if (prm->update_arith < ODWF_UPDATES_AUTO || prm->update_arith > ODWF_UPDATES_FF)
        return fail(ODWF_EINVAL, "solve: update_arith must be ODWF_UPDATES_AUTO, _F64 or _FF");
    if (prm->link_prec == ODWF_F16 && prm->link_recon == 18)
        return fail(ODWF_EINVAL, "solve: FP16 links are stored with 12 reals (link_recon 0 or 12)");
    return ODWF_OK;
}

namespace {
// An internal stream of the highest priority that starts after the work queued on the
// caller's stream and that the caller's stream waits for at the end.
struct SolveStream {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    int open(cudaStream_t user) {
        int least = 0, greatest = 0;
        ODWF_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        ODWF_CK(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest));
        ODWF_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ODWF_CK(cudaEventRecord(ev, user));
        ODWF_CK(cudaStreamWaitEvent(s, ev, 0));
        return ODWF_OK;
    }
    int close(cudaStream_t user) {
        int rc = ODWF_OK;
        if (s && ev) {
            if (cudaEventRecord(ev, s) != cudaSuccess || cudaStreamWaitEvent(user, ev, 0) != cudaSuccess)
                rc = fail(ODWF_ECUDA, "solve: joining the caller's stream failed");
        }
        if (ev) cudaEventDestroy(ev);
        if (s) cudaStreamDestroy(s);  // released once its queued work has completed
        s = nullptr;
        ev = nullptr;
        return rc;
    }
    ~SolveStream() {
        if (ev) cudaEventDestroy(ev);
        if (s) cudaStreamDestroy(s);
    }
};
}  // namespace

int Engine::solve(int nsys, void* const* x, const void* const* b, const double* mq_arr,
                  const odwf_solve_params* prm, odwf_solve_stats* stats, cudaStream_t st) {
    int rc = check_params(prm);
    if (rc) return rc;
    if (!gauge_set) return fail(ODWF_EINVAL, "solve: gauge field not set");
    if (nsys <= 0 || !x || !b) return fail(ODWF_EINVAL, "solve: bad system list");
    for (int i = 0; i < nsys; ++i)
        if (!x[i] || !b[i]) return fail(ODWF_EINVAL, "solve: null x or b");
    if (prm->system != ODWF_SYS_SCHUR_NORMAL) {
        if (nsys != 1) return fail(ODWF_EINVAL, "solve: batched solves support SCHUR_NORMAL only");
        return solve_full(x[0], b[0], prm, stats, st);
    }
    const auto t0 = std::chrono::steady_clock::now();
    // The solve runs on an internal stream of the highest priority (its reliable updates one
    // level below), joined to the caller's stream at both ends.
    SolveStream ss;
    if ((rc = ss.open(st))) return rc;
    rc = solve_on(nsys, x, b, mq_arr, prm, stats, ss.s);
    const int rc2 = ss.close(st);
    if (stats)
        for (int i = 0; i < nsys; ++i)
            stats[i].time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc ? rc : rc2;
}

int Engine::solve_on(int nsys, void* const* x, const void* const* b, const double* mq_arr,
                     const odwf_solve_params* prm, odwf_solve_stats* stats, cudaStream_t st) {
    int rc = 0;
    BatchCG bc;
    if ((rc = bc.init(this, nsys, *prm, st, 1))) return rc;
    const size_t eb = ext_bytes(ODWF_MODE_SCHUR_EVEN);
    for (int i = 0; i < nsys; ++i) {
        double m = mq;
        if (mq_arr) m = mq_arr[i];
        else if (std::isfinite(prm->mq)) m = prm->mq;
        if ((rc = bc.admit(i, (const double2*)b[i], m, st))) return rc;
    }
    const int every = prm->check_every > 0 ? prm->check_every : 8;
    while (true) {
        if ((rc = bc.resume(st, true))) return rc;
        if ((rc = bc.run_iterations(every, st))) return rc;
        if ((rc = bc.poll(st))) return rc;
        if ((rc = bc.service(st))) return rc;
        if (!bc.any_running()) break;
    }
    int first_bad = ODWF_OK;
    for (int i = 0; i < nsys; ++i) {
        const bool out_dev = is_device_ptr(x[i]);
        double2* dx = out_dev ? (double2*)x[i] : (double2*)get_ws("ext.out", eb, &rc);
        if (rc) return rc;
        double tr = 0.0;
        if ((rc = bc.finalize(i, dx, st, &tr))) return rc;
        if (!out_dev) ODWF_CK(cudaMemcpyAsync(x[i], dx, eb, cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
        const SysState& S = bc.st_host[i];
        int code = ODWF_OK;
        if (S.status == kBreakdown) code = ODWF_EBREAKDOWN;
        else if (S.status != kDone) code = ODWF_ENOCONV;
        if (code && !first_bad) first_bad = code;
        if (stats) {
            stats[i].iters = S.iter;
            stats[i].n_reliable = bc.n_reliable[i];
            stats[i].true_resid = tr;
            stats[i].status = code;
        }
    }
    if (first_bad == ODWF_ENOCONV) set_error("solve: max_iter reached before the tolerance");
    if (first_bad == ODWF_EBREAKDOWN) set_error("solve: CG breakdown");
    return first_bad;
}

}  // namespace odwf
