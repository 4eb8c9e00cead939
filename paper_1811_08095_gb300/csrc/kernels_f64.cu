// FP64 kernels, layout conversion, vector and gauge-packing kernels.
#include "kernels.cuh"
#include "kernels.h"

#include <atomic>

namespace odwf {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int lg2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

namespace {
constexpr int kBS = 256;

template <int F>
cudaError_t hop64(const HopParams<double>& P, int nsys, cudaStream_t st) {
    const size_t n = (size_t)P.g.Vh * P.ns;
    dim3 grid(blocks_for(n, kBS), nsys);
    note_launch(); hop_kernel<SpF64, SpF64, SpF64, SpF64, LinkD18, double, F><<<grid, kBS, 0, st>>>(P);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_hop_f64(const HopParams<double>& P, Epi e, int nsys, cudaStream_t st) {
    switch (e) {
        case Epi::MINV: return hop64<EPI_MINV>(P, nsys, st);
        case Epi::SCHUR: return hop64<EPI_SCHUR>(P, nsys, st);
        case Epi::SCHUR_NORM_MDINV: return hop64<EPI_SCHUR_NORM_MDINV>(P, nsys, st);
        case Epi::SCHUR_MDINV: return hop64<EPI_SCHUR_NORM_MDINV_STORE>(P, nsys, st);
        case Epi::FULL: return hop64<EPI_FULL>(P, nsys, st);
        case Epi::PLAIN: return hop64<EPI_PLAIN>(P, nsys, st);
        case Epi::ZMINUS_POSTMINV: return hop64<EPI_ZMINUS_POSTMINV>(P, nsys, st);
        case Epi::ZMINUS: return hop64<EPI_ZMINUS>(P, nsys, st);
        case Epi::D_MINVDAG: return hop64<EPID_MINVDAG>(P, nsys, st);
        case Epi::D_NORMAL: return hop64<EPID_NORMAL>(P, nsys, st);
        case Epi::D_NORMAL_CG: return hop64<EPID_NORMAL_CG>(P, nsys, st);
        case Epi::D_NORMAL_RESID: return hop64<EPID_NORMAL_RESID>(P, nsys, st);
        case Epi::D_ZMINUS: return hop64<EPID_ZMINUS>(P, nsys, st);
        case Epi::D_FULL: return hop64<EPID_FULL>(P, nsys, st);
        case Epi::D_PLAIN: return hop64<EPID_PLAIN>(P, nsys, st);
        case Epi::D_SCHUR2: return hop64<EPID_SCHUR2>(P, nsys, st);
        case Epi::D_ZMINUS_POSTMINVDAG: return hop64<EPID_ZMINUS_POSTMINVDAG>(P, nsys, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_m5_f64(const FieldRef& in, const FieldRef& out, size_t n_sites, int ns, const double* r_sys,
                          int sys_base, int nsys, int op, const Coef5<double>& cf, cudaStream_t st,
                          const SysState* gate_st, int need) {
    dim3 grid(blocks_for(n_sites * ns, kBS), nsys);
    note_launch();
    m5_kernel<SpF64, SpF64, double><<<grid, kBS, 0, st>>>(in, out, n_sites, ns, lg2(ns), r_sys, sys_base, op, cf,
                                                           gate_st, need);
    return cudaGetLastError();
}

cudaError_t launch_pack(Sp sp, const double2* ext, const FieldRef& out, const Geom& g, int p, int ns, int ext_mode,
                        cudaStream_t st) {
    const int grid = blocks_for((size_t)g.Vh * ns, kBS);
    const int lg = lg2(ns);
    switch (sp) {
        case Sp::F64: note_launch(); pack_kernel<SpF64><<<grid, kBS, 0, st>>>(ext, out, g, p, ns, lg, ext_mode); break;
        case Sp::F32: note_launch(); pack_kernel<SpF32><<<grid, kBS, 0, st>>>(ext, out, g, p, ns, lg, ext_mode); break;
        case Sp::F16: note_launch(); pack_kernel<SpF16><<<grid, kBS, 0, st>>>(ext, out, g, p, ns, lg, ext_mode); break;
        case Sp::BF16: note_launch(); pack_kernel<SpBF16><<<grid, kBS, 0, st>>>(ext, out, g, p, ns, lg, ext_mode); break;
        case Sp::FF: note_launch(); pack_kernel<SpFF><<<grid, kBS, 0, st>>>(ext, out, g, p, ns, lg, ext_mode); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(Sp sp, const FieldRef& in, double2* ext, const Geom& g, int p, int ns, int ext_mode,
                          cudaStream_t st) {
    const int grid = blocks_for((size_t)g.Vh * ns, kBS);
    const int lg = lg2(ns);
    switch (sp) {
        case Sp::F64: note_launch(); unpack_kernel<SpF64><<<grid, kBS, 0, st>>>(in, ext, g, p, ns, lg, ext_mode); break;
        case Sp::F32: note_launch(); unpack_kernel<SpF32><<<grid, kBS, 0, st>>>(in, ext, g, p, ns, lg, ext_mode); break;
        case Sp::F16: note_launch(); unpack_kernel<SpF16><<<grid, kBS, 0, st>>>(in, ext, g, p, ns, lg, ext_mode); break;
        case Sp::BF16: note_launch(); unpack_kernel<SpBF16><<<grid, kBS, 0, st>>>(in, ext, g, p, ns, lg, ext_mode); break;
        case Sp::FF: note_launch(); unpack_kernel<SpFF><<<grid, kBS, 0, st>>>(in, ext, g, p, ns, lg, ext_mode); break;
    }
    return cudaGetLastError();
}

thread_local unsigned long long* g_vec_prof = nullptr;  // counter for the next vec launch (profiling)

void set_vec_prof(unsigned long long* c) { g_vec_prof = c; }

namespace {
template <class SX, class SY, class R>
cudaError_t vec_t(const FieldRef& x, const FieldRef& y, size_t n5, int ns, int kind, double coef, SysState* st,
                  int gate, int need, double* partials, unsigned* counters, int part_stride, int sys_base, int nsys,
                  cudaStream_t stream) {
    dim3 grid(blocks_for(n5, kBS), nsys);
    note_launch(); vec_kernel<SX, SY, R><<<grid, kBS, 0, stream>>>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters,
                                                    part_stride, sys_base, g_vec_prof);
    return cudaGetLastError();
}

template <class SX>
cudaError_t vec_y(Sp spy, const FieldRef& x, const FieldRef& y, size_t n5, int ns, int kind, double coef,
                  SysState* st, int gate, int need, double* partials, unsigned* counters, int part_stride, int sys_base,
                  int nsys, cudaStream_t stream) {
    const bool dx = std::is_same<SX, SpF64>::value || std::is_same<SX, SpFF>::value;
    switch (spy) {
        case Sp::F64:
            return vec_t<SX, SpF64, double>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base,
                                            nsys, stream);
        case Sp::FF:  // float-float storage, FP64 arithmetic (vector work is a few operations per value)
            return vec_t<SX, SpFF, double>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base,
                                           nsys, stream);
        case Sp::F32:
            if (dx) return vec_t<SX, SpF32, double>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base, nsys, stream);
            return vec_t<SX, SpF32, float>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base,
                                           nsys, stream);
        case Sp::F16:
            if (dx) return vec_t<SX, SpF16, double>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base, nsys, stream);
            return vec_t<SX, SpF16, float>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base,
                                           nsys, stream);
        case Sp::BF16:
            if (dx) return vec_t<SX, SpBF16, double>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base, nsys, stream);
            return vec_t<SX, SpBF16, float>(x, y, n5, ns, kind, coef, st, gate, need, partials, counters,
                                            part_stride, sys_base, nsys, stream);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_vec(Sp spx, Sp spy, const FieldRef& x, const FieldRef& y, size_t n5, int ns, int kind,
                       double coef, SysState* st, int gate, int need, double* partials,
                       unsigned* counters, int sys_base, int nsys, cudaStream_t stream, int part_stride) {
    switch (spx) {
        case Sp::F64: return vec_y<SpF64>(spy, x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base, nsys, stream);
        case Sp::F32: return vec_y<SpF32>(spy, x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base, nsys, stream);
        case Sp::F16: return vec_y<SpF16>(spy, x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base, nsys, stream);
        case Sp::BF16: return vec_y<SpBF16>(spy, x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base, nsys, stream);
        case Sp::FF: return vec_y<SpFF>(spy, x, y, n5, ns, kind, coef, st, gate, need, partials, counters, part_stride, sys_base, nsys, stream);
    }
    return cudaErrorInvalidValue;
}

// One thread per system: CG bookkeeping between phases.
//   mode 0 (init):  bb = sum; mixed precision: rscale = |b|, rr = r_max = 1; plain CG:
//                   rr = sum, r_max = |b|; status running (done when b = 0)
//   mode 1 (after a reliable update, sum = ||b - A x||^2): done / max-iter / restart with
//                   the continued beta, rscale = |r| (mixed), rr, r_max (status kRestarting)
//   mode 2:         kRestarting -> kRunning (launched on the iteration stream)
__global__ void state_kernel(SysState* st, int nsys, int mode, double tol2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsys) return;
    SysState& S = st[i];
    if (mode == 0) {
        S.bb = S.sum;
        S.stop_rr = tol2 * S.sum;
        if (S.reliable && S.sum > 0.0) {
            S.rscale = sqrt(S.sum);
            S.rr = 1.0;
            S.r_max = 1.0;
            S.stop_in = tol2;
        } else {
            S.rscale = 1.0;
            S.rr = S.sum;
            S.r_max = sqrt(S.sum);
            S.stop_in = S.stop_rr;
        }
        S.iter = 0;
        S.alpha = S.beta = 0.0;
        // a non-finite right-hand side (NaN / Inf in b) is a breakdown, not a converged b = 0
        S.status = !isfinite(S.sum) ? kBreakdown : (S.sum > 0.0) ? kRunning : kDone;
    } else if (mode == 2) {
        if (S.status == kRestarting) S.status = kRunning;
    } else if (mode == 3) {
        S.status = kIdle;  // cancelled: every gated kernel skips the slot from now on
    } else {
        if (S.status != kNeedUpdate) return;
        const double rt = S.sum;  // true |r|^2 of the recomputed residual
        if (!isfinite(rt)) {
            S.status = kBreakdown;
        } else if (rt <= S.stop_rr) {
            S.status = kDone;
        } else if (S.iter >= S.max_iter) {
            S.status = kMaxIter;
        } else {
            // continue the search direction: p_true = r_true + beta_true p_true, written in
            // the new inner units (p_inner = p_true / rscale)
            const double s_old = S.rscale;
            const double s_new = S.reliable ? sqrt(rt) : 1.0;
            S.beta = rt / (S.rr * s_old * s_old) * (s_old / s_new);
            S.rscale = s_new;
            S.rr = rt / (s_new * s_new);
            S.r_max = sqrt(S.rr);
            S.stop_in = S.stop_rr / (s_new * s_new);
            S.status = kRestarting;
        }
    }
}


cudaError_t launch_state(SysState* st, int nsys, int mode, double tol2, cudaStream_t stream) {
    note_launch(); state_kernel<<<blocks_for(nsys, 128), 128, 0, stream>>>(st, nsys, mode, tol2);
    return cudaGetLastError();
}

// One thread per (parity, mu, half-site): U_mu(x) -> packed formats
__global__ void pack_links_kernel(const double2* __restrict__ U, double* d18, float* f18, float* f12, Geom g) {
    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nh = (size_t)g.Vh;
    if (gi >= 8 * nh) return;
    const int h = (int)(gi % nh);
    const int mu = (int)((gi / nh) % 4);
    const int p = (int)(gi / (4 * nh));
    int c[4];
    site_coords(g, p, h, c);
    const size_t V = 2 * nh;
    const size_t lex = (size_t)c[0] + (size_t)g.L[0] * (c[1] + (size_t)g.L[1] * (c[2] + (size_t)g.L[2] * c[3]));
    const double2* src = U + ((size_t)mu * V + lex) * 9;
    const size_t o = ((size_t)(p * 4 + mu) * nh + h);
    for (int k = 0; k < 9; ++k) {
        const double2 q = src[k];
        if (d18) { d18[o * 18 + 2 * k] = q.x; d18[o * 18 + 2 * k + 1] = q.y; }
        if (f18) { f18[o * 20 + 2 * k] = (float)q.x; f18[o * 20 + 2 * k + 1] = (float)q.y; }
        if (f12 && k < 6) { f12[o * 12 + 2 * k] = (float)q.x; f12[o * 12 + 2 * k + 1] = (float)q.y; }
    }
    if (f18) { f18[o * 20 + 18] = 0.f; f18[o * 20 + 19] = 0.f; }
}

__global__ void links_from_d18_kernel(const double* __restrict__ d18, float* f18, float* f12, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* src = d18 + i * 18;
    if (f18) {
        for (int k = 0; k < 18; ++k) f18[i * 20 + k] = (float)src[k];
        f18[i * 20 + 18] = 0.f;
        f18[i * 20 + 19] = 0.f;
    }
    if (f12)
        for (int k = 0; k < 12; ++k) f12[i * 12 + k] = (float)src[k];
}

__global__ void build_neighbours_kernel(int* nbr, Geom g) {
    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= 2 * (size_t)g.Vh) return;
    const int p = (int)(gi / g.Vh), h = (int)(gi % g.Vh);
    int c[4];
    site_coords(g, p, h, c);
    int* out = nbr + gi * 8;
    for (int mu = 0; mu < 4; ++mu) {
        const int Lm = g.L[mu];
        int cf[4] = {c[0], c[1], c[2], c[3]}, cb[4] = {c[0], c[1], c[2], c[3]};
        cf[mu] = c[mu] + 1 == Lm ? 0 : c[mu] + 1;
        cb[mu] = c[mu] == 0 ? Lm - 1 : c[mu] - 1;
        const bool flip_f = mu == 3 && g.tbc && c[3] == Lm - 1;
        const bool flip_b = mu == 3 && g.tbc && c[3] == 0;
        out[2 * mu] = (int)((unsigned)half_index(g, cf) | (flip_f ? 0x80000000u : 0u));
        out[2 * mu + 1] = (int)((unsigned)half_index(g, cb) | (flip_b ? 0x80000000u : 0u));
    }
}

cudaError_t launch_build_neighbours(int* nbr, const Geom& g, cudaStream_t st) {
    note_launch();
    build_neighbours_kernel<<<blocks_for(2 * (size_t)g.Vh, 256), 256, 0, st>>>(nbr, g);
    return cudaGetLastError();
}

cudaError_t launch_links_from_d18(const void* d18, void* f18, void* f12, size_t n_links, cudaStream_t st) {
    note_launch();
    links_from_d18_kernel<<<blocks_for(n_links, 256), 256, 0, st>>>((const double*)d18, (float*)f18, (float*)f12,
                                                                     n_links);
    return cudaGetLastError();
}

__global__ void links_h12_from_d18_kernel(const double* __restrict__ d18, __half2* h12, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* src = d18 + i * 18;
    for (int k = 0; k < 6; ++k) h12[i * 6 + k] = __halves2half2(__double2half(src[2 * k]), __double2half(src[2 * k + 1]));
}

cudaError_t launch_links_h12_from_d18(const void* d18, void* h12, size_t n_links, cudaStream_t st) {
    note_launch();
    links_h12_from_d18_kernel<<<blocks_for(n_links, 256), 256, 0, st>>>((const double*)d18, (__half2*)h12, n_links);
    return cudaGetLastError();
}

__global__ void links_site_major_kernel(const uint2* __restrict__ in, uint2* __restrict__ out, int words,
                                        const int* __restrict__ nbr, Geom g) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (p * Vh + h) * 8 + j
    if (i >= 16 * (size_t)g.Vh) return;
    const int j = (int)(i & 7);
    const size_t ph = i >> 3;
    const int p = (int)(ph / g.Vh), h = (int)(ph % g.Vh), mu = j >> 1;
    const size_t src = (j & 1) == 0 ? ((size_t)(p * 4 + mu) * g.Vh + h)
                                    : ((size_t)((1 - p) * 4 + mu) * g.Vh + (nbr[ph * 8 + j] & 0x7fffffff));
    for (int w = 0; w < words; ++w) out[i * words + w] = in[src * words + w];
}

cudaError_t launch_links_site_major(const void* in, void* out, int bytes, const int* nbr, const Geom& g,
                                    cudaStream_t st) {
    note_launch();
    links_site_major_kernel<<<blocks_for(16 * (size_t)g.Vh, 256), 256, 0, st>>>((const uint2*)in, (uint2*)out, bytes / 8,
                                                                               nbr, g);
    return cudaGetLastError();
}

cudaError_t launch_pack_links(const double2* U, void* d18, void* f18, void* f12, const Geom& g, cudaStream_t st) {
    const size_t n = 8 * (size_t)g.Vh;
    note_launch(); pack_links_kernel<<<blocks_for(n, 256), 256, 0, st>>>(U, (double*)d18, (float*)f18, (float*)f12, g);
    return cudaGetLastError();
}

}  // namespace odwf
