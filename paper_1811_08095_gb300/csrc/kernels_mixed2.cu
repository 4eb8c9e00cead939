// Mixed-precision CG kernels, second generation (Ns = 8, 16; FP16 / BF16 / FP32 storage).  For FP16 /
// BF16 storage the hops K1, K2 and K3 run as the two-s-per-lane kernels of kernels_mixed3.cu.
//
// The non-dagger hops read the chirally shifted field chi = B psi, written by the kernel
// that produces psi, so B is applied once per site on the producing side instead of once
// per (site, direction) on the consuming side:
//   P   p = r + beta p;  chi_p = B p                                   (stores p, chi_p)
//   K1  chi_t = B M^-1 (-1/2 W chi_p)                                  (t = M^-1 H_oe p)
//   K2  s = p - M^-1 (-1/2 W chi_t);  |s|^2 -> alpha;  a = M^-dag s    (s = S p)
//   K3  c = M^-dag (-1/2 B^dag W^dag a)
//   K4  A p = M^dag a + 1/2 B^dag W^dag c;  r -= alpha A p;  x += alpha p;  |r|^2 -> beta
// The eight links of an output site (stored contiguously per site, see launch_links_site_major)
// are loaded (and, for 12-real storage, completed to
// 18 reals) once per site: lane d < 8 of the site's lane group handles direction d and
// leaves it in shared memory, which the group's Ns lanes then read (the group lies in one
// warp, so a warp barrier suffices).  The per-site FP16/BF16 scale and the time-boundary
// sign of each neighbour are folded into the FMAs that accumulate its contribution.  Ns
// is a template parameter, so the fifth-dimension scans unroll.
#include <type_traits>

#include "kernels_mixed_common.cuh"

namespace odwf {

namespace {

using namespace mx;

constexpr int kBS2 = 256;

template <class SP, class LK, int NS, int KIND>
__global__ void __launch_bounds__(kBS2, 3) hop2_kernel(const HopParams<float> P) {
    constexpr int kLS = 18;            // floats per staged link: 9 x (ur, ui)
    constexpr int kSL = 8 * kLS + 4;   // floats per site (padding spreads banks)
    constexpr bool DAG = (KIND == K3 || KIND == K4);
    const int sys = blockIdx.y + P.sys_base;
    if (P.gate && P.st[sys].status != P.need_status) return;
    if (P.prof_count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(P.prof_count, 1ull);

    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(gi & (NS - 1));  // lane of the site's group; it holds s = s_of_lane(lane)
    const int s = s_of_lane(lane, NS);
    const size_t hh = gi / NS;
    const bool valid = hh < (size_t)P.g.Vh;
    const int h = valid ? (int)hh : 0;
    const float r = (float)P.r_sys[sys];
    const int p_out = P.p_out;

    // the eight neighbours of this site (half index) and their time-boundary signs (bit j)
    int nb[8];
    unsigned flip = 0;
    {
        const int4* tp = reinterpret_cast<const int4*>(P.nbr + ((size_t)p_out * P.g.Vh + h) * 8);
        const int4 n0 = __ldg(tp), n1 = __ldg(tp + 1);
        const int raw[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            nb[j] = checked_index(raw[j] & 0x7fffffff, P.g.Vh, P.bounds_flag, kBoundsNeighbour);
            flip |= ((unsigned)raw[j] >> 31) << j;
        }
    }

    // stage the site's eight links in shared memory as (ur, ui) pairs: lane d < 8 of the group
    // loads direction d from the site-major link array (the eight links of a site are contiguous,
    // so the loads neither wait for the neighbour table nor scatter); the group's Ns lanes then
    // read them (the group lies in one warp)
    __shared__ __align__(16) float s_links[(kBS2 / NS) * kSL];
    float* my_links = s_links + (threadIdx.x / NS) * kSL;
    if (lane < 8) {
        float u[18];
        link_load_cs<LK>(P.links, ((size_t)p_out * P.g.Vh + h) * 8 + lane, u);
        float2* dst = reinterpret_cast<float2*>(my_links + lane * kLS);
#pragma unroll
        for (int k = 0; k < 9; ++k) dst[k] = make_float2(u[2 * k], u[2 * k + 1]);
    }
    __syncwarp();

    const void* in = P.in.d(sys);
    const float* in_n = P.in.n(sys);
    float2 AUr[3], AUi[3], ADr[3], ADi[3], ADSr[3], ADSi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) AUr[c] = AUi[c] = ADr[c] = ADi[c] = ADSr[c] = ADSi[c] = make_float2(0.f, 0.f);
    const float2* L2p = reinterpret_cast<const float2*>(my_links);
    // forward hops use (1 - gamma) for D and (1 + gamma) for D^dag; backward the opposite
    constexpr float SF = DAG ? 1.f : -1.f;
    // neighbour j + 1 is fetched before neighbour j is processed
    RawSite<SP> rs[2];
    fetch_site<SP>(in, in_n, (unsigned)nb[0], s, NS, rs[0]);
#define ODWF_HOP_DIR(MU_, DIR_)                                                                                   \
    {                                                                                                             \
        constexpr int j_ = 2 * MU_ + DIR_;                                                                        \
        if (j_ < 7) fetch_site<SP>(in, in_n, (unsigned)nb[j_ + 1 < 8 ? j_ + 1 : 7], s, NS, rs[(j_ + 1) & 1]);        \
        const float sgn_ = (flip & (1u << j_)) ? -1.f : 1.f;                                                     \
        const LinkStaged2 ls_{L2p + j_ * 9};                                                                      \
        hop_dir_packed<SP, MU_, DIR_ == 1>(rs[j_ & 1], sgn_, DIR_ == 0 ? SF : -SF, ls_, AUr, AUi, ADr, ADi, ADSr,  \
                                           ADSi);                                                                 \
    }
    ODWF_HOP_DIR(0, 0); ODWF_HOP_DIR(0, 1);
    ODWF_HOP_DIR(1, 0); ODWF_HOP_DIR(1, 1);
    ODWF_HOP_DIR(2, 0); ODWF_HOP_DIR(2, 1);
    ODWF_HOP_DIR(3, 0); ODWF_HOP_DIR(3, 1);
#undef ODWF_HOP_DIR
    // y = W psi (or W^dag psi) in pairs; the lower half gathers AD and the swapped ADS
    Half6 up, dn;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        up.R[c] = AUr[c];
        up.I[c] = AUi[c];
        dn.R[c] = __fadd2_rn(ADr[c], make_float2(ADSr[c].y, ADSr[c].x));
        dn.I[c] = __fadd2_rn(ADi[c], make_float2(ADSi[c].y, ADSi[c].x));
    }

    const Coef5<float>& cf = P.cf;
    float nrm = 0.f;  // per-thread partial sums in FP32, FP64 across warps and blocks (block_sum)
    float v[24];
    if (KIND == K1) {
        // chi_t = B M^-1 (-1/2 y)
        minv_pairs<NS>(up, dn, cf, r, s, false, -0.5f);
        bidiag_pairs<NS>(up, dn, cf.rho[s], cf.sigma[s], r, s, false);
        pairs_to_mem(up, dn, v);
        if (valid) SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s, NS, v);
    } else if (KIND == K2) {
        // s = p - M^-1 (-1/2 y) = p + M^-1 (y/2);  |s|^2;  a = M^-dag s
        minv_pairs<NS>(up, dn, cf, r, s, false, 0.5f);
        if (valid) {
            spinor_load_cs<SP, NS>(P.z.d(sys), P.z.n(sys), (size_t)h, s, v);
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] = 0.f;
        }
        Half6 zu, zd;
        mem_to_pairs(v, zu, zd);
        float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            up.p(k) = __fadd2_rn(up.p(k), zu.p(k));
            dn.p(k) = __fadd2_rn(dn.p(k), zd.p(k));
            n2 = fma2(up.p(k), up.p(k), n2);
            n2 = fma2(dn.p(k), dn.p(k), n2);
        }
        nrm = valid ? n2.x + n2.y : 0.f;  // a site past the end computed site 0's neighbours: no contribution
        minv_pairs<NS>(up, dn, cf, r, s, true, 1.f);
        pairs_to_mem(up, dn, v);
        if (valid) SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s, NS, v);
    } else if (KIND == K3) {
        // c = M^-dag (-1/2 B^dag y)
        bidiag_pairs<NS>(up, dn, cf.rho[s], cf.sigma[s], r, s, true);
        minv_pairs<NS>(up, dn, cf, r, s, true, -0.5f);
        pairs_to_mem(up, dn, v);
        if (valid) SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s, NS, v);
    } else {
        // A p = M^dag a + 1/2 B^dag y;  r -= alpha A p;  x += alpha p
        bidiag_pairs<NS>(up, dn, cf.rho[s], cf.sigma[s], r, s, true);
        if (valid) {
            spinor_load_cs<SP, NS>(P.z.d(sys), P.z.n(sys), (size_t)h, s, v);
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] = 0.f;
        }
        Half6 zu, zd;
        mem_to_pairs(v, zu, zd);
        bidiag_pairs<NS>(zu, zd, cf.d[s], cf.e[s], r, s, true);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            up.p(k) = fma2(f2(0.5f), up.p(k), zu.p(k));
            dn.p(k) = fma2(f2(0.5f), dn.p(k), zd.p(k));
        }
        pairs_to_mem(up, dn, v);  // v = A p
        const float alpha = (float)P.st[sys].alpha;
        if (valid) {
            float rv[24], xv[24], pv[24];
            spinor_load_cs<SpF32, NS>(P.cg_r.d(sys), nullptr, (size_t)h, s, rv);
            spinor_load_cs<SpF32, NS>(P.cg_x.d(sys), nullptr, (size_t)h, s, xv);
            spinor_load_cs<SP, NS>(P.cg_p.d(sys), P.cg_p.n(sys), (size_t)h, s, pv);
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                rv[k] = fmaf(-alpha, v[k], rv[k]);
                xv[k] = fmaf(alpha, pv[k], xv[k]);
                nrm = fmaf(rv[k], rv[k], nrm);
            }
            f32_store_cs<NS>(P.cg_r.d(sys), (size_t)h, s, rv);
            f32_store_cs<NS>(P.cg_x.d(sys), (size_t)h, s, xv);
        }
    }
    if (KIND == K2) reduce_and_finalize(nrm, P.partials, P.counters, P.st, sys, FIN_ALPHA, P.part_stride);
    if (KIND == K4) reduce_and_finalize(nrm, P.partials, P.counters, P.st, sys, FIN_BETA, P.part_stride);
}

// p = r + beta p (mode 1) or p = r (mode 0);  chi = B p.  One thread per (site, s), lane groups of NS.
template <class SP, int NS>
__global__ void __launch_bounds__(kBS2) p_update2_kernel(FieldRef rr, FieldRef pp, FieldRef chi, size_t n_sites,
                                                          int mode, Coef5<float> cf, const double* r_sys,
                                                          SysState* st, int gate, int need, int sys_base,
                                                          unsigned long long* prof_count) {
    const int sys = blockIdx.y + sys_base;
    if (gate && st[sys].status != need) return;
    if (prof_count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof_count, 1ull);
    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = (int)(gi & (NS - 1));
    const size_t h = gi / NS;
    const bool valid = h < n_sites;
    float v[24];
    if (valid) {
        SpinorIO<SpF32, float>::load(rr.d(sys), nullptr, h, s, NS, v);
        if (mode == 1) {
            const float beta = (float)st[sys].beta;
            float pv[24];
            SpinorIO<SP, float>::load(pp.d(sys), pp.n(sys), h, s, NS, pv);
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] = fmaf(beta, pv[k], v[k]);
        }
        SpinorIO<SP, float>::store(pp.d(sys), pp.n(sys), h, s, NS, v);
    } else {
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = 0.f;
    }
    // chi = B p, from the stored (rounded) p so that chi matches the p the hops see
    if (valid) SpinorIO<SP, float>::load(pp.d(sys), pp.n(sys), h, s, NS, v);
    bidiag_apply(v, cf.rho[s], cf.sigma[s], (float)r_sys[sys], s, NS, false);
    if (valid) SpinorIO<SP, float>::store(chi.d(sys), chi.n(sys), h, s, NS, v);
}

template <class SP, class LK, int NS>
cudaError_t hop2_k(const HopParams<float>& P, int kind, int nsys, cudaStream_t st) {
    const size_t n = (size_t)P.g.Vh * NS;
    dim3 grid(blocks_for(n, kBS2), nsys);
    note_launch();
    switch (kind) {
        case K1: hop2_kernel<SP, LK, NS, K1><<<grid, kBS2, 0, st>>>(P); break;
        case K2: hop2_kernel<SP, LK, NS, K2><<<grid, kBS2, 0, st>>>(P); break;
        case K3: hop2_kernel<SP, LK, NS, K3><<<grid, kBS2, 0, st>>>(P); break;
        default: hop2_kernel<SP, LK, NS, K4><<<grid, kBS2, 0, st>>>(P); break;
    }
    return cudaGetLastError();
}

template <class SP, class LK>
cudaError_t hop2_ns(const HopParams<float>& P, int kind, int nsys, cudaStream_t st) {
    switch (P.ns) {
        case 8: return hop2_k<SP, LK, 8>(P, kind, nsys, st);
        case 16: return hop2_k<SP, LK, 16>(P, kind, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

template <class SP>
cudaError_t hop2_lk(const HopParams<float>& P, int kind, Lk lk, int nsys, cudaStream_t st) {
    switch (lk) {
        case Lk::F12: return hop2_ns<SP, LinkF12>(P, kind, nsys, st);
        case Lk::F18: return hop2_ns<SP, LinkF18>(P, kind, nsys, st);
        case Lk::H12: return hop2_ns<SP, LinkH12>(P, kind, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

template <class SP, int NS>
cudaError_t pupd_k(const FieldRef& r, const FieldRef& p, const FieldRef& chi, size_t n_sites, int mode,
                   const Coef5<float>& cf, const double* r_sys, SysState* st, int gate, int need, int sys_base,
                   int nsys, unsigned long long* prof, cudaStream_t stream) {
    dim3 grid(blocks_for(n_sites * NS, kBS2), nsys);
    note_launch();
    p_update2_kernel<SP, NS><<<grid, kBS2, 0, stream>>>(r, p, chi, n_sites, mode, cf, r_sys, st, gate, need,
                                                         sys_base, prof);
    return cudaGetLastError();
}

template <class SP>
cudaError_t pupd_ns(int ns, const FieldRef& r, const FieldRef& p, const FieldRef& chi, size_t n_sites, int mode,
                    const Coef5<float>& cf, const double* r_sys, SysState* st, int gate, int need, int sys_base,
                    int nsys, unsigned long long* prof, cudaStream_t stream) {
    switch (ns) {
        case 8: return pupd_k<SP, 8>(r, p, chi, n_sites, mode, cf, r_sys, st, gate, need, sys_base, nsys, prof, stream);
        case 16: return pupd_k<SP, 16>(r, p, chi, n_sites, mode, cf, r_sys, st, gate, need, sys_base, nsys, prof, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool hop2_supported(int ns, Sp low, size_t vh) {
    // 32-bit chunk indices: a half field must have fewer than 2^32 16-byte chunks
    const size_t chunks = vh * (size_t)ns * (low == Sp::F32 ? 6 : 3);
    return (ns == 8 || ns == 16) && (low == Sp::F16 || low == Sp::BF16 || low == Sp::F32) && chunks < (1ull << 32);
}

cudaError_t launch_hop2(const HopParams<float>& P, int kind, Sp low, Lk lk, int nsys, cudaStream_t st) {
    switch (low) {
        case Sp::F16: return hop2_lk<SpF16>(P, kind, lk, nsys, st);
        case Sp::BF16: return hop2_lk<SpBF16>(P, kind, lk, nsys, st);
        case Sp::F32: return hop2_lk<SpF32>(P, kind, lk, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_p_update2(Sp low, int ns, const FieldRef& r, const FieldRef& p, const FieldRef& chi,
                             size_t n_sites, int mode, const Coef5<float>& cf, const double* r_sys, SysState* st,
                             int gate, int need, int sys_base, int nsys, unsigned long long* prof,
                             cudaStream_t stream) {
    switch (low) {
        case Sp::F16: return pupd_ns<SpF16>(ns, r, p, chi, n_sites, mode, cf, r_sys, st, gate, need, sys_base, nsys, prof, stream);
        case Sp::BF16: return pupd_ns<SpBF16>(ns, r, p, chi, n_sites, mode, cf, r_sys, st, gate, need, sys_base, nsys, prof, stream);
        case Sp::F32: return pupd_ns<SpF32>(ns, r, p, chi, n_sites, mode, cf, r_sys, st, gate, need, sys_base, nsys, prof, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace odwf
