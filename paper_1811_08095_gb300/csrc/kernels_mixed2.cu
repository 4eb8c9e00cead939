// Mixed-precision CG kernels, second generation (Ns = 8, 16; FP16 / BF16 / FP32 storage).
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

#include "kernels.cuh"
#include "kernels.h"

namespace odwf {

namespace {

constexpr int kBS2 = 256;

enum { K1 = 1, K2 = 2, K3 = 3, K4 = 4 };

// ---------------------------------------------------------------- packed FP32 pairs
// A "spin pair" holds one colour and one real/imaginary part of the two spins of a
// chirality half: R[c] = (spin_a.re, spin_b.re), I[c] = (spin_a.im, spin_b.im).  Pair
// arithmetic uses the FP32x2 FMA of sm_100+ (one instruction for two lanes of work).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Raw stored words of one 5D site (fetched ahead of use so that the next neighbour's loads
// are in flight while the current one is processed) and their unpacking into spin pairs:
// up half (spins 0, 1) and down half (spins 2, 3; in the order (3, 2) when SWAP_DN).
template <class SP>
struct RawSite;
template <>
struct RawSite<SpF16> { uint4 q[3]; float sc; };
template <>
struct RawSite<SpBF16> { uint4 q[3]; float sc; };
template <>
struct RawSite<SpF32> { float4 q[6]; float sc; };

// 32-bit chunk index of (h, s): h * nch * ns + s (hop2_supported bounds the field size).
// Threads past the last site load site 0's neighbours (valid addresses) and store nothing.
template <class SP>
__device__ __forceinline__ void fetch_site(const void* base, const float* norm, unsigned h, int s, int ns,
                                           RawSite<SP>& r) {
    if (std::is_same<SP, SpF32>::value) {
        const float4* p = reinterpret_cast<const float4*>(base) + (h * (6u * ns) + (unsigned)s);
        float4* q = reinterpret_cast<float4*>(&r);
#pragma unroll
        for (int k = 0; k < 6; ++k) q[k] = __ldg(p + k * ns);
        r.sc = 1.f;
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(base) + (h * (3u * ns) + (unsigned)s);
        uint4* q = reinterpret_cast<uint4*>(&r);
#pragma unroll
        for (int k = 0; k < 3; ++k) q[k] = __ldg(p + k * ns);
        r.sc = __ldg(norm + (h * (unsigned)ns + (unsigned)s));
    }
}

template <class SP, bool SWAP_DN>
__device__ __forceinline__ void unpack_site(const RawSite<SP>& r, float2 Ur[3], float2 Ui[3], float2 Dr[3],
                                            float2 Di[3]) {
    float2 f[12];  // word w = (spin w/3, colour w%3): (re, im)
    if (std::is_same<SP, SpF32>::value) {
        const float* v = reinterpret_cast<const float*>(&r);
#pragma unroll
        for (int w = 0; w < 12; ++w) f[w] = make_float2(v[2 * w], v[2 * w + 1]);
    } else {
        using H2 = typename std::conditional<std::is_same<SP, SpF16>::value, __half2, __nv_bfloat162>::type;
        const uint32_t* wd = reinterpret_cast<const uint32_t*>(&r);
#pragma unroll
        for (int w = 0; w < 12; ++w) {
            H2 hv;
            *reinterpret_cast<uint32_t*>(&hv) = wd[w];
            f[w] = Half2Cvt<H2>::to_f2(hv);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ur[c] = make_float2(f[c].x, f[3 + c].x);
        Ui[c] = make_float2(f[c].y, f[3 + c].y);
        if (SWAP_DN) {
            Dr[c] = make_float2(f[9 + c].x, f[6 + c].x);
            Di[c] = make_float2(f[9 + c].y, f[6 + c].y);
        } else {
            Dr[c] = make_float2(f[6 + c].x, f[9 + c].x);
            Di[c] = make_float2(f[6 + c].y, f[9 + c].y);
        }
    }
}

// One hop direction in spin pairs.  H = v^up + sg G v^dn (G of gamma_mu in the chiral basis,
// gamma_mu = [[0, G], [G^dag, 0]]); W = U H (or U^dag H); then
//   AU += sc W,  lower spins += sg sc G^dag W,
// accumulated in AD (order (2, 3)) for mu = 2, 3 and in ADS (order (3, 2)) for mu = 0, 1, so
// that no pair ever needs its halves exchanged.  The link source returns element (a, b) of U
// as the broadcast pairs (ur, ur), (ui, ui).
// Link source for hop_dir_packed: nine float2 (ur, ui) in shared memory, element (a, b) at
// index 3a + b, returned as the broadcast pairs (ur, ur), (ui, ui) that the spin-pair FMAs need.
struct LinkStaged2 {
    const float2* q;
    __device__ __forceinline__ void get(int a, int b, float2& ur, float2& ui) const {
        const float2 v = q[3 * a + b];
        ur = make_float2(v.x, v.x);
        ui = make_float2(v.y, v.y);
    }
};
template <class SP, int MU, bool DAGU, class LF>
__device__ __forceinline__ void hop_dir_packed(const RawSite<SP>& raw, float sc_sign, float sg, const LF& lnk,
                                               float2 AUr[3], float2 AUi[3], float2 ADr[3], float2 ADi[3],
                                               float2 ADSr[3], float2 ADSi[3]) {
    constexpr bool SW = (MU == 0 || MU == 1);
    float2 Ur[3], Ui[3], Dr[3], Di[3];
    unpack_site<SP, SW>(raw, Ur, Ui, Dr, Di);
    const float sc = raw.sc * sc_sign;
    // projection
    float2 Hr[3], Hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) {          // G = -i s1:  G d = -i (d1, d0)
            Hr[c] = fma2(Di[c], make_float2(sg, sg), Ur[c]);
            Hi[c] = fma2(Dr[c], make_float2(-sg, -sg), Ui[c]);
        } else if (MU == 1) {   // G = -i s2:  G d = (-d1, d0)
            Hr[c] = fma2(Dr[c], make_float2(-sg, sg), Ur[c]);
            Hi[c] = fma2(Di[c], make_float2(-sg, sg), Ui[c]);
        } else if (MU == 2) {   // G = -i s3:  G d = (-i d0, i d1)
            Hr[c] = fma2(Di[c], make_float2(sg, -sg), Ur[c]);
            Hi[c] = fma2(Dr[c], make_float2(-sg, sg), Ui[c]);
        } else {                // G = 1
            Hr[c] = fma2(Dr[c], make_float2(sg, sg), Ur[c]);
            Hi[c] = fma2(Di[c], make_float2(sg, sg), Ui[c]);
        }
    }
    // SU(3) product
    float2 Nh[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Nh[c] = DAGU ? make_float2(-Hr[c].x, -Hr[c].y) : make_float2(-Hi[c].x, -Hi[c].y);
    float2 Wr[3], Wi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Wr[a] = make_float2(0.f, 0.f);
        Wi[a] = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float2 ur, ui;
            if (DAGU) lnk.get(b, a, ur, ui); else lnk.get(a, b, ur, ui);
            if (!DAGU) {
                Wr[a] = fma2(ur, Hr[b], fma2(ui, Nh[b], Wr[a]));
                Wi[a] = fma2(ur, Hi[b], fma2(ui, Hr[b], Wi[a]));
            } else {
                Wr[a] = fma2(ur, Hr[b], fma2(ui, Hi[b], Wr[a]));
                Wi[a] = fma2(ur, Hi[b], fma2(ui, Nh[b], Wi[a]));
            }
        }
    }
    // accumulation
    const float m = sc, md = sg * sc;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        AUr[a] = fma2(make_float2(m, m), Wr[a], AUr[a]);
        AUi[a] = fma2(make_float2(m, m), Wi[a], AUi[a]);
        if (MU == 0) {          // G^dag = i s1: lower (3, 2) order = i W
            ADSr[a] = fma2(make_float2(-md, -md), Wi[a], ADSr[a]);
            ADSi[a] = fma2(make_float2(md, md), Wr[a], ADSi[a]);
        } else if (MU == 1) {   // G^dag = [[0, 1], [-1, 0]]: lower (3, 2) order = W (-1, 1)
            ADSr[a] = fma2(make_float2(-md, md), Wr[a], ADSr[a]);
            ADSi[a] = fma2(make_float2(-md, md), Wi[a], ADSi[a]);
        } else if (MU == 2) {   // G^dag = i s3: lower = (i w0, -i w1)
            ADr[a] = fma2(make_float2(-md, md), Wi[a], ADr[a]);
            ADi[a] = fma2(make_float2(md, -md), Wr[a], ADi[a]);
        } else {                // G^dag = 1
            ADr[a] = fma2(make_float2(md, md), Wr[a], ADr[a]);
            ADi[a] = fma2(make_float2(md, md), Wi[a], ADi[a]);
        }
    }
}

// ---------------------------------------------------------------- fifth-dimension epilogue on spin pairs
// One chirality half of a 5D site in the hop's own register layout: for colour c,
// R[c] = (spin_a.re, spin_b.re), I[c] = (spin_a.im, spin_b.im); up = spins (0, 1), down = (2, 3).
// The fifth-dimension operators act identically on all twelve reals of a chirality, so they run
// on these pairs directly (packed FMAs, no repacking into memory order).
struct Half6 {
    float2 R[3], I[3];
    __device__ __forceinline__ float2& p(int k) { return k < 3 ? R[k] : I[k - 3]; }
};

__device__ __forceinline__ float2 shfl2_idx(float2 v, int src, int w) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src, w), __shfl_sync(0xffffffffu, v.y, src, w));
}
__device__ __forceinline__ float2 shfl2_up(float2 v, int d, int w) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d, w), __shfl_up_sync(0xffffffffu, v.y, d, w));
}
__device__ __forceinline__ float2 shfl2_down(float2 v, int d, int w) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d, w), __shfl_down_sync(0xffffffffu, v.y, d, w));
}
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Bidiagonal X = diag(a) + diag(b) L (dag = false) or its adjoint a + L^dag b (dag = true) on both
// chiralities (L: up from s-1, down from s+1, corners -r; L^dag the reverse), as bidiag_apply.
template <int NS>
__device__ __forceinline__ void bidiag_pairs(Half6& up, Half6& dn, float a_s, float b_s, float r, int s, bool dag) {
    const int sm = (s + NS - 1) & (NS - 1), sp = (s + 1) & (NS - 1);
    if (!dag) {
        const float2 cm = f2(s == 0 ? -r * b_s : b_s), cp = f2(s == NS - 1 ? -r * b_s : b_s);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 u = shfl2_idx(up.p(k), sm, NS), d = shfl2_idx(dn.p(k), sp, NS);
            up.p(k) = fma2(f2(a_s), up.p(k), __fmul2_rn(cm, u));
            dn.p(k) = fma2(f2(a_s), dn.p(k), __fmul2_rn(cp, d));
        }
    } else {
        const float2 cu = f2(s == NS - 1 ? -r : 1.f), cd = f2(s == 0 ? -r : 1.f);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 u = shfl2_idx(__fmul2_rn(f2(b_s), up.p(k)), sp, NS);
            const float2 d = shfl2_idx(__fmul2_rn(f2(b_s), dn.p(k)), sm, NS);
            up.p(k) = fma2(cu, u, __fmul2_rn(f2(a_s), up.p(k)));
            dn.p(k) = fma2(cd, d, __fmul2_rn(f2(a_s), dn.p(k)));
        }
    }
}

// Cyclic bidiagonal solve along s of pre * v on one chirality (six pairs), as cyclic_solve12:
//   forward:  d_s w_s + c_s w_{s-1} = pre v_s,  w_{-1} := -r w_{Ns-1}
//   backward: d_s w_s + c_s w_{s+1} = pre v_s,  w_{Ns} := -r w_0
template <int NS>
__device__ __forceinline__ void cyclic_pairs(Half6& v, float pre, float inv_d, float c_s, float r, int s, bool fwd) {
    float coef = -c_s * inv_d;
    const float2 sc = f2(pre * inv_d);
#pragma unroll
    for (int k = 0; k < 6; ++k) v.p(k) = __fmul2_rn(sc, v.p(k));
    const int q = fwd ? s : NS - 1 - s;
#pragma unroll
    for (int off = 1; off < NS; off <<= 1) {
        const float pc = fwd ? __shfl_up_sync(0xffffffffu, coef, off, NS) : __shfl_down_sync(0xffffffffu, coef, off, NS);
        const float2 cm = f2(q >= off ? coef : 0.f);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 pv = fwd ? shfl2_up(v.p(k), off, NS) : shfl2_down(v.p(k), off, NS);
            v.p(k) = fma2(cm, pv, v.p(k));
        }
        if (q >= off) coef *= pc;
    }
    const int last = fwd ? NS - 1 : 0;
    const float Al = __shfl_sync(0xffffffffu, coef, last, NS);
    const float2 cf = f2(coef * (-r / (1.f + r * Al)));
#pragma unroll
    for (int k = 0; k < 6; ++k) v.p(k) = fma2(cf, shfl2_idx(v.p(k), last, NS), v.p(k));
}

// M^-1 (dag = false) or M^-dag (dag = true) of pre * v, as minv_apply
template <int NS>
__device__ __forceinline__ void minv_pairs(Half6& up, Half6& dn, const Coef5<float>& cf, float r, int s, bool dag,
                                           float pre) {
    const float inv_d = cf.inv_d[s];
    if (!dag) {
        cyclic_pairs<NS>(up, pre, inv_d, cf.e[s], r, s, true);
        cyclic_pairs<NS>(dn, pre, inv_d, cf.e[s], r, s, false);
    } else {
        cyclic_pairs<NS>(up, pre, inv_d, cf.e[(s + 1) & (NS - 1)], r, s, false);
        cyclic_pairs<NS>(dn, pre, inv_d, cf.e[(s + NS - 1) & (NS - 1)], r, s, true);
    }
}

// Fields a kernel touches once per site (the CG vectors r, x, p and the z operand) are read and
// written with the evict-first (streaming) cache policy, so that they do not push the neighbour
// field, which each site's eight neighbours read again, out of L2.
template <class SP, int NS>
__device__ __forceinline__ void spinor_load_cs(const void* base, const float* norm, size_t h, int s, float v[24]) {
    if (std::is_same<SP, SpF32>::value) {
        const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 q = __ldcs(p + chunk_off(h, k, 6, NS, s));
            v[4 * k] = q.x;
            v[4 * k + 1] = q.y;
            v[4 * k + 2] = q.z;
            v[4 * k + 3] = q.w;
        }
    } else {
        using H2 = typename std::conditional<std::is_same<SP, SpF16>::value, __half2, __nv_bfloat162>::type;
        const uint4* p = reinterpret_cast<const uint4*>(base);
        const float sc = __ldcs(norm + h * NS + s);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 q = __ldcs(p + chunk_off(h, k, 3, NS, s));
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                H2 hv;
                *reinterpret_cast<uint32_t*>(&hv) = w[j];
                const float2 f = Half2Cvt<H2>::to_f2(hv);
                v[8 * k + 2 * j] = f.x * sc;
                v[8 * k + 2 * j + 1] = f.y * sc;
            }
        }
    }
}

// The site-major link array is also read exactly once per launch (the eight links of a site).
template <class LK>
__device__ __forceinline__ void link_load_cs(const void* base, size_t idx, float u[18]) {
    if (std::is_same<LK, LinkF12>::value) {
        const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) + idx * 48);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 q = __ldcs(p + k);
            u[4 * k] = q.x; u[4 * k + 1] = q.y; u[4 * k + 2] = q.z; u[4 * k + 3] = q.w;
        }
        su3_third_row(u);
    } else if (std::is_same<LK, LinkH12>::value) {
        const uint2* p = reinterpret_cast<const uint2*>(reinterpret_cast<const char*>(base) + idx * 24);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 q = __ldcs(p + k);
            __half2 a, b;
            *reinterpret_cast<uint32_t*>(&a) = q.x;
            *reinterpret_cast<uint32_t*>(&b) = q.y;
            const float2 fa = __half22float2(a), fb = __half22float2(b);
            u[4 * k] = fa.x; u[4 * k + 1] = fa.y; u[4 * k + 2] = fb.x; u[4 * k + 3] = fb.y;
        }
        su3_third_row(u);
    } else {
        const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) + idx * 80);
        float t[20];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float4 q = __ldcs(p + k);
            t[4 * k] = q.x; t[4 * k + 1] = q.y; t[4 * k + 2] = q.z; t[4 * k + 3] = q.w;
        }
#pragma unroll
        for (int k = 0; k < 18; ++k) u[k] = t[k];
    }
}

template <int NS>
__device__ __forceinline__ void f32_store_cs(void* base, size_t h, int s, const float v[24]) {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k)
        __stcs(p + chunk_off(h, k, 6, NS, s), make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
}

// memory order [spin][colour][re, im] <-> pairs
__device__ __forceinline__ void pairs_to_mem(const Half6& up, const Half6& dn, float v[24]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[2 * c] = up.R[c].x;
        v[2 * c + 1] = up.I[c].x;
        v[6 + 2 * c] = up.R[c].y;
        v[6 + 2 * c + 1] = up.I[c].y;
        v[12 + 2 * c] = dn.R[c].x;
        v[12 + 2 * c + 1] = dn.I[c].x;
        v[18 + 2 * c] = dn.R[c].y;
        v[18 + 2 * c + 1] = dn.I[c].y;
    }
}
__device__ __forceinline__ void mem_to_pairs(const float v[24], Half6& up, Half6& dn) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        up.R[c] = make_float2(v[2 * c], v[6 + 2 * c]);
        up.I[c] = make_float2(v[2 * c + 1], v[6 + 2 * c + 1]);
        dn.R[c] = make_float2(v[12 + 2 * c], v[18 + 2 * c]);
        dn.I[c] = make_float2(v[12 + 2 * c + 1], v[18 + 2 * c + 1]);
    }
}

template <class SP, class LK, int NS, int KIND>
__global__ void __launch_bounds__(kBS2, 3) hop2_kernel(const HopParams<float> P) {
    constexpr int kLS = 18;            // floats per staged link: 9 x (ur, ui)
    constexpr int kSL = 8 * kLS + 4;   // floats per site (padding spreads banks)
    constexpr bool DAG = (KIND == K3 || KIND == K4);
    const int sys = blockIdx.y + P.sys_base;
    if (P.gate && P.st[sys].status != P.need_status) return;
    if (P.prof_count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(P.prof_count, 1ull);

    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = (int)(gi & (NS - 1));
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
            nb[j] = raw[j] & 0x7fffffff;
            flip |= ((unsigned)raw[j] >> 31) << j;
        }
    }

    // stage the site's eight links in shared memory as (ur, ui) pairs: lane d < 8 of the group
    // loads direction d from the site-major link array (the eight links of a site are contiguous,
    // so the loads neither wait for the neighbour table nor scatter); the group's Ns lanes then
    // read them (the group lies in one warp)
    __shared__ __align__(16) float s_links[(kBS2 / NS) * kSL];
    float* my_links = s_links + (threadIdx.x / NS) * kSL;
    if (s < 8) {
        float u[18];
        link_load_cs<LK>(P.links, ((size_t)p_out * P.g.Vh + h) * 8 + s, u);
        float2* dst = reinterpret_cast<float2*>(my_links + s * kLS);
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
    if (KIND == K2) reduce_and_finalize(nrm, P.partials, P.counters, P.st, sys, FIN_ALPHA);
    if (KIND == K4) reduce_and_finalize(nrm, P.partials, P.counters, P.st, sys, FIN_BETA);
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
