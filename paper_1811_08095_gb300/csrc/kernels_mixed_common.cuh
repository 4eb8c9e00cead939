// Device building blocks shared by the production mixed-precision hop kernels (kernels_mixed2.cu:
// one s per lane; kernels_mixed3.cu: two adjacent s per lane): the FP16/BF16/FP32 neighbour
// fetch, one hop direction on FP32x2 spin pairs, link staging, the fifth-dimension operators on
// spin pairs, and loads/stores with the streaming cache policy.
#pragma once

#include <type_traits>

#include "kernels.cuh"
#include "kernels.h"

namespace odwf {
namespace mx {

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

// 32-bit chunk index of (h, s): h * nch * ns + slot(s) (hop2_supported bounds the field size).
// Threads past the last site load site 0's neighbours (valid addresses) and store nothing.
template <class SP>
__device__ __forceinline__ void fetch_site(const void* base, const float* norm, unsigned h, int s, int ns,
                                           RawSite<SP>& r) {
    if (std::is_same<SP, SpF32>::value) {
        const float4* p = reinterpret_cast<const float4*>(base) + (h * (6u * ns) + (unsigned)chunk_slot(s, ns));
        float4* q = reinterpret_cast<float4*>(&r);
#pragma unroll
        for (int k = 0; k < 6; ++k) q[k] = __ldg(p + k * ns);
        r.sc = 1.f;
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(base) + (h * (3u * ns) + (unsigned)chunk_slot(s, ns));
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
// Spin projection of one direction: H = v^up + sg G v^dn on spin pairs (G of gamma_mu in the
// chiral basis; the down pair comes in the order (3, 2) for mu = 0, 1, see unpack_site).
template <int MU>
__device__ __forceinline__ void project_pairs(const float2 Ur[3], const float2 Ui[3], const float2 Dr[3],
                                              const float2 Di[3], float sg, float2 Hr[3], float2 Hi[3]) {
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
}

// Row a of W = U H (or U^dag H): W_a = sum_b U_ab H_b, with the link element as broadcast pairs;
// Nh = -Hi (U) or -Hr (U^dag) supplies the sign of the imaginary cross term.
template <bool DAGU>
__device__ __forceinline__ void su3_row_acc(float2 ur, float2 ui, float2 Hr, float2 Hi, float2 Nh, float2& Wr,
                                            float2& Wi) {
    if (!DAGU) {
        Wr = fma2(ur, Hr, fma2(ui, Nh, Wr));
        Wi = fma2(ur, Hi, fma2(ui, Hr, Wi));
    } else {
        Wr = fma2(ur, Hr, fma2(ui, Hi, Wr));
        Wi = fma2(ur, Hi, fma2(ui, Nh, Wi));
    }
}

// Accumulate row a of W, scaled by m (upper spins) and md = sg m (lower spins, sg G^dag W).
template <int MU>
__device__ __forceinline__ void accumulate_row(float m, float md, float2 Wr, float2 Wi, float2& AUr, float2& AUi,
                                               float2& ADr, float2& ADi, float2& ADSr, float2& ADSi) {
    AUr = fma2(make_float2(m, m), Wr, AUr);
    AUi = fma2(make_float2(m, m), Wi, AUi);
    if (MU == 0) {          // G^dag = i s1: lower (3, 2) order = i W
        ADSr = fma2(make_float2(-md, -md), Wi, ADSr);
        ADSi = fma2(make_float2(md, md), Wr, ADSi);
    } else if (MU == 1) {   // G^dag = [[0, 1], [-1, 0]]: lower (3, 2) order = W (-1, 1)
        ADSr = fma2(make_float2(-md, md), Wr, ADSr);
        ADSi = fma2(make_float2(-md, md), Wi, ADSi);
    } else if (MU == 2) {   // G^dag = i s3: lower = (i w0, -i w1)
        ADr = fma2(make_float2(-md, md), Wi, ADr);
        ADi = fma2(make_float2(md, -md), Wr, ADi);
    } else {                // G^dag = 1
        ADr = fma2(make_float2(md, md), Wr, ADr);
        ADi = fma2(make_float2(md, md), Wi, ADi);
    }
}

template <class SP, int MU, bool DAGU, class LF>
__device__ __forceinline__ void hop_dir_packed(const RawSite<SP>& raw, float sc_sign, float sg, const LF& lnk,
                                               float2 AUr[3], float2 AUi[3], float2 ADr[3], float2 ADi[3],
                                               float2 ADSr[3], float2 ADSi[3]) {
    constexpr bool SW = (MU == 0 || MU == 1);
    float2 Ur[3], Ui[3], Dr[3], Di[3];
    unpack_site<SP, SW>(raw, Ur, Ui, Dr, Di);
    const float sc = raw.sc * sc_sign;
    float2 Hr[3], Hi[3], Nh[3];
    project_pairs<MU>(Ur, Ui, Dr, Di, sg, Hr, Hi);
#pragma unroll
    for (int c = 0; c < 3; ++c) Nh[c] = DAGU ? make_float2(-Hr[c].x, -Hr[c].y) : make_float2(-Hi[c].x, -Hi[c].y);
    // all three rows of W first, then the accumulation (this order keeps hop2's registers lowest)
    float2 Wr[3], Wi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Wr[a] = make_float2(0.f, 0.f);
        Wi[a] = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float2 ur, ui;
            if (DAGU) lnk.get(b, a, ur, ui); else lnk.get(a, b, ur, ui);
            su3_row_acc<DAGU>(ur, ui, Hr[b], Hi[b], Nh[b], Wr[a], Wi[a]);
        }
    }
    const float m = sc, md = sg * sc;
#pragma unroll
    for (int a = 0; a < 3; ++a) accumulate_row<MU>(m, md, Wr[a], Wi[a], AUr[a], AUi[a], ADr[a], ADi[a], ADSr[a], ADSi[a]);
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

// In these one-s-per-lane operators the lane holding s is chunk_slot(s, Ns) (lanes read the
// spinor slots in order, so a quarter warp's loads stay within one 128-byte line), so every
// exchange along s names its source lane through chunk_slot.
__device__ __forceinline__ int lane_of(int s, int ns) { return chunk_slot(s, ns); }
// s held by lane i of a site's group (inverse of lane_of)
__device__ __forceinline__ int s_of_lane(int i, int ns) { return i < (ns >> 1) ? 2 * i : 2 * (i - (ns >> 1)) + 1; }

// Bidiagonal X = diag(a) + diag(b) L (dag = false) or its adjoint a + L^dag b (dag = true) on both
// chiralities (L: up from s-1, down from s+1, corners -r; L^dag the reverse), as bidiag_apply.
template <int NS>
__device__ __forceinline__ void bidiag_pairs(Half6& up, Half6& dn, float a_s, float b_s, float r, int s, bool dag) {
    const int sm = lane_of((s + NS - 1) & (NS - 1), NS), sp = lane_of((s + 1) & (NS - 1), NS);
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
        // the lane holding s - off (forward) or s + off (backward); unused where q < off
        const int src = lane_of(fwd ? ((s - off) & (NS - 1)) : ((s + off) & (NS - 1)), NS);
        const float pc = __shfl_sync(0xffffffffu, coef, src, NS);
        const float2 cm = f2(q >= off ? coef : 0.f);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 pv = shfl2_idx(v.p(k), src, NS);
            v.p(k) = fma2(cm, pv, v.p(k));
        }
        if (q >= off) coef *= pc;
    }
    const int last = lane_of(fwd ? NS - 1 : 0, NS);
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


}  // namespace mx
}  // namespace odwf
