// Internal definitions of the GB300 ODWF library: geometry, storage formats, and the
// per-lane building blocks of the fused hopping kernel.
//
// Work decomposition used by every kernel: one thread per (4D site, s).  The Ns
// threads of a 4D site are consecutive lanes of one warp (Ns divides 32), so
// operations along the fifth dimension -- the chiral shift B = rho + sigma L of
// Sec. 2's operator, the site-local M = (4-m0) B + 1 - L, its adjoint and its
// inverse -- run as register shuffles inside the Ns-lane group.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ff.cuh"

namespace odwf {

constexpr int kMaxNs = 32;

// ---------------------------------------------------------------- geometry
struct Geom {
    int L[4];  // Lx, Ly, Lz, Lt (all even)
    int Lxh;   // Lx / 2
    int Vh;    // half volume
    int tbc;   // 1: antiperiodic time boundary
};

// coordinates of half-site h of parity p (lex = x + Lx (y + Ly (z + Lz t)), lex/2 = h)
__device__ __forceinline__ void site_coords(const Geom& g, int p, int h, int c[4]) {
    const int xh = h % g.Lxh;
    int rest = h / g.Lxh;
    c[1] = rest % g.L[1];
    rest /= g.L[1];
    c[2] = rest % g.L[2];
    c[3] = rest / g.L[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

__device__ __forceinline__ int half_index(const Geom& g, const int c[4]) {
    return (c[0] >> 1) + g.Lxh * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

// ---------------------------------------------------------------- fifth-dimension coefficients
// M = diag(d) + diag(e) L with d_s = (4-m0) rho_s + 1, e_s = (4-m0) sigma_s - 1;
// B = diag(rho) + diag(sigma) L.  Only the corner of L depends on the mass (r).
template <class R>
struct Coef5 {
    R rho[kMaxNs], sigma[kMaxNs], d[kMaxNs], e[kMaxNs], inv_d[kMaxNs];
};

// ---------------------------------------------------------------- storage formats
// Spinor half field: 24 reals per 5D site in the order [spin][colour][re,im]
// (spins 0, 1 = P_+ "up", 2, 3 = P_- "down"), stored chunked so that the lanes of a site read
// consecutive 16-byte words: byte address of chunk k of (h, s) is
//   ((h * NCH + k) * Ns + slot(s)) * 16,   slot(s) = s / 2 (s even), Ns / 2 + s / 2 (s odd).
// The slot order puts the even s of a site first and the odd s second, so that kernels whose
// lane l holds the adjacent pair s = 2l, 2l + 1 read two runs of consecutive words, as kernels
// with one s per lane read one.  Half-precision formats carry one FP32 scale per 5D site,
// value = stored * scale, at norm[h * Ns + s] (not permuted).
struct SpF64 { using T = double; static constexpr int NCH = 12; static constexpr bool kNorm = false; };
struct SpF32 { using T = float; static constexpr int NCH = 6; static constexpr bool kNorm = false; };
struct SpF16 { using T = __half; static constexpr int NCH = 3; static constexpr bool kNorm = true; };
struct SpBF16 { using T = __nv_bfloat16; static constexpr int NCH = 3; static constexpr bool kNorm = true; };

template <class SP>
__host__ __device__ constexpr size_t spinor_bytes(size_t sites5) { return sites5 * SP::NCH * 16; }

__host__ __device__ __forceinline__ int chunk_slot(int s, int ns) { return (s & 1) * (ns >> 1) + (s >> 1); }

__device__ __forceinline__ size_t chunk_off(size_t h, int k, int nch, int ns, int s) {
    return ((h * nch + k) * (size_t)ns + chunk_slot(s, ns));
}

template <class SP, class R>
struct SpinorIO;

template <class R>
struct SpinorIO<SpF64, R> {
    static __device__ __forceinline__ void load(const void* base, const float*, size_t h, int s, int ns, R v[24]) {
        const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 q = __ldg(p + chunk_off(h, k, 12, ns, s));
            v[2 * k] = (R)q.x;
            v[2 * k + 1] = (R)q.y;
        }
    }
    static __device__ __forceinline__ void store(void* base, float*, size_t h, int s, int ns, const R v[24]) {
        double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[chunk_off(h, k, 12, ns, s)] = make_double2((double)v[2 * k], (double)v[2 * k + 1]);
    }
};

template <class R>
struct SpinorIO<SpF32, R> {
    static __device__ __forceinline__ void load(const void* base, const float*, size_t h, int s, int ns, R v[24]) {
        const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 q = __ldg(p + chunk_off(h, k, 6, ns, s));
            v[4 * k] = q.x;
            v[4 * k + 1] = q.y;
            v[4 * k + 2] = q.z;
            v[4 * k + 3] = q.w;
        }
    }
    static __device__ __forceinline__ void store(void* base, float*, size_t h, int s, int ns, const R v[24]) {
        float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            p[chunk_off(h, k, 6, ns, s)] = make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2], (float)v[4 * k + 3]);
    }
};

template <class H2>
struct Half2Cvt;
template <>
struct Half2Cvt<__half2> {
    static __device__ __forceinline__ float2 to_f2(__half2 a) { return __half22float2(a); }
    static __device__ __forceinline__ __half2 from_f2(float a, float b) { return __floats2half2_rn(a, b); }
};
template <>
struct Half2Cvt<__nv_bfloat162> {
    static __device__ __forceinline__ float2 to_f2(__nv_bfloat162 a) { return __bfloat1622float2(a); }
    static __device__ __forceinline__ __nv_bfloat162 from_f2(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

template <class H2, class R>
struct HalfIO {
    static __device__ __forceinline__ void load(const void* base, const float* norm, size_t h, int s, int ns, R v[24]) {
        const uint4* p = reinterpret_cast<const uint4*>(base);
        const float sc = __ldg(norm + h * ns + s);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 q = __ldg(p + chunk_off(h, k, 3, ns, s));
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                H2 hv;
                *reinterpret_cast<uint32_t*>(&hv) = w[j];
                const float2 f = Half2Cvt<H2>::to_f2(hv);
                v[8 * k + 2 * j] = (R)f.x * (R)sc;  // exact for R = double (the unpacked stored value)
                v[8 * k + 2 * j + 1] = (R)f.y * (R)sc;
            }
        }
    }
    static __device__ __forceinline__ void store(void* base, float* norm, size_t h, int s, int ns, const R v[24]) {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) mx = fmaxf(mx, fabsf((float)v[k]));
        const float sc = mx > 0.f ? mx : 1.f;
        const float inv = 1.f / sc;
        uint4* p = reinterpret_cast<uint4*>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                H2 hv = Half2Cvt<H2>::from_f2((float)v[8 * k + 2 * j] * inv, (float)v[8 * k + 2 * j + 1] * inv);
                w[j] = *reinterpret_cast<uint32_t*>(&hv);
            }
            p[chunk_off(h, k, 3, ns, s)] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        norm[h * ns + s] = sc;
    }
};

template <class R>
struct SpinorIO<SpF16, R> : HalfIO<__half2, R> {};
template <class R>
struct SpinorIO<SpBF16, R> : HalfIO<__nv_bfloat162, R> {};

// Float-float storage (reliable updates of the mixed-precision CG): each real as an FP32 pair
// (hi, lo), 192 bytes per 5D site in the FP64 chunk layout (a 16-byte chunk holds two values).
struct SpFF { using T = float; static constexpr int NCH = 12; static constexpr bool kNorm = false; };

template <class R>
struct SpinorIO<SpFF, R> {
    static __device__ __forceinline__ void load(const void* base, const float*, size_t h, int s, int ns, R v[24]) {
        const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float4 q = __ldg(p + chunk_off(h, k, 12, ns, s));
            v[2 * k] = ff_to<R>(ff(q.x, q.y));
            v[2 * k + 1] = ff_to<R>(ff(q.z, q.w));
        }
    }
    static __device__ __forceinline__ void store(void* base, float*, size_t h, int s, int ns, const R v[24]) {
        float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const ff a = to_ff(v[2 * k]), b = to_ff(v[2 * k + 1]);
            p[chunk_off(h, k, 12, ns, s)] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
    }
};

// Link field: for each parity p, direction mu and half-site h, U_mu(x) of site (p, h),
// row-major 3x3 complex.  LinkD18: 18 doubles; LinkF18: 18 floats padded to 20;
// LinkF12: rows 0 and 1 as 12 floats, row 2 = conj(row0 x row1) rebuilt in registers;
// LinkH12: rows 0 and 1 as 12 FP16 values (no scale: every entry of an SU(3) matrix has
// modulus <= 1, inside FP16's normal range), row 2 rebuilt in FP32.
// Address: ((p * 4 + mu) * Vh + h) * BYTES.
struct LinkD18 { static constexpr int BYTES = 144; };
struct LinkF18 { static constexpr int BYTES = 80; };
struct LinkF12 { static constexpr int BYTES = 48; };
struct LinkH12 { static constexpr int BYTES = 24; };
struct LinkFF18 { static constexpr int BYTES = 144; };  // 18 float-float pairs (the FP64 links split)

template <class LK, class R>
struct LinkIO;

template <class R>
struct LinkIO<LinkFF18, R> {
    static __device__ __forceinline__ void load(const void* base, size_t idx, R u[18]) {
        const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) + idx * 144);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 q = __ldg(p + k);
            u[2 * k] = ff_to<R>(ff(q.x, q.y));
            u[2 * k + 1] = ff_to<R>(ff(q.z, q.w));
        }
    }
};

template <class R>
struct LinkIO<LinkD18, R> {
    static __device__ __forceinline__ void load(const void* base, size_t idx, R u[18]) {
        const double2* p = reinterpret_cast<const double2*>(reinterpret_cast<const char*>(base) + idx * 144);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double2 q = __ldg(p + k);
            u[2 * k] = (R)q.x;
            u[2 * k + 1] = (R)q.y;
        }
    }
};

template <class R>
struct LinkIO<LinkF18, R> {
    static __device__ __forceinline__ void load(const void* base, size_t idx, R u[18]) {
        const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) + idx * 80);
        float t[20];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float4 q = __ldg(p + k);
            t[4 * k] = q.x; t[4 * k + 1] = q.y; t[4 * k + 2] = q.z; t[4 * k + 3] = q.w;
        }
#pragma unroll
        for (int k = 0; k < 18; ++k) u[k] = (R)t[k];
    }
};

template <class R>
struct LinkIO<LinkF12, R> {
    static __device__ __forceinline__ void load(const void* base, size_t idx, R u[18]) {
        const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) + idx * 48);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 q = __ldg(p + k);
            u[4 * k] = (R)q.x; u[4 * k + 1] = (R)q.y; u[4 * k + 2] = (R)q.z; u[4 * k + 3] = (R)q.w;
        }
        // row2[j] = conj(row0[j+1] row1[j+2] - row0[j+2] row1[j+1]) (indices mod 3)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int a = (j + 1) % 3, b = (j + 2) % 3;
            const R ar = u[2 * a], ai = u[2 * a + 1], br = u[2 * b], bi = u[2 * b + 1];
            const R cr = u[6 + 2 * a], ci = u[6 + 2 * a + 1], dr = u[6 + 2 * b], di = u[6 + 2 * b + 1];
            const R re = (ar * dr - ai * di) - (br * cr - bi * ci);
            const R im = (ar * di + ai * dr) - (br * ci + bi * cr);
            u[12 + 2 * j] = re;
            u[12 + 2 * j + 1] = -im;
        }
    }
};

// row2[j] = conj(row0[j+1] row1[j+2] - row0[j+2] row1[j+1]) (indices mod 3): the third row of
// an SU(3) matrix from its first two (u[0..11] = rows 0, 1; fills u[12..17])
template <class R>
__device__ __forceinline__ void su3_third_row(R u[18]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int a = (j + 1) % 3, b = (j + 2) % 3;
        const R ar = u[2 * a], ai = u[2 * a + 1], br = u[2 * b], bi = u[2 * b + 1];
        const R cr = u[6 + 2 * a], ci = u[6 + 2 * a + 1], dr = u[6 + 2 * b], di = u[6 + 2 * b + 1];
        const R re = (ar * dr - ai * di) - (br * cr - bi * ci);
        const R im = (ar * di + ai * dr) - (br * ci + bi * cr);
        u[12 + 2 * j] = re;
        u[12 + 2 * j + 1] = -im;
    }
}

template <class R>
struct LinkIO<LinkH12, R> {
    static __device__ __forceinline__ void load(const void* base, size_t idx, R u[18]) {
        const uint2* p = reinterpret_cast<const uint2*>(reinterpret_cast<const char*>(base) + idx * 24);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 q = __ldg(p + k);
            __half2 a, b;
            *reinterpret_cast<uint32_t*>(&a) = q.x;
            *reinterpret_cast<uint32_t*>(&b) = q.y;
            const float2 fa = __half22float2(a), fb = __half22float2(b);
            u[4 * k] = (R)fa.x; u[4 * k + 1] = (R)fa.y; u[4 * k + 2] = (R)fb.x; u[4 * k + 3] = (R)fb.y;
        }
        su3_third_row(u);
    }
};

// ---------------------------------------------------------------- bounds checks (debug builds)
// Built with ODWF_BOUNDS_CHECK (libodwf_check.so): an index gathered from a table or computed
// from coordinates that falls outside [0, n) sets `code` in *flag and is replaced by 0, so that
// no access leaves its buffer; the host reports the flag as an error after the call.  In the
// release build this compiles to the index itself.
__device__ __forceinline__ int checked_index(int i, int n, unsigned* flag, unsigned code) {
#ifdef ODWF_BOUNDS_CHECK
    if ((unsigned)i >= (unsigned)n) {
        if (flag) atomicOr(flag, code);
        return 0;
    }
#else
    (void)n;
    (void)flag;
    (void)code;
#endif
    return i;
}
enum : unsigned { kBoundsNeighbour = 1u, kBoundsSite = 2u };

// ---------------------------------------------------------------- lane-group shuffles
template <class R>
__device__ __forceinline__ R shfl_idx(R v, int src, int width) { return __shfl_sync(0xffffffffu, v, src, width); }
template <class R>
__device__ __forceinline__ R shfl_up(R v, int d, int width) { return __shfl_up_sync(0xffffffffu, v, d, width); }
template <class R>
__device__ __forceinline__ R shfl_down(R v, int d, int width) { return __shfl_down_sync(0xffffffffu, v, d, width); }
template <>
__device__ __forceinline__ ff shfl_idx<ff>(ff v, int src, int width) {
    return ff(__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width));
}
template <>
__device__ __forceinline__ ff shfl_up<ff>(ff v, int d, int width) {
    return ff(__shfl_up_sync(0xffffffffu, v.hi, d, width), __shfl_up_sync(0xffffffffu, v.lo, d, width));
}
template <>
__device__ __forceinline__ ff shfl_down<ff>(ff v, int d, int width) {
    return ff(__shfl_down_sync(0xffffffffu, v.hi, d, width), __shfl_down_sync(0xffffffffu, v.lo, d, width));
}

// Bidiagonal fifth-dimension operator on the lane group (cyclic, corner -r):
//   dag = false:  (X v)_s = a_s v_s + b_s (L v)_s          (X = B with a=rho, b=sigma; X = M with a=d, b=e)
//   dag = true:   (X^dag v)_s = a_s v_s + (L^dag (b v))_s
// (L v)^up_s = v^up_{s-1} (s > 0) or -r v^up_{Ns-1};  (L v)^dn_s = v^dn_{s+1} (s < Ns-1) or -r v^dn_0;
// (L^dag u)^up_s = u^up_{s+1} (s < Ns-1) or -r u^up_0;  (L^dag u)^dn_s = u^dn_{s-1} (s > 0) or -r u^dn_{Ns-1}.
template <class R>
__device__ __forceinline__ void bidiag_apply(R v[24], R a_s, R b_s, R r, int s, int ns, bool dag) {
    const int sm = (s + ns - 1) & (ns - 1), sp = (s + 1) & (ns - 1);
    if (!dag) {
        const R cm = (s == 0) ? -r * b_s : b_s;       // coefficient of v^up_{s-1}
        const R cp = (s == ns - 1) ? -r * b_s : b_s;  // coefficient of v^dn_{s+1}
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const R up = shfl_idx(v[k], sm, ns);
            const R dn = shfl_idx(v[12 + k], sp, ns);
            v[k] = a_s * v[k] + cm * up;
            v[12 + k] = a_s * v[12 + k] + cp * dn;
        }
    } else {
        const R cu = (s == ns - 1) ? -r : (R)1;  // on (b v)^up_{s+1}
        const R cd = (s == 0) ? -r : (R)1;       // on (b v)^dn_{s-1}
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const R up = shfl_idx(b_s * v[k], sp, ns);
            const R dn = shfl_idx(b_s * v[12 + k], sm, ns);
            v[k] = a_s * v[k] + cu * up;
            v[12 + k] = a_s * v[12 + k] + cd * dn;
        }
    }
}

// Cyclic bidiagonal solve along s for 12 reals (one chirality), O(log Ns) shuffle steps:
//   forward:  d_s w_s + c_s w_{s-1} = v_s,  w_{-1} := -r w_{Ns-1}
//   backward: d_s w_s + c_s w_{s+1} = v_s,  w_{Ns} := -r w_0
// Each lane holds the affine map w_{prev} -> w_s = beta + alpha w_prev; a Hillis-Steele
// scan composes the maps (g_s = solution with zero corner, A_s = product of alphas),
// then the corner value follows from w_corner = -r (g_last + A_last w_corner).
template <class R>
__device__ __forceinline__ void cyclic_solve12(R v[12], R inv_d, R c_s, R r, int s, int ns, bool forward) {
    R coef = -c_s * inv_d;
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] *= inv_d;
    const int q = forward ? s : ns - 1 - s;  // position in scan order
    for (int off = 1; off < ns; off <<= 1) {
        R pc;
        if (forward) pc = shfl_up(coef, off, ns); else pc = shfl_down(coef, off, ns);
        const bool take = q >= off;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            R pv;
            if (forward) pv = shfl_up(v[k], off, ns); else pv = shfl_down(v[k], off, ns);
            if (take) v[k] += coef * pv;
        }
        if (take) coef *= pc;
    }
    const int last = forward ? ns - 1 : 0;
    const R Al = shfl_idx(coef, last, ns);
    const R fac = -r / ((R)1 + r * Al);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const R gl = shfl_idx(v[k], last, ns);
        v[k] += coef * fac * gl;
    }
}

// M^-1 (dag = false) or M^-dag (dag = true) on the lane group.
//   M^-1:   up forward  with c_s = e_s;          down backward with c_s = e_s
//   M^-dag: up backward with c_s = e_{s+1};      down forward  with c_s = e_{s-1}   (cyclic indices)
template <class R>
__device__ __forceinline__ void minv_apply(R v[24], const Coef5<R>& cf, R r, int s, int ns, bool dag) {
    const R inv_d = cf.inv_d[s];
    if (!dag) {
        cyclic_solve12(v, inv_d, cf.e[s], r, s, ns, true);
        cyclic_solve12(v + 12, inv_d, cf.e[s], r, s, ns, false);
    } else {
        cyclic_solve12(v, inv_d, cf.e[(s + 1) & (ns - 1)], r, s, ns, false);
        cyclic_solve12(v + 12, inv_d, cf.e[(s + ns - 1) & (ns - 1)], r, s, ns, true);
    }
}

// FP32 form of cyclic_solve12 for the mixed-precision kernels: the same scan, with the
// 12 reals handled as six FP32x2 pairs (one packed FMA per pair and step) and an extra
// factor `pre` folded into the 1/d_s scaling (v <- pre v before the solve).
template <bool PACK>
__device__ __forceinline__ void cyclic_solve12_f(float v[12], float pre, float inv_d, float c_s, float r, int s,
                                                 int ns, bool forward) {
    if (!PACK) {  // scalar FMAs (fewer register-pair constraints where registers are tight)
        float coef = -c_s * inv_d;
        const float sc = pre * inv_d;
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] *= sc;
        const int q = forward ? s : ns - 1 - s;
        for (int off = 1; off < ns; off <<= 1) {
            const float pc = forward ? shfl_up(coef, off, ns) : shfl_down(coef, off, ns);
            const float cm = q >= off ? coef : 0.f;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float pv = forward ? shfl_up(v[k], off, ns) : shfl_down(v[k], off, ns);
                v[k] = fmaf(cm, pv, v[k]);
            }
            if (q >= off) coef *= pc;
        }
        const int last = forward ? ns - 1 : 0;
        const float Al = shfl_idx(coef, last, ns);
        const float cf = coef * (-r / (1.f + r * Al));
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = fmaf(cf, shfl_idx(v[k], last, ns), v[k]);
        return;
    }
    float coef = -c_s * inv_d;
    const float sc = pre * inv_d;
    float2 w[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = make_float2(v[2 * k] * sc, v[2 * k + 1] * sc);
    const int q = forward ? s : ns - 1 - s;
    for (int off = 1; off < ns; off <<= 1) {
        const float pc = forward ? shfl_up(coef, off, ns) : shfl_down(coef, off, ns);
        const float cm = q >= off ? coef : 0.f;
        const float2 cm2 = make_float2(cm, cm);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float2 pv;
            pv.x = forward ? shfl_up(w[k].x, off, ns) : shfl_down(w[k].x, off, ns);
            pv.y = forward ? shfl_up(w[k].y, off, ns) : shfl_down(w[k].y, off, ns);
            w[k] = __ffma2_rn(cm2, pv, w[k]);
        }
        if (q >= off) coef *= pc;
    }
    const int last = forward ? ns - 1 : 0;
    const float Al = shfl_idx(coef, last, ns);
    const float cf = coef * (-r / (1.f + r * Al));
    const float2 cf2 = make_float2(cf, cf);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float2 gl = make_float2(shfl_idx(w[k].x, last, ns), shfl_idx(w[k].y, last, ns));
        w[k] = __ffma2_rn(cf2, gl, w[k]);
        v[2 * k] = w[k].x;
        v[2 * k + 1] = w[k].y;
    }
}

// M^-1 / M^-dag (as minv_apply) of pre * v, FP32
template <bool PACK = true>
__device__ __forceinline__ void minv_apply_f(float v[24], const Coef5<float>& cf, float r, int s, int ns, bool dag,
                                             float pre) {
    const float inv_d = cf.inv_d[s];
    if (!dag) {
        cyclic_solve12_f<PACK>(v, pre, inv_d, cf.e[s], r, s, ns, true);
        cyclic_solve12_f<PACK>(v + 12, pre, inv_d, cf.e[s], r, s, ns, false);
    } else {
        cyclic_solve12_f<PACK>(v, pre, inv_d, cf.e[(s + 1) & (ns - 1)], r, s, ns, false);
        cyclic_solve12_f<PACK>(v + 12, pre, inv_d, cf.e[(s + ns - 1) & (ns - 1)], r, s, ns, true);
    }
}

// ---------------------------------------------------------------- CG scalar state (device)
// kRestarting: a reliable update has recomputed the residual and restarted the inner
// iteration on the update stream; the iteration stream switches it back to kRunning once
// it has waited for that work (state_kernel mode 2).
enum SysStatus : int { kRunning = 0, kNeedUpdate = 1, kDone = 2, kBreakdown = 3, kIdle = 4, kMaxIter = 5,
                       kRestarting = 6 };

struct SysState {
    double rr;       // inner ||r||^2 of the current iterate
    double pAp;      // p^dag A p of this iteration
    double alpha, beta;
    double r_max;    // largest inner ||r|| since the last reliable update
    double rr_new;   // ||r||^2 after this iteration's update
    double bb;       // ||b||^2
    double stop_rr;  // tol^2 ||b||^2
    double delta;    // reliable-update threshold
    double sum;      // generic reduction result
    // Mixed precision solves the inner system for r / rscale, rscale = |r| at the last
    // (re)start, so the inner fields stay near unit norm (FP16/BF16 range, and no FP32
    // underflow of squared components late in a solve); plain CG keeps rscale = 1.
    // rr, r_max and stop_in are in inner units, bb, stop_rr and sum in true units.
    double rscale;
    double stop_in;  // inner stopping threshold on rr

    int status;
    int iter;
    int max_iter;
    int reliable;    // 1: mixed precision (reliable updates), 0: plain CG
};

}  // namespace odwf
