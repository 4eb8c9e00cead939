// Production mixed-precision hop kernels with two adjacent s per lane (Ns = 8, 16; FP16 / BF16
// storage): the hops K1 (chi_t = B M^-1 (-1/2 W chi_p)), K2 (s = p - M^-1 (-1/2 W chi_t), |s|^2,
// a = M^-dag s) and K3 (c = M^-dag (-1/2 B^dag W^dag a)) of kernels_mixed2.cu, with lane l of a
// site's Ns/2-lane group holding the 5D sites s = 2l and 2l + 1.  K4, which also streams the FP32
// CG vectors r and x in and out, stays with one s per lane: at the higher occupancy of that kernel
// its streams are hidden better (measured on 32^4 x 16, one system: K1 509 -> 422 us, K3 524 ->
// 425 us, K2 784 -> 708 us here; K4 922 us there against 982 us here).
//
// Why two s per lane: on GB300 the one-s-per-lane hops are bound by the L1/shared-memory data
// path, not by HBM.  With two s per lane
//   - every link element read from shared memory serves two spinors,
//   - B's fifth-dimension shift needs one shuffle per component for two values, the other
//     neighbour being in the lane,
//   - the cyclic M5^-1 solve composes the lane's two recurrence steps locally and scans over
//     Ns/2 lanes, one step fewer, with one extra shuffle to rebuild the lane's first value,
// so shared-memory wavefronts and shuffles per 5D site roughly halve.  Neighbour loads stay
// coalesced because the spinor layout stores the even s of a site first and the odd s second
// (chunk_slot), so lanes l = 0 .. Ns/2-1 read consecutive words for s = 2l and again for 2l + 1.
#include <type_traits>

#include "kernels_mixed_common.cuh"

namespace odwf {

namespace {

using namespace mx;

constexpr int kBS3 = 128;

// Raw stored words of the lane's two 5D sites (h, 2l) and (h, 2l + 1)
struct RawPair {
    uint4 q[2][3];
    float2 sc;
};

template <int NS>
__device__ __forceinline__ void fetch_pair(const void* base, const float* norm, unsigned h, int l, RawPair& r) {
    constexpr unsigned LPS = NS / 2;
    const uint4* p = reinterpret_cast<const uint4*>(base) + (h * (3u * NS) + (unsigned)l);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.q[0][k] = __ldg(p + k * NS);        // slot l: s = 2l
        r.q[1][k] = __ldg(p + k * NS + LPS);  // slot Ns/2 + l: s = 2l + 1
    }
    r.sc = __ldg(reinterpret_cast<const float2*>(norm + (size_t)h * NS) + l);  // scales of s = 2l, 2l + 1
}

template <class SP>
__device__ __forceinline__ RawSite<SP> raw_of(const RawPair& r, int v) {
    RawSite<SP> o;
#pragma unroll
    for (int k = 0; k < 3; ++k) o.q[k] = r.q[v][k];
    o.sc = v ? r.sc.y : r.sc.x;
    return o;
}

struct Acc {
    float2 AUr[3], AUi[3], ADr[3], ADi[3], ADSr[3], ADSi[3];
};

// One hop direction for both values of the lane: the link element (a, b) is read from shared
// memory once and multiplied into both spinors.
template <class SP, int MU, bool DAGU>
__device__ __forceinline__ void hop_dir_pair(const RawPair& raw, float sgn, float sg, const float2* L, Acc& A,
                                             Acc& B) {
    constexpr bool SW = (MU == 0 || MU == 1);
    float2 HrA[3], HiA[3], NhA[3], HrB[3], HiB[3], NhB[3];
    {
        float2 Ur[3], Ui[3], Dr[3], Di[3];
        unpack_site<SP, SW>(raw_of<SP>(raw, 0), Ur, Ui, Dr, Di);
        project_pairs<MU>(Ur, Ui, Dr, Di, sg, HrA, HiA);
        unpack_site<SP, SW>(raw_of<SP>(raw, 1), Ur, Ui, Dr, Di);
        project_pairs<MU>(Ur, Ui, Dr, Di, sg, HrB, HiB);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        NhA[c] = DAGU ? make_float2(-HrA[c].x, -HrA[c].y) : make_float2(-HiA[c].x, -HiA[c].y);
        NhB[c] = DAGU ? make_float2(-HrB[c].x, -HrB[c].y) : make_float2(-HiB[c].x, -HiB[c].y);
    }
    const float mA = raw.sc.x * sgn, mB = raw.sc.y * sgn;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 WrA = make_float2(0.f, 0.f), WiA = WrA, WrB = WrA, WiB = WrA;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float2 v = DAGU ? L[3 * b + a] : L[3 * a + b];
            const float2 ur = make_float2(v.x, v.x), ui = make_float2(v.y, v.y);
            su3_row_acc<DAGU>(ur, ui, HrA[b], HiA[b], NhA[b], WrA, WiA);
            su3_row_acc<DAGU>(ur, ui, HrB[b], HiB[b], NhB[b], WrB, WiB);
        }
        accumulate_row<MU>(mA, sg * mA, WrA, WiA, A.AUr[a], A.AUi[a], A.ADr[a], A.ADi[a], A.ADSr[a], A.ADSi[a]);
        accumulate_row<MU>(mB, sg * mB, WrB, WiB, B.AUr[a], B.AUi[a], B.ADr[a], B.ADi[a], B.ADSr[a], B.ADSi[a]);
    }
}

// ---------------------------------------------------------------- fifth dimension, two s per lane
// The lane's values: A = s0 = 2l, B = s1 = 2l + 1; lanes of a site form a group of LPS = Ns/2.
// Each Half6 is one chirality of one value (six spin pairs).

// Bidiagonal X = diag(a) + diag(b) L (dag = false) or X^dag = a + L^dag b (dag = true), as
// bidiag_apply: L takes up from s - 1 and down from s + 1 with the -r corners, L^dag the reverse.
template <int NS>
__device__ __forceinline__ void bidiag2(Half6& upA, Half6& dnA, Half6& upB, Half6& dnB, float a0, float b0,
                                        float a1, float b1, float r, int l, bool dag) {
    constexpr int LPS = NS / 2;
    const int lm = (l + LPS - 1) & (LPS - 1), lp = (l + 1) & (LPS - 1);
    if (!dag) {
        const float2 cmA = f2(l == 0 ? -r * b0 : b0);        // on v^up_{s0 - 1} (lane l-1's B)
        const float2 cpB = f2(l == LPS - 1 ? -r * b1 : b1);  // on v^dn_{s1 + 1} (lane l+1's A)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 prevB = shfl2_idx(upB.p(k), lm, LPS);
            const float2 nextA = shfl2_idx(dnA.p(k), lp, LPS);
            const float2 uA = upA.p(k), dB = dnB.p(k);
            upA.p(k) = fma2(f2(a0), uA, __fmul2_rn(cmA, prevB));
            upB.p(k) = fma2(f2(a1), upB.p(k), __fmul2_rn(f2(b1), uA));
            dnA.p(k) = fma2(f2(a0), dnA.p(k), __fmul2_rn(f2(b0), dB));
            dnB.p(k) = fma2(f2(a1), dB, __fmul2_rn(cpB, nextA));
        }
    } else {
        const float2 cuB = f2(l == LPS - 1 ? -r : 1.f);  // on (b v)^up_{s1 + 1} (lane l+1's A)
        const float2 cdA = f2(l == 0 ? -r : 1.f);        // on (b v)^dn_{s0 - 1} (lane l-1's B)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 uuA = __fmul2_rn(f2(b0), upA.p(k)), uuB = __fmul2_rn(f2(b1), upB.p(k));
            const float2 udA = __fmul2_rn(f2(b0), dnA.p(k)), udB = __fmul2_rn(f2(b1), dnB.p(k));
            const float2 nextU = shfl2_idx(uuA, lp, LPS);
            const float2 prevD = shfl2_idx(udB, lm, LPS);
            upA.p(k) = fma2(f2(a0), upA.p(k), uuB);
            upB.p(k) = fma2(f2(a1), upB.p(k), __fmul2_rn(cuB, nextU));
            dnA.p(k) = fma2(f2(a0), dnA.p(k), __fmul2_rn(cdA, prevD));
            dnB.p(k) = fma2(f2(a1), dnB.p(k), udA);
        }
    }
}

// Cyclic bidiagonal solve of pre * v along s for one chirality, two values per lane:
//   forward:  d_s w_s + c_s w_{s-1} = pre v_s,  w_{-1} := -r w_{Ns-1}
//   backward: d_s w_s + c_s w_{s+1} = pre v_s,  w_{Ns} := -r w_0
// w_s = beta_s + alpha_s w_prev (beta = pre v / d, alpha = -c / d).  The lane composes its two
// steps into one affine map, the maps are scanned over the lane group (zero corner), the corner
// value follows from w_corner = -r (g_end + A_end w_corner), and the lane's other value is one
// step from its neighbour's result.
template <int NS>
__device__ __forceinline__ void cyclic2(Half6& A, Half6& B, float pre, float inv_d0, float c0, float inv_d1,
                                        float c1, float r, int l, bool fwd) {
    constexpr int LPS = NS / 2;
    const float al0 = -c0 * inv_d0, al1 = -c1 * inv_d1;
    const float2 sc0 = f2(pre * inv_d0), sc1 = f2(pre * inv_d1);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        A.p(k) = __fmul2_rn(sc0, A.p(k));  // beta of s0
        B.p(k) = __fmul2_rn(sc1, B.p(k));  // beta of s1
    }
    // lane map over its two steps: forward w_{s1} = (b1 + a1 b0) + a1 a0 w_{s0 - 1};
    // backward w_{s0} = (b0 + a0 b1) + a0 a1 w_{s1 + 1}
    Half6 G;
    float coef = al0 * al1;
#pragma unroll
    for (int k = 0; k < 6; ++k) G.p(k) = fwd ? fma2(f2(al1), A.p(k), B.p(k)) : fma2(f2(al0), B.p(k), A.p(k));
    const int q = fwd ? l : LPS - 1 - l;
#pragma unroll
    for (int off = 1; off < LPS; off <<= 1) {
        const float pc = fwd ? __shfl_up_sync(0xffffffffu, coef, off, LPS) : __shfl_down_sync(0xffffffffu, coef, off, LPS);
        const float2 cm = f2(q >= off ? coef : 0.f);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 pv = fwd ? shfl2_up(G.p(k), off, LPS) : shfl2_down(G.p(k), off, LPS);
            G.p(k) = fma2(cm, pv, G.p(k));
        }
        if (q >= off) coef *= pc;
    }
    const int end = fwd ? LPS - 1 : 0;
    const float Aend = __shfl_sync(0xffffffffu, coef, end, LPS);
    const float fac = -r / (1.f + r * Aend);
    const bool edge = fwd ? (l == 0) : (l == LPS - 1);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float2 gend = shfl2_idx(G.p(k), end, LPS);
        const float2 wc = __fmul2_rn(f2(fac), gend);       // the corner value w_{-1} (or w_{Ns})
        const float2 w = fma2(f2(coef), wc, G.p(k));       // this lane's s1 (forward) or s0 (backward)
        const float2 nb = fwd ? shfl2_up(w, 1, LPS) : shfl2_down(w, 1, LPS);
        const float2 prev = edge ? wc : nb;                // w_{s0 - 1} (forward) or w_{s1 + 1} (backward)
        if (fwd) {
            A.p(k) = fma2(f2(al0), prev, A.p(k));
            B.p(k) = w;
        } else {
            B.p(k) = fma2(f2(al1), prev, B.p(k));
            A.p(k) = w;
        }
    }
}

// M^-1 (dag = false) or M^-dag (dag = true) of pre * v, as minv_apply
template <int NS>
__device__ __forceinline__ void minv2(Half6& upA, Half6& dnA, Half6& upB, Half6& dnB, const Coef5<float>& cf,
                                      float r, int l, bool dag, float pre) {
    const int s0 = 2 * l, s1 = 2 * l + 1;
    const float id0 = cf.inv_d[s0], id1 = cf.inv_d[s1];
    if (!dag) {
        cyclic2<NS>(upA, upB, pre, id0, cf.e[s0], id1, cf.e[s1], r, l, true);
        cyclic2<NS>(dnA, dnB, pre, id0, cf.e[s0], id1, cf.e[s1], r, l, false);
    } else {
        cyclic2<NS>(upA, upB, pre, id0, cf.e[(s0 + 1) & (NS - 1)], id1, cf.e[(s1 + 1) & (NS - 1)], r, l, false);
        cyclic2<NS>(dnA, dnB, pre, id0, cf.e[(s0 + NS - 1) & (NS - 1)], id1, cf.e[(s1 + NS - 1) & (NS - 1)], r, l,
                    true);
    }
}

__device__ __forceinline__ void to_pairs(const Acc& a, Half6& up, Half6& dn) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        up.R[c] = a.AUr[c];
        up.I[c] = a.AUi[c];
        dn.R[c] = __fadd2_rn(a.ADr[c], make_float2(a.ADSr[c].y, a.ADSr[c].x));
        dn.I[c] = __fadd2_rn(a.ADi[c], make_float2(a.ADSi[c].y, a.ADSi[c].x));
    }
}

// Blocks per SM: K2, which also streams p in and keeps two scans' state, runs faster at four
// (128 registers, a few spilled: 764 -> 708 us on 32^4 x 16); K1 and K3 at three (168 registers).
template <int KIND>
constexpr int hop3_min_blocks() { return KIND == K2 ? 4 : 3; }

template <class SP, class LK, int NS, int KIND>
__global__ void __launch_bounds__(kBS3, hop3_min_blocks<KIND>()) hop3_kernel(const HopParams<float> P) {
    constexpr int LPS = NS / 2;            // lanes per site
    constexpr int kLS = 18;                // floats per staged link: 9 x (ur, ui)
    constexpr int kSL = 8 * kLS + 4;       // floats per site
    static_assert(KIND == K1 || KIND == K2 || KIND == K3, "hop3 implements the hops K1, K2 and K3");
    constexpr bool DAG = (KIND == K3);
    const int sys = blockIdx.y + P.sys_base;
    if (P.gate && P.st[sys].status != P.need_status) return;
    if (P.prof_count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(P.prof_count, 1ull);

    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int l = (int)(gi & (LPS - 1));
    const int s0 = 2 * l, s1 = s0 + 1;
    const size_t hh = gi / LPS;
    const bool valid = hh < (size_t)P.g.Vh;
    const int h = valid ? (int)hh : 0;
    const float r = (float)P.r_sys[sys];
    const int p_out = P.p_out;

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

    // the site's eight links as (ur, ui) pairs in shared memory, from the site-major array:
    // lane d of the group loads links d, d + LPS, ... (each link once per site)
    __shared__ __align__(16) float s_links[(kBS3 / LPS) * kSL];
    float* my_links = s_links + (threadIdx.x / LPS) * kSL;
#pragma unroll
    for (int d = l; d < 8; d += LPS) {
        float u[18];
        link_load_cs<LK>(P.links, ((size_t)p_out * P.g.Vh + h) * 8 + d, u);
        float2* dst = reinterpret_cast<float2*>(my_links + d * kLS);
#pragma unroll
        for (int k = 0; k < 9; ++k) dst[k] = make_float2(u[2 * k], u[2 * k + 1]);
    }
    __syncwarp();

    const void* in = P.in.d(sys);
    const float* in_n = P.in.n(sys);
    Acc A, B;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        A.AUr[c] = A.AUi[c] = A.ADr[c] = A.ADi[c] = A.ADSr[c] = A.ADSi[c] = make_float2(0.f, 0.f);
        B.AUr[c] = B.AUi[c] = B.ADr[c] = B.ADi[c] = B.ADSr[c] = B.ADSi[c] = make_float2(0.f, 0.f);
    }
    const float2* L2p = reinterpret_cast<const float2*>(my_links);
    constexpr float SF = DAG ? 1.f : -1.f;
    RawPair rp;
#define ODWF_HOP3_DIR(MU_, DIR_)                                                                   \
    {                                                                                              \
        constexpr int j_ = 2 * MU_ + DIR_;                                                         \
        fetch_pair<NS>(in, in_n, (unsigned)nb[j_], l, rp);                                         \
        const float sgn_ = (flip & (1u << j_)) ? -1.f : 1.f;                                      \
        hop_dir_pair<SP, MU_, DIR_ == 1>(rp, sgn_, DIR_ == 0 ? SF : -SF, L2p + j_ * 9, A, B);      \
    }
    ODWF_HOP3_DIR(0, 0); ODWF_HOP3_DIR(0, 1);
    ODWF_HOP3_DIR(1, 0); ODWF_HOP3_DIR(1, 1);
    ODWF_HOP3_DIR(2, 0); ODWF_HOP3_DIR(2, 1);
    ODWF_HOP3_DIR(3, 0); ODWF_HOP3_DIR(3, 1);
#undef ODWF_HOP3_DIR
    Half6 upA, dnA, upB, dnB;
    to_pairs(A, upA, dnA);
    to_pairs(B, upB, dnB);

    const Coef5<float>& cf = P.cf;
    float v[24];
    if (KIND == K1) {
        minv2<NS>(upA, dnA, upB, dnB, cf, r, l, false, -0.5f);
        bidiag2<NS>(upA, dnA, upB, dnB, cf.rho[s0], cf.sigma[s0], cf.rho[s1], cf.sigma[s1], r, l, false);
        if (valid) {
            pairs_to_mem(upA, dnA, v);
            SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s0, NS, v);
            pairs_to_mem(upB, dnB, v);
            SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s1, NS, v);
        }
    } else if (KIND == K2) {
        // s = p - M^-1 (-1/2 y) = p + M^-1 (y/2);  |s|^2;  a = M^-dag s
        minv2<NS>(upA, dnA, upB, dnB, cf, r, l, false, 0.5f);
        float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            Half6& U = w ? upB : upA;
            Half6& D = w ? dnB : dnA;
            if (valid) {
                spinor_load_cs<SP, NS>(P.z.d(sys), P.z.n(sys), (size_t)h, w ? s1 : s0, v);
            } else {
#pragma unroll
                for (int k = 0; k < 24; ++k) v[k] = 0.f;
            }
            Half6 zu, zd;
            mem_to_pairs(v, zu, zd);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                U.p(k) = __fadd2_rn(U.p(k), zu.p(k));
                D.p(k) = __fadd2_rn(D.p(k), zd.p(k));
                n2 = fma2(U.p(k), U.p(k), n2);
                n2 = fma2(D.p(k), D.p(k), n2);
            }
        }
        // a site past the end computed site 0's neighbours: no contribution
        const float nrm = valid ? n2.x + n2.y : 0.f;
        minv2<NS>(upA, dnA, upB, dnB, cf, r, l, true, 1.f);
        if (valid) {
            pairs_to_mem(upA, dnA, v);
            SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s0, NS, v);
            pairs_to_mem(upB, dnB, v);
            SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s1, NS, v);
        }
        reduce_and_finalize(nrm, P.partials, P.counters, P.st, sys, FIN_ALPHA, P.part_stride);
    } else if (KIND == K3) {
        bidiag2<NS>(upA, dnA, upB, dnB, cf.rho[s0], cf.sigma[s0], cf.rho[s1], cf.sigma[s1], r, l, true);
        minv2<NS>(upA, dnA, upB, dnB, cf, r, l, true, -0.5f);
        if (valid) {
            pairs_to_mem(upA, dnA, v);
            SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s0, NS, v);
            pairs_to_mem(upB, dnB, v);
            SpinorIO<SP, float>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s1, NS, v);
        }
    }
}

template <class SP, class LK, int NS>
cudaError_t hop3_k(const HopParams<float>& P, int kind, int nsys, cudaStream_t st) {
    const size_t n = (size_t)P.g.Vh * (NS / 2);
    dim3 grid(blocks_for(n, kBS3), nsys);
    note_launch();
    switch (kind) {
        case K1: hop3_kernel<SP, LK, NS, K1><<<grid, kBS3, 0, st>>>(P); break;
        case K2: hop3_kernel<SP, LK, NS, K2><<<grid, kBS3, 0, st>>>(P); break;
        case K3: hop3_kernel<SP, LK, NS, K3><<<grid, kBS3, 0, st>>>(P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class SP, class LK>
cudaError_t hop3_ns(const HopParams<float>& P, int kind, int nsys, cudaStream_t st) {
    switch (P.ns) {
        case 8: return hop3_k<SP, LK, 8>(P, kind, nsys, st);
        case 16: return hop3_k<SP, LK, 16>(P, kind, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

template <class SP>
cudaError_t hop3_lk(const HopParams<float>& P, int kind, Lk lk, int nsys, cudaStream_t st) {
    switch (lk) {
        case Lk::F12: return hop3_ns<SP, LinkF12>(P, kind, nsys, st);
        case Lk::F18: return hop3_ns<SP, LinkF18>(P, kind, nsys, st);
        case Lk::H12: return hop3_ns<SP, LinkH12>(P, kind, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool hop3_supported(int ns, Sp low, int kind) {
    return (ns == 8 || ns == 16) && (low == Sp::F16 || low == Sp::BF16) && kind != K4;
}

cudaError_t launch_hop3(const HopParams<float>& P, int kind, Sp low, Lk lk, int nsys, cudaStream_t st) {
    switch (low) {
        case Sp::F16: return hop3_lk<SpF16>(P, kind, lk, nsys, st);
        case Sp::BF16: return hop3_lk<SpBF16>(P, kind, lk, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_hop_prod(const HopParams<float>& P, int kind, Sp low, Lk lk, int nsys, cudaStream_t st) {
    return hop3_supported(P.ns, low, kind) ? launch_hop3(P, kind, low, lk, nsys, st)
                                           : launch_hop2(P, kind, low, lk, nsys, st);
}

}  // namespace odwf
