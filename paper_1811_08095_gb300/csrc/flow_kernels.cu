// Gradient flow of the gauge field and the flow observables (Sec. 2 scale condition t^2 <E> = 0.3;
// Sec. 3 admissibility bound and clover topological charge).
//
// Definitions (lattice spacing 1, mu = 0..3 <-> x, y, z, t):
//   P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+          plaquette
//   ta(X)        = (X - X^+)/2 - tr(X - X^+)/6                          traceless anti-Hermitian part
//   Z_mu(x)      = -ta(U_mu(x) S_mu(x))                                 flow force (S_mu: staple sum)
//   dV/dt        = Z(V) V, third-order Runge-Kutta scheme of Luscher (JHEP 2010), three stages
//                  W <- exp(X_i) W with X_0 = eps Z_0 / 4, X_1 = 8/9 eps Z_1 - 17/36 eps Z_0,
//                  X_2 = 3/4 eps Z_2 - X_1
//   F_{mu nu}(x) = clover field strength from the four plaquette loops around x (Sec. 3)
//
// GB300 layout and arithmetic:
//   * links as float-float pairs (hi + lo, two FP32 arrays) of their first two rows, [mu][3][V]
//     float4 (two complex entries each); the third row of an SU(3) matrix is conj(row0 x row1)
//     and is rebuilt where a kernel needs it, so a link moves 48 bytes instead of 72.  The
//     stencils read only hi (FP32); the stage update adds its FP32 increment into (hi, lo) with an
//     error-free two-sum, so the accumulated links keep ~48 bits over thousands of stages without
//     any FP64 arithmetic (the FP64 pipe of this part runs at a small fraction of FP32);
//   * per stage two kernels.  plaq_kernel writes A_{mu nu}(x) = ta(P_{mu nu}(x)) for the six planes
//     (8 reals each, FP32).  update_kernel assembles the force from A at x and at x - nu:
//        ta(U_mu(x) S_mu(x)) = sum_nu [A_{mu nu}(x) - U_nu(x-nu)^+ A_{mu nu}(x-nu) U_nu(x-nu)]
//     (the lower staple loop is the plaquette at x - nu transported to x and reversed), forms the
//     stage exponent, exponentiates it in closed form (Cayley-Hamilton) and updates its own links
//     into the other buffer of a ping-pong pair (neighbours still read the old links);
//   * the clover field is assembled from the same A: each leaf is a plaquette transported to x,
//     so F_{mu nu}(x) = -i/4 [A(x) + T_{-mu} A(x-mu) + T_{-nu} A(x-nu) + T_{-mu-nu} A(x-mu-nu)];
//   * sites are visited in slabs of bt time slices, (x, y) planes fastest, then t inside a slab,
//     then z, so that the t-neighbours a stencil reads are a few planes away (L2 hits) even when
//     one time slice of links is larger than L2;
//   * lattice sums: per block in FP64, then one block sums the partials in a fixed order
//     (deterministic), writing one observable record on the device.
#include <cuda_runtime.h>

#include <cstdint>

#include "flow.h"

namespace odwf {
namespace flow {
namespace {

constexpr int kBS = 128;   // plaquette and clover kernels: one thread per site
constexpr int kSites = 32;  // update kernel: 32 sites per block, one warp per link direction

// complex fused multiply-adds, four FMAs each
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {  // acc + a b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfma_nc(float2 a, float2 b, float2 acc) {  // acc + a conj(b)
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.y, b.x, acc.y);
    acc.y = fmaf(-a.x, b.y, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfma_cn(float2 a, float2 b, float2 acc) {  // acc + conj(a) b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfms_cn(float2 a, float2 b, float2 acc) {  // acc - conj(a) b
    acc.x = fmaf(-a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(-a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cfma_i(float d, float2 u, float2 acc) {  // acc + (i d) u
    acc.x = fmaf(-d, u.y, acc.x);
    acc.y = fmaf(d, u.x, acc.y);
    return acc;
}

struct M3 {
    float2 m[9];  // row-major
};

// traceless anti-Hermitian 3x3: diag i(d0, d1, -d0-d1), upper z01, z02, z12 (lower = -conj)
struct AH {
    float d0, d1;
    float2 z01, z02, z12;
};

__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.m[3 * i + j] = cfma(a.m[3 * i + 2], b.m[6 + j], cfma(a.m[3 * i + 1], b.m[3 + j], cmul(a.m[3 * i], b.m[j])));
    return c;
}

// ta(a b^+): entries (a b^+)_ij = sum_k a_ik conj(b_jk); also Re tr(a b^+)
__device__ __forceinline__ AH ta_mul_dag(const M3& a, const M3& b, float* retr) {
    float2 p[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float2 s = make_float2(0.f, 0.f);
            s = cfma_nc(a.m[3 * i], b.m[3 * j], s);
            s = cfma_nc(a.m[3 * i + 1], b.m[3 * j + 1], s);
            p[i][j] = cfma_nc(a.m[3 * i + 2], b.m[3 * j + 2], s);
        }
    *retr = p[0][0].x + p[1][1].x + p[2][2].x;
    const float im3 = (p[0][0].y + p[1][1].y + p[2][2].y) * (1.0f / 3.0f);
    AH r;
    r.d0 = p[0][0].y - im3;
    r.d1 = p[1][1].y - im3;
    r.z01 = make_float2(0.5f * (p[0][1].x - p[1][0].x), 0.5f * (p[0][1].y + p[1][0].y));
    r.z02 = make_float2(0.5f * (p[0][2].x - p[2][0].x), 0.5f * (p[0][2].y + p[2][0].y));
    r.z12 = make_float2(0.5f * (p[1][2].x - p[2][1].x), 0.5f * (p[1][2].y + p[2][1].y));
    return r;
}

// ta(u^+ a u) for anti-Hermitian traceless a (the result is already anti-Hermitian; the
// projection only removes the rounding in its trace).  T = a u uses the imaginary diagonal and
// the anti-Hermitian lower triangle of a; only the diagonal and the upper triangle of u^+ T are formed.
__device__ __forceinline__ AH conj_by(const M3& u, const AH& a) {
    const float d2 = -a.d0 - a.d1;
    float2 T[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float2 t0 = make_float2(0.f, 0.f), t1 = t0, t2 = t0;
        t0 = cfma_i(a.d0, u.m[j], t0);
        t0 = cfma(a.z01, u.m[3 + j], t0);
        t0 = cfma(a.z02, u.m[6 + j], t0);
        t1 = cfms_cn(a.z01, u.m[j], t1);
        t1 = cfma_i(a.d1, u.m[3 + j], t1);
        t1 = cfma(a.z12, u.m[6 + j], t1);
        t2 = cfms_cn(a.z02, u.m[j], t2);
        t2 = cfms_cn(a.z12, u.m[3 + j], t2);
        t2 = cfma_i(d2, u.m[6 + j], t2);
        T[j] = t0;
        T[3 + j] = t1;
        T[6 + j] = t2;
    }
    float cd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {  // Im (u^+ T)_ii = sum_k Re u_ki Im T_ki - Im u_ki Re T_ki
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s = fmaf(u.m[3 * k + i].x, T[3 * k + i].y, s);
            s = fmaf(-u.m[3 * k + i].y, T[3 * k + i].x, s);
        }
        cd[i] = s;
    }
    const float im3 = (cd[0] + cd[1] + cd[2]) * (1.0f / 3.0f);
    AH r;
    r.d0 = cd[0] - im3;
    r.d1 = cd[1] - im3;
    float2 z = make_float2(0.f, 0.f);
    z = cfma_cn(u.m[0], T[1], z);
    z = cfma_cn(u.m[3], T[4], z);
    r.z01 = cfma_cn(u.m[6], T[7], z);
    z = make_float2(0.f, 0.f);
    z = cfma_cn(u.m[0], T[2], z);
    z = cfma_cn(u.m[3], T[5], z);
    r.z02 = cfma_cn(u.m[6], T[8], z);
    z = make_float2(0.f, 0.f);
    z = cfma_cn(u.m[1], T[2], z);
    z = cfma_cn(u.m[4], T[5], z);
    r.z12 = cfma_cn(u.m[7], T[8], z);
    return r;
}

__device__ __forceinline__ void ah_axpy(AH& y, float s, const AH& x) {
    y.d0 = fmaf(s, x.d0, y.d0);
    y.d1 = fmaf(s, x.d1, y.d1);
    y.z01.x = fmaf(s, x.z01.x, y.z01.x);
    y.z01.y = fmaf(s, x.z01.y, y.z01.y);
    y.z02.x = fmaf(s, x.z02.x, y.z02.x);
    y.z02.y = fmaf(s, x.z02.y, y.z02.y);
    y.z12.x = fmaf(s, x.z12.x, y.z12.x);
    y.z12.y = fmaf(s, x.z12.y, y.z12.y);
}

__device__ __forceinline__ AH ah_zero() {
    AH r;
    r.d0 = r.d1 = 0.f;
    r.z01 = r.z02 = r.z12 = make_float2(0.f, 0.f);
    return r;
}

// -tr(a b) for traceless anti-Hermitian a, b: sum_i a_i b_i + 2 sum_{i<j} Re(a_ij conj(b_ij))
__device__ __forceinline__ float ah_dot(const AH& a, const AH& b) {
    const float a2 = -a.d0 - a.d1, b2 = -b.d0 - b.d1;
    float s = a.d0 * b.d0 + a.d1 * b.d1 + a2 * b2;
    s += 2.f * (a.z01.x * b.z01.x + a.z01.y * b.z01.y + a.z02.x * b.z02.x + a.z02.y * b.z02.y +
                a.z12.x * b.z12.x + a.z12.y * b.z12.y);
    return s;
}

__device__ __forceinline__ int plane_of(int mu, int nu) {  // mu < nu
    return mu == 0 ? nu - 1 : (mu == 1 ? nu + 1 : 5);
}

// ---------------------------------------------------------------------------------------------
// site traversal and neighbours

struct Site {
    size_t s;  // lexicographic index
    int c[4];
};

__device__ __forceinline__ bool site_of(const FlowGeom& g, size_t i, Site& st) {
    if (i >= g.V) return false;
    const size_t P = (size_t)g.L[0] * g.L[1];
    const size_t k = i / P;
    const size_t j = i - k * P;
    const size_t lzbt = (size_t)g.L[2] * g.bt;
    const size_t slab = k / lzbt;
    const int r = (int)(k - slab * lzbt);
    const int z = r / g.bt;
    const int t = (int)(slab * g.bt) + (r - z * g.bt);
    st.c[0] = (int)(j % g.L[0]);
    st.c[1] = (int)(j / g.L[0]);
    st.c[2] = z;
    st.c[3] = t;
    st.s = j + P * ((size_t)z + (size_t)g.L[2] * t);
    return true;
}

__device__ __forceinline__ size_t step(const FlowGeom& g, const Site& st, int mu, int dir) {
    const int x = st.c[mu];
    if (dir > 0) return x + 1 == g.L[mu] ? st.s - (size_t)(g.L[mu] - 1) * g.stride[mu] : st.s + g.stride[mu];
    return x == 0 ? st.s + (size_t)(g.L[mu] - 1) * g.stride[mu] : st.s - g.stride[mu];
}

// step from an arbitrary lexicographic index whose coordinate along mu is x
__device__ __forceinline__ size_t step_from(const FlowGeom& g, size_t s, int x, int mu, int dir) {
    if (dir > 0) return x + 1 == g.L[mu] ? s - (size_t)(g.L[mu] - 1) * g.stride[mu] : s + g.stride[mu];
    return x == 0 ? s + (size_t)(g.L[mu] - 1) * g.stride[mu] : s - g.stride[mu];
}

// third row of an SU(3) matrix from the first two: conj(row0 x row1)
__device__ __forceinline__ void third_row(M3& u) {
    const float2* a = u.m;
    const float2* b = u.m + 3;
    const float2 c0 = cfma(make_float2(-a[2].x, -a[2].y), b[1], cmul(a[1], b[2]));
    const float2 c1 = cfma(make_float2(-a[0].x, -a[0].y), b[2], cmul(a[2], b[0]));
    const float2 c2 = cfma(make_float2(-a[1].x, -a[1].y), b[0], cmul(a[0], b[1]));
    u.m[6] = make_float2(c0.x, -c0.y);
    u.m[7] = make_float2(c1.x, -c1.y);
    u.m[8] = make_float2(c2.x, -c2.y);
}

// links are stored as their first two rows, three float4 (two complex entries each) per link
__device__ __forceinline__ void load_rows(const float4* __restrict__ L4, size_t V, int mu, size_t s, M3& u) {
    const float4* p = L4 + (size_t)mu * 3 * V + s;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float4 v = __ldg(p + (size_t)j * V);
        u.m[2 * j] = make_float2(v.x, v.y);
        u.m[2 * j + 1] = make_float2(v.z, v.w);
    }
}

__device__ __forceinline__ M3 load_link(const float4* __restrict__ hi, size_t V, int mu, size_t s) {
    M3 u;
    load_rows(hi, V, mu, s, u);
    third_row(u);
    return u;
}

__device__ __forceinline__ AH load_ah(const float4* __restrict__ A, size_t V, int p, size_t s) {
    const float4 a = __ldg(A + (size_t)(2 * p) * V + s);
    const float4 b = __ldg(A + (size_t)(2 * p + 1) * V + s);
    AH r;
    r.d0 = a.x;
    r.d1 = a.y;
    r.z01 = make_float2(a.z, a.w);
    r.z02 = make_float2(b.x, b.y);
    r.z12 = make_float2(b.z, b.w);
    return r;
}

// the carried stage combination K is read and then rewritten by the same thread: plain loads
__device__ __forceinline__ AH load_ah_rw(const float4* A, size_t V, int p, size_t s) {
    const float4 a = A[(size_t)(2 * p) * V + s];
    const float4 b = A[(size_t)(2 * p + 1) * V + s];
    AH r;
    r.d0 = a.x;
    r.d1 = a.y;
    r.z01 = make_float2(a.z, a.w);
    r.z02 = make_float2(b.x, b.y);
    r.z12 = make_float2(b.z, b.w);
    return r;
}

__device__ __forceinline__ void store_ah(float4* A, size_t V, int p, size_t s, const AH& r) {
    A[(size_t)(2 * p) * V + s] = make_float4(r.d0, r.d1, r.z01.x, r.z01.y);
    A[(size_t)(2 * p + 1) * V + s] = make_float4(r.z02.x, r.z02.y, r.z12.x, r.z12.y);
}

// ---------------------------------------------------------------------------------------------
// block reductions (fixed order)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

template <int NT>
__device__ __forceinline__ void block_sum2(double a, double b, double* out_a, double* out_b) {
    __shared__ double sa[NT / 32], sb[NT / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0, tb = 0;
        for (int i = 0; i < NT / 32; ++i) {
            ta += sa[i];
            tb += sb[i];
        }
        *out_a = ta;
        *out_b = tb;
    }
}

template <int NT>
__device__ __forceinline__ void block_sum_min(double a, float m, double* out_a, float* out_m) {
    __shared__ double sa[NT / 32];
    __shared__ float sm[NT / 32];
    a = warp_sum(a);
    m = warp_min(m);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = a;
        sm[w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0;
        float tm = sm[0];
        for (int i = 0; i < NT / 32; ++i) {
            ta += sa[i];
            tm = fminf(tm, sm[i]);
        }
        *out_a = ta;
        *out_m = tm;
    }
}

// ---------------------------------------------------------------------------------------------
// kernels

// A_{mu nu}(x) = ta(P_{mu nu}(x)) for the six planes, one thread per site.  With MEASURE,
// per-block sum and minimum of Re tr P over the block's plaquettes.
// rows 0 and 1 of a b (a given by its first two rows), row 2 rebuilt: a b is in SU(3)
__device__ __forceinline__ M3 mul_rows01(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.m[3 * i + j] = cfma(a.m[3 * i + 2], b.m[6 + j], cfma(a.m[3 * i + 1], b.m[3 + j], cmul(a.m[3 * i], b.m[j])));
    third_row(c);
    return c;
}

// A_{mu nu}(x) = ta(P_{mu nu}(x)) for the six planes, one thread per site.  The site's own four
// links are read once and kept as their first two rows (they are only ever left factors); the
// two products of each plaquette are formed as two rows with the third rebuilt (they are SU(3)).
// With MEASURE, per-block sum and minimum of Re tr P over the block's plaquettes.
template <bool MEASURE>
__global__ void __launch_bounds__(kBS) plaq_kernel(FlowGeom g, const float4* __restrict__ hi, float4* __restrict__ A,
                                                   double* __restrict__ part_retr, float* __restrict__ part_min) {
    Site st;
    const bool ok = site_of(g, (size_t)blockIdx.x * kBS + threadIdx.x, st);
    double rsum = 0.0;
    float rmin = 3.0f;
    if (ok) {
        M3 own[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) load_rows(hi, g.V, mu, st.s, own[mu]);
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            const size_t xm = step(g, st, mu, +1);
#pragma unroll
            for (int nu = mu + 1; nu < 4; ++nu) {
                const size_t xn = step(g, st, nu, +1);
                const M3 t1 = mul_rows01(own[mu], load_link(hi, g.V, nu, xm));  // U_mu(x) U_nu(x+mu)
                const M3 t2 = mul_rows01(own[nu], load_link(hi, g.V, mu, xn));  // U_nu(x) U_mu(x+nu)
                float retr;
                store_ah(A, g.V, plane_of(mu, nu), st.s, ta_mul_dag(t1, t2, &retr));
                if (MEASURE) {
                    rsum += retr;
                    rmin = fminf(rmin, retr);
                }
            }
        }
    }
    if (MEASURE) block_sum_min<kBS>(rsum, rmin, part_retr + blockIdx.x, part_min + blockIdx.x);
}

// exp(X) - 1 for traceless anti-Hermitian X by Cayley-Hamilton: X^3 = s X + d 1 with
// s = tr(X^2)/2 and d = tr(X^3)/3, so X^n = a_n 1 + b_n X + c_n X^2 with
// (a, b, c)_{n+1} = (c_n d, a_n + c_n s, b_n); the exponential series is summed on the scalars
// until the terms fall below 1e-10 of the leading ones.
__device__ __forceinline__ M3 expm1_ah(const AH& x) {
    const float d2 = -x.d0 - x.d1;
    // X^2 is Hermitian: (X^2)_ii = -sum_k |X_ik|^2, (X^2)_ij = sum_k X_ik X_kj (i < j)
    const float n01 = x.z01.x * x.z01.x + x.z01.y * x.z01.y;
    const float n02 = x.z02.x * x.z02.x + x.z02.y * x.z02.y;
    const float n12 = x.z12.x * x.z12.x + x.z12.y * x.z12.y;
    const float q0 = -(x.d0 * x.d0 + n01 + n02);
    const float q1 = -(x.d1 * x.d1 + n01 + n12);
    const float q2 = -(d2 * d2 + n02 + n12);
    // X_00 X_01 + X_01 X_11 + X_02 X_21 = i (d0 + d1) z01 - z02 conj(z12)
    float2 q01 = make_float2(-(x.d0 + x.d1) * x.z01.y, (x.d0 + x.d1) * x.z01.x);
    q01 = make_float2(q01.x - (x.z02.x * x.z12.x + x.z02.y * x.z12.y), q01.y - (x.z02.y * x.z12.x - x.z02.x * x.z12.y));
    // X_00 X_02 + X_01 X_12 + X_02 X_22 = i (d0 + d2) z02 + z01 z12
    float2 q02 = cmul(x.z01, x.z12);
    q02 = cfma_i(x.d0 + d2, x.z02, q02);
    // X_10 X_02 + X_11 X_12 + X_12 X_22 = -conj(z01) z02 + i (d1 + d2) z12
    float2 q12 = make_float2(0.f, 0.f);
    q12 = cfms_cn(x.z01, x.z02, q12);
    q12 = cfma_i(x.d1 + d2, x.z12, q12);
    const float s = 0.5f * (q0 + q1 + q2);
    // d = tr(X X^2)/3 = (i/3) [sum_i d_i q_i + 2 sum_{i<j} Im(X_ij conj(q_ij))]
    float dim = x.d0 * q0 + x.d1 * q1 + d2 * q2;
    dim += 2.f * ((x.z01.y * q01.x - x.z01.x * q01.y) + (x.z02.y * q02.x - x.z02.x * q02.y) +
                  (x.z12.y * q12.x - x.z12.x * q12.y));
    dim *= (1.0f / 3.0f);
    const float nrm = sqrtf(fmaxf(-2.0f * s, 0.f));  // Frobenius norm of X
    // the n = 1 and n = 2 terms (X and X^2/2) are in f1, f2; (a, b, c) holds the state of n = 2
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f), c = make_float2(1.f, 0.f);
    float2 f0 = make_float2(0.f, 0.f), f1 = make_float2(1.f, 0.f), f2 = make_float2(0.5f, 0.f);
    float inv_fact = 0.5f, bound = 0.5f * nrm * nrm;
#pragma unroll 1
    for (int n = 3; n < 64; ++n) {
        // (a, b, c) <- (c d, a + c s, b), d = i dim
        const float2 na = make_float2(-c.y * dim, c.x * dim);
        const float2 nb = make_float2(fmaf(c.x, s, a.x), fmaf(c.y, s, a.y));
        a = na;
        c = b;
        b = nb;
        inv_fact /= (float)n;
        f0.x = fmaf(a.x, inv_fact, f0.x);
        f0.y = fmaf(a.y, inv_fact, f0.y);
        f1.x = fmaf(b.x, inv_fact, f1.x);
        f1.y = fmaf(b.y, inv_fact, f1.y);
        f2.x = fmaf(c.x, inv_fact, f2.x);
        f2.y = fmaf(c.y, inv_fact, f2.y);
        bound *= nrm / (float)n;
        if (bound < 1e-10f * fmaxf(nrm, 1e-30f) || bound == 0.f) break;
    }
    // E1 = f0 1 + f1 X + f2 X^2
    M3 e;
    e.m[0] = cadd(f0, cadd(cmul(f1, make_float2(0.f, x.d0)), make_float2(f2.x * q0, f2.y * q0)));
    e.m[4] = cadd(f0, cadd(cmul(f1, make_float2(0.f, x.d1)), make_float2(f2.x * q1, f2.y * q1)));
    e.m[8] = cadd(f0, cadd(cmul(f1, make_float2(0.f, d2)), make_float2(f2.x * q2, f2.y * q2)));
    e.m[1] = cfma(f2, q01, cmul(f1, x.z01));
    e.m[2] = cfma(f2, q02, cmul(f1, x.z02));
    e.m[5] = cfma(f2, q12, cmul(f1, x.z12));
    // lower triangle: X_ji = -conj(X_ij), (X^2)_ji = conj((X^2)_ij)
    e.m[3] = cfma(f2, make_float2(q01.x, -q01.y), cmul(f1, make_float2(-x.z01.x, x.z01.y)));
    e.m[6] = cfma(f2, make_float2(q02.x, -q02.y), cmul(f1, make_float2(-x.z02.x, x.z02.y)));
    e.m[7] = cfma(f2, make_float2(q12.x, -q12.y), cmul(f1, make_float2(-x.z12.x, x.z12.y)));
    return e;
}

// error-free hi + d, with the rounding error carried into lo
__device__ __forceinline__ void ff_add(float& hi, float& lo, float d) {
    const float s = hi + d;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (d - bb);
    const float l = lo + err;
    const float h2 = s + l;
    lo = l - (h2 - s);
    hi = h2;
}

// One Runge-Kutta stage: 32 sites per block, warp mu updates U_mu.  Force from A, exponent X
// (and the carried combination K), and W <- exp(X) W into the other link buffer.
template <int STAGE>
__global__ void __launch_bounds__(4 * kSites) update_kernel(FlowGeom g, const float4* __restrict__ hi,
                                                            const float4* __restrict__ lo, float4* __restrict__ hi_out,
                                                            float4* __restrict__ lo_out, const float4* __restrict__ A,
                                                            float4* __restrict__ K, float eps) {
    const int mu = threadIdx.x >> 5;
    Site st;
    if (!site_of(g, (size_t)blockIdx.x * kSites + (threadIdx.x & 31), st)) return;
    // Z_mu = sum_{nu != mu} [-A_{mu nu}(x) + U_nu(x-nu)^+ A_{mu nu}(x-nu) U_nu(x-nu)],  A_{nu mu} = -A_{mu nu}
    AH z = ah_zero();
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const int p = mu < nu ? plane_of(mu, nu) : plane_of(nu, mu);
        const float sg = mu < nu ? 1.f : -1.f;
        ah_axpy(z, -sg, load_ah(A, g.V, p, st.s));
        const size_t xb = step(g, st, nu, -1);
        ah_axpy(z, sg, conj_by(load_link(hi, g.V, nu, xb), load_ah(A, g.V, p, xb)));
    }
    constexpr float cz = STAGE == 0 ? 0.25f : (STAGE == 1 ? 8.0f / 9.0f : 0.75f);
    AH x = ah_zero();
    ah_axpy(x, cz * eps, z);
    if (STAGE > 0) ah_axpy(x, STAGE == 1 ? -17.0f / 36.0f : -1.0f, load_ah_rw(K, g.V, mu, st.s));
    if (STAGE == 0) {
        AH k = ah_zero();
        ah_axpy(k, eps, z);
        store_ah(K, g.V, mu, st.s, k);
    } else if (STAGE == 1) {
        store_ah(K, g.V, mu, st.s, x);
    }
    const M3 e1 = expm1_ah(x);
    M3 w;
    load_rows(hi, g.V, mu, st.s, w);
    third_row(w);
    // rows 0 and 1 of exp(X) W = W + E1 W; the third row stays implicit
    float2 d[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            d[3 * i + j] = cfma(e1.m[3 * i + 2], w.m[6 + j], cfma(e1.m[3 * i + 1], w.m[3 + j], cmul(e1.m[3 * i], w.m[j])));
    const size_t base = (size_t)mu * 3 * g.V + st.s;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float4 h = make_float4(w.m[2 * j].x, w.m[2 * j].y, w.m[2 * j + 1].x, w.m[2 * j + 1].y);
        float4 l = __ldg(lo + base + (size_t)j * g.V);
        ff_add(h.x, l.x, d[2 * j].x);
        ff_add(h.y, l.y, d[2 * j].y);
        ff_add(h.z, l.z, d[2 * j + 1].x);
        ff_add(h.w, l.w, d[2 * j + 1].y);
        hi_out[base + (size_t)j * g.V] = h;
        lo_out[base + (size_t)j * g.V] = l;
    }
}

// Clover field strength from A and the per-site energy density and charge density; per-block
// sums (and optional per-site outputs).
__global__ void __launch_bounds__(kBS, 2) clover_kernel(FlowGeom g, const float4* __restrict__ hi,
                                                        const float4* __restrict__ A, double* __restrict__ part_e,
                                                        double* __restrict__ part_q, float* __restrict__ e_site,
                                                        float* __restrict__ q_site) {
    Site st;
    const bool ok = site_of(g, (size_t)blockIdx.x * kBS + threadIdx.x, st);
    double e = 0.0, q = 0.0;
    if (ok) {
        AH f[6];
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            const size_t xm = step(g, st, mu, -1);
            const M3 u1 = load_link(hi, g.V, mu, xm);  // U_mu(x-mu)
#pragma unroll
            for (int nu = mu + 1; nu < 4; ++nu) {
                const int p = plane_of(mu, nu);
                const size_t xn = step(g, st, nu, -1);
                const size_t xmn = step_from(g, xm, st.c[nu], nu, -1);  // x - mu - nu
                AH acc = load_ah(A, g.V, p, st.s);
                ah_axpy(acc, 1.f, conj_by(u1, load_ah(A, g.V, p, xm)));
                const M3 u2 = load_link(hi, g.V, nu, xn);  // U_nu(x-nu)
                ah_axpy(acc, 1.f, conj_by(u2, load_ah(A, g.V, p, xn)));
                const M3 c = mul(load_link(hi, g.V, mu, xmn), u2);  // U_mu(x-mu-nu) U_nu(x-nu)
                ah_axpy(acc, 1.f, conj_by(c, load_ah(A, g.V, p, xmn)));
                AH r = ah_zero();
                ah_axpy(r, 0.25f, acc);
                f[p] = r;
            }
        }
        float ef = 0.f;
#pragma unroll
        for (int p = 0; p < 6; ++p) ef += ah_dot(f[p], f[p]);
        // planes: 0 xy, 1 xz, 2 xt, 3 yz, 4 yt, 5 zt
        const float qf = (ah_dot(f[0], f[5]) - ah_dot(f[1], f[4]) + ah_dot(f[2], f[3])) *
                         (float)(1.0 / (4.0 * 3.14159265358979323846 * 3.14159265358979323846));
        e = ef;
        q = qf;
        if (e_site) e_site[st.s] = ef;
        if (q_site) q_site[st.s] = qf;
    }
    block_sum2<kBS>(e, q, part_e + blockIdx.x, part_q + blockIdx.x);
}

// One block: sums the per-block partials in a fixed order and writes one observable record.
constexpr int kRed = 256;
__global__ void __launch_bounds__(kRed) reduce_kernel(int nb_plaq, int nb_clover, const double* __restrict__ part_retr,
                                                      const float* __restrict__ part_min, const double* __restrict__ part_e,
                                                      const double* __restrict__ part_q, double t, double V,
                                                      FlowObsDev* __restrict__ out) {
    double r = 0, e = 0, q = 0;
    float m = 3.0f;
    for (int i = threadIdx.x; i < nb_plaq; i += kRed) {
        r += part_retr[i];
        m = fminf(m, part_min[i]);
    }
    for (int i = threadIdx.x; i < nb_clover; i += kRed) {
        e += part_e[i];
        q += part_q[i];
    }
    __shared__ double sr[kRed], se[kRed], sq[kRed];
    __shared__ float sm[kRed];
    sr[threadIdx.x] = r;
    se[threadIdx.x] = e;
    sq[threadIdx.x] = q;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int w = kRed / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            se[threadIdx.x] += se[threadIdx.x + w];
            sq[threadIdx.x] += sq[threadIdx.x + w];
            sm[threadIdx.x] = fminf(sm[threadIdx.x], sm[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->t = t;
        out->e_plaq = 2.0 * (18.0 * V - sr[0]) / V;  // 2 sum_{6 planes} (3 - Re tr P), site average
        out->e_clover = se[0] / V;
        out->q_clover = sq[0];
        out->plaq_min = (double)sm[0] / 3.0;
        out->plaq_mean = sr[0] / (18.0 * V);
    }
}

// external complex128 U[mu][site][a][b] <-> float-float pairs of the first two rows [mu][j][site]
// (float4 j holds entries 2j and 2j+1); the third row is rebuilt from the first two in FP64
__global__ void split_kernel(const double2* __restrict__ U, float4* __restrict__ hi, float4* __restrict__ lo, size_t V,
                             int mu) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * V) return;
    const size_t s = i / 3;
    const int j = (int)(i - s * 3);
    const double2 u0 = U[s * 9 + 2 * j], u1 = U[s * 9 + 2 * j + 1];
    const float4 h = make_float4((float)u0.x, (float)u0.y, (float)u1.x, (float)u1.y);
    const size_t o = ((size_t)mu * 3 + j) * V + s;
    hi[o] = h;
    lo[o] = make_float4((float)(u0.x - (double)h.x), (float)(u0.y - (double)h.y), (float)(u1.x - (double)h.z),
                        (float)(u1.y - (double)h.w));
}

__global__ void join_kernel(const float4* __restrict__ hi, const float4* __restrict__ lo, double2* __restrict__ U, size_t V,
                            int mu) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    double2 m[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const size_t o = ((size_t)mu * 3 + j) * V + s;
        const float4 h = hi[o], l = lo[o];
        m[2 * j] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
        m[2 * j + 1] = make_double2((double)h.z + (double)l.z, (double)h.w + (double)l.w);
    }
    // row 2 = conj(row0 x row1)
    const double2 *a = m, *b = m + 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const double re = (a[k1].x * b[k2].x - a[k1].y * b[k2].y) - (a[k2].x * b[k1].x - a[k2].y * b[k1].y);
        const double im = (a[k1].x * b[k2].y + a[k1].y * b[k2].x) - (a[k2].x * b[k1].y + a[k2].y * b[k1].x);
        m[6 + k] = make_double2(re, -im);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) U[s * 9 + k] = m[k];
}

}  // namespace

size_t plaq_blocks(const FlowGeom& g) { return (g.V + kBS - 1) / kBS; }
size_t update_blocks(const FlowGeom& g) { return (g.V + kSites - 1) / kSites; }
size_t clover_blocks(const FlowGeom& g) { return (g.V + kBS - 1) / kBS; }

cudaError_t launch_plaq(const FlowGeom& g, const float4* hi, float4* A, double* part_retr, float* part_min, bool measure,
                        cudaStream_t st) {
    const dim3 grid((unsigned)plaq_blocks(g));
    if (measure)
        plaq_kernel<true><<<grid, kBS, 0, st>>>(g, hi, A, part_retr, part_min);
    else
        plaq_kernel<false><<<grid, kBS, 0, st>>>(g, hi, A, part_retr, part_min);
    return cudaGetLastError();
}

cudaError_t launch_update(const FlowGeom& g, int stage, const float4* hi, const float4* lo, float4* hi_out,
                          float4* lo_out, const float4* A, float4* K, float eps, cudaStream_t st) {
    const dim3 grid((unsigned)update_blocks(g));
    if (stage == 0)
        update_kernel<0><<<grid, 4 * kSites, 0, st>>>(g, hi, lo, hi_out, lo_out, A, K, eps);
    else if (stage == 1)
        update_kernel<1><<<grid, 4 * kSites, 0, st>>>(g, hi, lo, hi_out, lo_out, A, K, eps);
    else
        update_kernel<2><<<grid, 4 * kSites, 0, st>>>(g, hi, lo, hi_out, lo_out, A, K, eps);
    return cudaGetLastError();
}

cudaError_t launch_clover(const FlowGeom& g, const float4* hi, const float4* A, double* part_e, double* part_q,
                          float* e_site, float* q_site, cudaStream_t st) {
    clover_kernel<<<(unsigned)clover_blocks(g), kBS, 0, st>>>(g, hi, A, part_e, part_q, e_site, q_site);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const FlowGeom& g, const double* part_retr, const float* part_min, const double* part_e,
                          const double* part_q, double t, FlowObsDev* out, cudaStream_t st) {
    reduce_kernel<<<1, kRed, 0, st>>>((int)plaq_blocks(g), (int)clover_blocks(g), part_retr, part_min, part_e, part_q, t,
                                      (double)g.V, out);
    return cudaGetLastError();
}

cudaError_t launch_split(const double2* U, float4* hi, float4* lo, size_t V, int mu, cudaStream_t st) {
    const size_t n = 3 * V;
    split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, hi, lo, V, mu);
    return cudaGetLastError();
}

cudaError_t launch_join(const float4* hi, const float4* lo, double2* U, size_t V, int mu, cudaStream_t st) {
    const size_t n = V;
    join_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(hi, lo, U, V, mu);
    return cudaGetLastError();
}

}  // namespace flow
}  // namespace odwf
