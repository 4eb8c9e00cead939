// Kernel templates of the ODWF library (instantiated in kernels_f64.cu / kernels_mixed.cu).
//
// The fused hopping kernel computes, for every output site x of parity p_out and every s,
//   non-dagger:  y = W (B psi),     H psi     = -1/2 y
//   dagger:      y = W^dag psi,     H^dag psi = -1/2 B^dag y
// with W = sum_mu [(1 - gamma_mu) U_mu(x) delta_{x+mu} + (1 + gamma_mu) U_mu(x-mu)^dag delta_{x-mu}]
// (W^dag swaps the projectors), B = rho + sigma L (Sec. 2's operator, written as
// D = D_w B + 1 - L, D_w = (4 - m0) - W/2), followed by a fused epilogue:
//   res = zop(z) + sign * hop_op(H psi),   zop in {none, 1, M, M^dag}, hop_op in {1, M^-1, M^-dag}
//   [norm: accumulate |res|^2]  [post: res <- M^-1 res or M^-dag res]
//   [resid: out = b - res, norm of out]  [cg: r -= alpha res, x += alpha p, norm of r]
// Reductions are deterministic: per-block FP64 partials, summed in fixed order by the
// last block to finish, which also updates the per-system CG scalars.
#pragma once

#include "odwf_internal.h"

namespace odwf {

// ---------------------------------------------------------------- epilogue flags
enum : int {
    F_DAG = 1 << 0,
    F_ZOP_SHIFT = 1, F_ZOP_MASK = 3 << 1,  // 0 none, 1 identity, 2 M, 3 M^dag
    F_HOP_SHIFT = 3, F_HOP_MASK = 3 << 3,  // 0 identity, 1 M^-1, 2 M^-dag
    F_NEG = 1 << 5,
    F_POST_SHIFT = 6, F_POST_MASK = 3 << 6,  // 0 none, 1 M^-1, 2 M^-dag
    F_NORM = 1 << 8,
    F_CG = 1 << 9,
    F_RESID = 1 << 10,
    F_FIN_SHIFT = 11, F_FIN_MASK = 3 << 11,  // 0 store sum, 1 alpha, 2 beta
};
enum { ZOP_NONE = 0, ZOP_ID = 1, ZOP_M = 2, ZOP_MDAG = 3 };
enum { OP_ID = 0, OP_MINV = 1, OP_MINVDAG = 2 };
enum { FIN_STORE = 0, FIN_ALPHA = 1, FIN_BETA = 2 };

constexpr int mkflags(bool dag, int zop, int hop, bool neg, int post, bool norm, bool cg, bool resid, int fin) {
    return (dag ? F_DAG : 0) | (zop << F_ZOP_SHIFT) | (hop << F_HOP_SHIFT) | (neg ? F_NEG : 0) |
           (post << F_POST_SHIFT) | (norm ? F_NORM : 0) | (cg ? F_CG : 0) | (resid ? F_RESID : 0) |
           (fin << F_FIN_SHIFT);
}

// Named epilogues of the solver (see solver.cpp for where each is used)
constexpr int EPI_MINV = mkflags(false, ZOP_NONE, OP_MINV, false, 0, false, false, false, 0);       // t = M^-1 H p
constexpr int EPI_SCHUR = mkflags(false, ZOP_ID, OP_MINV, true, 0, false, false, false, 0);        // z - M^-1 H t
constexpr int EPI_SCHUR_NORM_MDINV =                                                               // M^-dag (z - M^-1 H t), |.|^2 -> alpha
    mkflags(false, ZOP_ID, OP_MINV, true, OP_MINVDAG, true, false, false, FIN_ALPHA);
constexpr int EPI_SCHUR_NORM_MDINV_STORE =
    mkflags(false, ZOP_ID, OP_MINV, true, OP_MINVDAG, false, false, false, 0);
constexpr int EPI_FULL = mkflags(false, ZOP_M, OP_ID, false, 0, false, false, false, 0);           // M z + H p
constexpr int EPI_PLAIN = mkflags(false, ZOP_NONE, OP_ID, false, 0, false, false, false, 0);       // H p
constexpr int EPI_ZMINUS_POSTMINV = mkflags(false, ZOP_ID, OP_ID, true, OP_MINV, false, false, false, 0);  // M^-1 (z - H p)
constexpr int EPI_ZMINUS = mkflags(false, ZOP_ID, OP_ID, true, 0, false, false, false, 0);         // z - H p
constexpr int EPID_MINVDAG = mkflags(true, ZOP_NONE, OP_MINVDAG, false, 0, false, false, false, 0);  // M^-dag H^dag a
constexpr int EPID_NORMAL = mkflags(true, ZOP_MDAG, OP_ID, true, 0, false, false, false, 0);         // M^dag z - H^dag c
constexpr int EPID_NORMAL_CG =                                                                        // fused CG update
    mkflags(true, ZOP_MDAG, OP_ID, true, 0, false, true, false, FIN_BETA);
constexpr int EPID_NORMAL_RESID =                                                                     // b - (M^dag z - H^dag c)
    mkflags(true, ZOP_MDAG, OP_ID, true, 0, false, false, true, FIN_STORE);
constexpr int EPID_ZMINUS = mkflags(true, ZOP_ID, OP_ID, true, 0, false, false, false, 0);           // z - H^dag c
constexpr int EPID_FULL = mkflags(true, ZOP_MDAG, OP_ID, false, 0, false, false, false, 0);          // M^dag z + H^dag p
constexpr int EPID_PLAIN = mkflags(true, ZOP_NONE, OP_ID, false, 0, false, false, false, 0);         // H^dag p
constexpr int EPID_SCHUR2 = mkflags(true, ZOP_ID, OP_MINVDAG, true, 0, false, false, false, 0);      // z - M^-dag H^dag t
constexpr int EPID_ZMINUS_POSTMINVDAG = mkflags(true, ZOP_ID, OP_ID, true, OP_MINVDAG, false, false, false, 0);

// ---------------------------------------------------------------- kernel parameters
struct FieldRef {
    void* data;
    float* norm;          // scales of FP16/BF16 fields (nullptr otherwise)
    size_t sys_stride;    // bytes between systems
    size_t norm_stride;   // floats between systems
    __device__ __forceinline__ void* d(int sys) const { return (char*)data + sys * sys_stride; }
    __device__ __forceinline__ float* n(int sys) const { return norm ? norm + sys * norm_stride : nullptr; }
};

template <class R>
struct HopParams {
    Geom g;
    int ns;
    int lg_ns;
    int p_out;           // parity of the output sites
    int preshifted;      // non-dagger hops: `in` already holds chi = B psi (skip B per neighbour)
    FieldRef in, z, out;
    FieldRef cg_r, cg_x, cg_p;  // F_CG: r and x (accumulator format), p (input format)
    FieldRef b;                 // F_RESID: right-hand side (accumulator format)
    const void* links;
    const int* nbr;             // neighbour table (second-generation hops), see launch_build_neighbours
    const double* r_sys;        // per-system r = m_q / (2 m0)
    int gate;                   // 1: run only systems whose st[sys].status == need_status
    int need_status;
    SysState* st;               // per-system scalars (gate / norm / cg / resid)
    double* partials;           // [sys][part_stride] (part_stride 0: gridDim.x)
    int part_stride;            // partials per system, fixed for every launch of one batch
    unsigned* counters;         // [sys]
    int sys_base;               // system index offset (blockIdx.y + sys_base)
    unsigned long long* prof_count;  // optional: counts running (system, launch) pairs
    unsigned* bounds_flag;           // debug builds: where out-of-range indices are recorded
    Coef5<R> cf;
};

// ---------------------------------------------------------------- spin algebra (chiral basis)
// gamma_mu = [[0, G_mu], [G_mu^dag, 0]]:  G_1 = -i s1, G_2 = -i s2, G_3 = -i s3, G_4 = 1.
// (1 + sg gamma_mu) chi = [h ; sg G^dag h] with h = chi^up + sg G chi^dn.
template <class R>
__device__ __forceinline__ void project(int mu, R sg, const R v[24], R h[12]) {
    // v index: (spin*3 + col)*2 + reim; up spins 0,1 (v[0..11]), down spins 2,3 (v[12..23])
    const R* u0 = v;
    const R* u1 = v + 6;
    const R* d0 = v + 12;
    const R* d1 = v + 18;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R g0r, g0i, g1r, g1i;  // (G chi^dn) spin 0 and 1
        switch (mu) {
            case 0:  // G = -i s1: (-i d1, -i d0)
                g0r = d1[2 * c + 1]; g0i = -d1[2 * c];
                g1r = d0[2 * c + 1]; g1i = -d0[2 * c];
                break;
            case 1:  // G = -i s2 = [[0,-1],[1,0]]: (-d1, d0)
                g0r = -d1[2 * c]; g0i = -d1[2 * c + 1];
                g1r = d0[2 * c]; g1i = d0[2 * c + 1];
                break;
            case 2:  // G = -i s3: (-i d0, i d1)
                g0r = d0[2 * c + 1]; g0i = -d0[2 * c];
                g1r = -d1[2 * c + 1]; g1i = d1[2 * c];
                break;
            default:  // G = 1
                g0r = d0[2 * c]; g0i = d0[2 * c + 1];
                g1r = d1[2 * c]; g1i = d1[2 * c + 1];
                break;
        }
        h[2 * c] = u0[2 * c] + sg * g0r;
        h[2 * c + 1] = u0[2 * c + 1] + sg * g0i;
        h[6 + 2 * c] = u1[2 * c] + sg * g1r;
        h[6 + 2 * c + 1] = u1[2 * c + 1] + sg * g1i;
    }
}

// acc += [w ; sg G^dag w]
template <class R>
__device__ __forceinline__ void accumulate(int mu, R sg, const R w[12], R acc[24]) {
    const R* w0 = w;
    const R* w1 = w + 6;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[2 * c] += w0[2 * c];
        acc[2 * c + 1] += w0[2 * c + 1];
        acc[6 + 2 * c] += w1[2 * c];
        acc[6 + 2 * c + 1] += w1[2 * c + 1];
        R l0r, l0i, l1r, l1i;  // G^dag w, spins 0 and 1
        switch (mu) {
            case 0:  // G^dag = i s1: (i w1, i w0)
                l0r = -w1[2 * c + 1]; l0i = w1[2 * c];
                l1r = -w0[2 * c + 1]; l1i = w0[2 * c];
                break;
            case 1:  // G^dag = [[0,1],[-1,0]]: (w1, -w0)
                l0r = w1[2 * c]; l0i = w1[2 * c + 1];
                l1r = -w0[2 * c]; l1i = -w0[2 * c + 1];
                break;
            case 2:  // G^dag = i s3: (i w0, -i w1)
                l0r = -w0[2 * c + 1]; l0i = w0[2 * c];
                l1r = w1[2 * c + 1]; l1i = -w1[2 * c];
                break;
            default:
                l0r = w0[2 * c]; l0i = w0[2 * c + 1];
                l1r = w1[2 * c]; l1i = w1[2 * c + 1];
                break;
        }
        acc[12 + 2 * c] += sg * l0r;
        acc[12 + 2 * c + 1] += sg * l0i;
        acc[18 + 2 * c] += sg * l1r;
        acc[18 + 2 * c + 1] += sg * l1i;
    }
}

// w = U h (dag = false) or U^dag h (dag = true) for both spins of the half spinor
template <class R>
__device__ __forceinline__ void su3_mul(const R u[18], const R h[12], R w[12], bool dag) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R re = 0, im = 0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int ix = dag ? (3 * b + a) : (3 * a + b);
                const R ur = u[2 * ix], ui = dag ? -u[2 * ix + 1] : u[2 * ix + 1];
                const R hr = h[6 * sp + 2 * b], hi = h[6 * sp + 2 * b + 1];
                re += ur * hr - ui * hi;
                im += ur * hi + ui * hr;
            }
            w[6 * sp + 2 * a] = re;
            w[6 * sp + 2 * a + 1] = im;
        }
}

// Float-float instance: each output component is a six-term dot product, summed as a compensated
// dot product (two-product of the leading parts plus the cross terms, two-sum of the running
// total, the rounding errors gathered in a second word and added once at the end), as accurate as
// the float-float operators of ff.cuh with about two thirds of their FP32 operations.
__device__ __forceinline__ void ff_dot_acc(float& s, float& c, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);  // ah bh - p, exact
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));  // s + p - t, exact
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}
__device__ __forceinline__ void su3_mul(const ff u[18], const ff h[12], ff w[12], bool dag) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int ix = dag ? (3 * b + a) : (3 * a + b);
                const ff ur = u[2 * ix], ui = dag ? -u[2 * ix + 1] : u[2 * ix + 1];
                const ff hr = h[6 * sp + 2 * b], hi = h[6 * sp + 2 * b + 1];
                ff_dot_acc(rs, rc, ur.hi, ur.lo, hr.hi, hr.lo);
                ff_dot_acc(rs, rc, -ui.hi, -ui.lo, hi.hi, hi.lo);
                ff_dot_acc(is, ic, ur.hi, ur.lo, hi.hi, hi.lo);
                ff_dot_acc(is, ic, ui.hi, ui.lo, hr.hi, hr.lo);
            }
            w[6 * sp + 2 * a] = ff_fast_two_sum(rs, rc);
            w[6 * sp + 2 * a + 1] = ff_fast_two_sum(is, ic);
        }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ ff warp_sum(ff v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += shfl_down(v, off, 32);
    return v;
}

// Deterministic block sum (fixed tree for a fixed blockDim); result valid in thread 0.
// The per-thread values and the sum over a warp are taken in the kernel's arithmetic type
// R (FP32 in the mixed-precision kernels: GB300's FP64 rate is a small fraction of its
// FP32 rate), the sums across warps, blocks and the grid in FP64.
template <class R>
__device__ __forceinline__ double block_sum(R v, double* sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sm[wid] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < nw ? sm[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

__device__ __forceinline__ void finalize_scalar(SysState* st, double total, int fin) {
    if (fin == FIN_STORE) {
        st->sum = total;
    } else if (fin == FIN_ALPHA) {
        st->pAp = total;
        if (!(total > 0.0) || !isfinite(total)) {
            st->status = kBreakdown;
        } else {
            st->alpha = st->rr / total;
        }
    } else {  // FIN_BETA
        const double rr_new = total;
        st->rr_new = rr_new;
        st->iter += 1;
        if (!isfinite(rr_new)) {
            st->status = kBreakdown;
        } else if (rr_new <= st->stop_in || st->iter >= st->max_iter ||
                   (st->reliable && sqrt(rr_new) < st->delta * st->r_max)) {
            // park the system: the host recomputes the true residual in FP64 (and, in mixed
            // precision, folds the inner solution into the FP64 one) before it continues
            st->status = kNeedUpdate;
        } else {
            st->beta = rr_new / st->rr;
            st->rr = rr_new;
            st->r_max = fmax(st->r_max, sqrt(rr_new));
        }
    }
}

// Block-level reduction of `v` for system `sys`; the last block to arrive sums the
// partials in index order and finalizes.
// Per-block sum of v (the kernel's arithmetic type within a warp, FP64 across warps), written to
// the system's partial of this block; the last block to finish (counted atomically) sums the
// partials in index order and finalizes the scalar.  One block barrier: after it the other warps
// leave and warp 0 alone writes the partial and, in the last block, sums all partials.  The sum
// order is fixed whatever block finishes last, so results are deterministic.  Must be the
// kernel's last statement (warps other than 0 return here).
// System sys's partials start at sys * part_stride (part_stride >= every grid's block count, the same
// for every launch of a batch, so that launches of different block counts for different systems can
// run concurrently); part_stride 0 means gridDim.x.
template <class R>
__device__ __forceinline__ void reduce_and_finalize(R v, double* partials, unsigned* counters, SysState* st,
                                                    int sys, int fin, int part_stride) {
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) sm[wid] = (double)v;
    __syncthreads();
    if (wid != 0) return;
    double bs = lane < nw ? sm[lane] : 0.0;
    bs = warp_sum(bs);
    const int nb = gridDim.x;
    double* part = partials + (size_t)sys * (size_t)(part_stride > 0 ? part_stride : nb);
    unsigned prev = 0;
    if (lane == 0) {
        part[blockIdx.x] = bs;
        __threadfence();
        prev = atomicAdd(counters + sys, 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != (unsigned)(nb - 1)) return;
    __threadfence();
    double t = 0.0;
    for (int i = lane; i < nb; i += 32) t += *((volatile double*)(part + i));
    t = warp_sum(t);
    if (lane == 0) {
        finalize_scalar(st + sys, t, fin);
        counters[sys] = 0u;
    }
}

// ---------------------------------------------------------------- the fused hopping kernel
// The body of the generic hop (one thread per 5D site); hop_kernel below launches it at 256
// threads per block, other instances (float-float) at their own bounds.
template <class SPin, class SPz, class SPout, class SPacc, class LK, class R, int F>
__device__ __forceinline__ void hop_body(const HopParams<R>& P) {
    constexpr bool DAG = (F & F_DAG) != 0;
    constexpr int ZOP = (F & F_ZOP_MASK) >> F_ZOP_SHIFT;
    constexpr int HOPOP = (F & F_HOP_MASK) >> F_HOP_SHIFT;
    constexpr bool NEG = (F & F_NEG) != 0;
    constexpr int POST = (F & F_POST_MASK) >> F_POST_SHIFT;
    constexpr bool NORM = (F & F_NORM) != 0;
    constexpr bool CG = (F & F_CG) != 0;
    constexpr bool RESID = (F & F_RESID) != 0;
    constexpr int FIN = (F & F_FIN_MASK) >> F_FIN_SHIFT;
    constexpr bool REDUCE = NORM || CG || RESID;

    const int sys = blockIdx.y + P.sys_base;
    if (P.gate && P.st[sys].status != P.need_status) return;  // uniform over the block
    if (P.prof_count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(P.prof_count, 1ull);

    const int ns = P.ns;
    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = (int)(gi & (size_t)(ns - 1));
    const size_t hh = gi >> P.lg_ns;
    const bool valid = hh < (size_t)P.g.Vh;
    const int h = valid ? (int)hh : 0;
    const R r = (R)P.r_sys[sys];

    int c[4];
    site_coords(P.g, P.p_out, h, c);
    const int p_in = 1 - P.p_out;

    const void* in = P.in.d(sys);
    const float* in_n = P.in.n(sys);

    R acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;

#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            int cn[4] = {c[0], c[1], c[2], c[3]};
            const int Lm = P.g.L[mu];
            cn[mu] = dir == 0 ? (c[mu] + 1 == Lm ? 0 : c[mu] + 1) : (c[mu] == 0 ? Lm - 1 : c[mu] - 1);
            const int hn = checked_index(half_index(P.g, cn), P.g.Vh, P.bounds_flag, kBoundsNeighbour);
            bool flip = false;
            if (mu == 3 && P.g.tbc) flip = dir == 0 ? (c[3] == Lm - 1) : (c[3] == 0);

            R v[24];
            if (valid) {
                SpinorIO<SPin, R>::load(in, in_n, (size_t)hn, s, ns, v);
            } else {
#pragma unroll
                for (int k = 0; k < 24; ++k) v[k] = 0;
            }
            if (!DAG && !P.preshifted) bidiag_apply(v, P.cf.rho[s], P.cf.sigma[s], r, s, ns, false);  // chi = B psi

            // forward hop uses (1 - gamma) for D and (1 + gamma) for D^dag; backward the opposite
            const R sg = DAG ? (dir == 0 ? (R)1 : (R)-1) : (dir == 0 ? (R)-1 : (R)1);
            R hp[12];
            project(mu, sg, v, hp);
            if (flip) {
#pragma unroll
                for (int k = 0; k < 12; ++k) hp[k] = -hp[k];
            }
            R u[18];
            const size_t lidx = dir == 0 ? ((size_t)(P.p_out * 4 + mu) * P.g.Vh + h)
                                         : ((size_t)(p_in * 4 + mu) * P.g.Vh + hn);
            LinkIO<LK, R>::load(P.links, lidx, u);
            R w[12];
            su3_mul(u, hp, w, dir == 1);
            accumulate(mu, sg, w, acc);
        }
    }

    if (DAG) bidiag_apply(acc, P.cf.rho[s], P.cf.sigma[s], r, s, ns, true);  // B^dag y
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] *= (R)-0.5;  // H psi  (or H^dag psi)
    if (HOPOP == OP_MINV) minv_apply(acc, P.cf, r, s, ns, false);
    if (HOPOP == OP_MINVDAG) minv_apply(acc, P.cf, r, s, ns, true);

    R res[24];
    if (ZOP != ZOP_NONE) {
        R zz[24];
        if (valid) {
            SpinorIO<SPz, R>::load(P.z.d(sys), P.z.n(sys), (size_t)h, s, ns, zz);
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) zz[k] = 0;
        }
        if (ZOP == ZOP_M) bidiag_apply(zz, P.cf.d[s], P.cf.e[s], r, s, ns, false);
        if (ZOP == ZOP_MDAG) bidiag_apply(zz, P.cf.d[s], P.cf.e[s], r, s, ns, true);
#pragma unroll
        for (int k = 0; k < 24; ++k) res[k] = NEG ? zz[k] - acc[k] : zz[k] + acc[k];
    } else {
#pragma unroll
        for (int k = 0; k < 24; ++k) res[k] = NEG ? -acc[k] : acc[k];
    }

    R nrm = R(0);  // per-thread partial sum in the arithmetic type (see block_sum)
    if (NORM && valid) {
#pragma unroll
        for (int k = 0; k < 24; ++k) nrm += res[k] * res[k];
    }
    if (POST == OP_MINV) minv_apply(res, P.cf, r, s, ns, false);
    if (POST == OP_MINVDAG) minv_apply(res, P.cf, r, s, ns, true);

    if (CG) {
        // res = A p;  r <- r - alpha A p;  x <- x + alpha p;  nrm = |r|^2
        const R alpha = (R)P.st[sys].alpha;
        if (valid) {
            R rv[24], xv[24], pv[24];
            SpinorIO<SPacc, R>::load(P.cg_r.d(sys), P.cg_r.n(sys), (size_t)h, s, ns, rv);
            SpinorIO<SPacc, R>::load(P.cg_x.d(sys), P.cg_x.n(sys), (size_t)h, s, ns, xv);
            SpinorIO<SPin, R>::load(P.cg_p.d(sys), P.cg_p.n(sys), (size_t)h, s, ns, pv);
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                rv[k] -= alpha * res[k];
                xv[k] += alpha * pv[k];
                nrm += rv[k] * rv[k];
            }
            SpinorIO<SPacc, R>::store(P.cg_r.d(sys), P.cg_r.n(sys), (size_t)h, s, ns, rv);
            SpinorIO<SPacc, R>::store(P.cg_x.d(sys), P.cg_x.n(sys), (size_t)h, s, ns, xv);
        }
    } else if (RESID) {
        if (valid) {
            R bv[24];
            SpinorIO<SPacc, R>::load(P.b.d(sys), P.b.n(sys), (size_t)h, s, ns, bv);
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                res[k] = bv[k] - res[k];
                nrm += res[k] * res[k];
            }
            SpinorIO<SPout, R>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s, ns, res);
        }
    } else {
        if (valid) SpinorIO<SPout, R>::store(P.out.d(sys), P.out.n(sys), (size_t)h, s, ns, res);
    }

    if (REDUCE) reduce_and_finalize(nrm, P.partials, P.counters, P.st, sys, FIN, P.part_stride);
}

template <class SPin, class SPz, class SPout, class SPacc, class LK, class R, int F>
__global__ void __launch_bounds__(256) hop_kernel(const HopParams<R> P) {
    hop_body<SPin, SPz, SPout, SPacc, LK, R, F>(P);
}

// ---------------------------------------------------------------- site-local kernels
// out = op(in) with op in {M, M^dag, M^-1, M^-dag, B} on n_sites * Ns 5D sites (lane groups of Ns)
template <class SPin, class SPout, class R>
__global__ void __launch_bounds__(256) m5_kernel(FieldRef in, FieldRef out, size_t n_sites, int ns, int lg_ns,
                                                 const double* r_sys, int sys_base, int op, Coef5<R> cf,
                                                 const SysState* gate_st, int need) {
    const int sys = blockIdx.y + sys_base;
    if (gate_st && gate_st[sys].status != need) return;  // optional: only systems with this status
    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = (int)(gi & (size_t)(ns - 1));
    const size_t h = gi >> lg_ns;
    const bool valid = h < n_sites;
    const R r = (R)r_sys[sys];
    R v[24];
    if (valid) {
        SpinorIO<SPin, R>::load(in.d(sys), in.n(sys), h, s, ns, v);
    } else {
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = 0;
    }
    if (op == 0) bidiag_apply(v, cf.d[s], cf.e[s], r, s, ns, false);
    else if (op == 1) bidiag_apply(v, cf.d[s], cf.e[s], r, s, ns, true);
    else if (op == 2) minv_apply(v, cf, r, s, ns, false);
    else if (op == 3) minv_apply(v, cf, r, s, ns, true);
    else bidiag_apply(v, cf.rho[s], cf.sigma[s], r, s, ns, false);  // op 4: chi = B psi (internal)
    if (valid) SpinorIO<SPout, R>::store(out.d(sys), out.n(sys), h, s, ns, v);
}

// ---------------------------------------------------------------- layout conversion
// External complex128 field <-> internal half field of parity p.
//   ext_mode 0 (FULL):       ext[s][lex][12 complex], lex of site (p, h)
//   ext_mode 1 (HALF):       ext[s][h][12 complex]   (SCHUR_EVEN layout when p = 0)
template <class SP>
__global__ void __launch_bounds__(256) pack_kernel(const double2* __restrict__ ext, FieldRef out, Geom g, int p,
                                                   int ns, int lg_ns, int ext_mode) {
    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = (int)(gi & (size_t)(ns - 1));
    const size_t h = gi >> lg_ns;
    if (h >= (size_t)g.Vh) return;
    size_t site;
    if (ext_mode == 0) {
        int c[4];
        site_coords(g, p, (int)h, c);
        site = (size_t)c[0] + (size_t)g.L[0] * (c[1] + (size_t)g.L[1] * (c[2] + (size_t)g.L[2] * c[3]));
    } else {
        site = h;
    }
    const size_t nsite = ext_mode == 0 ? 2 * (size_t)g.Vh : (size_t)g.Vh;
    const double2* src = ext + ((size_t)s * nsite + site) * 12;
    double v[24];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 q = src[k];
        v[2 * k] = q.x;
        v[2 * k + 1] = q.y;
    }
    SpinorIO<SP, double>::store(out.d(0), out.n(0), h, s, ns, v);
}

template <class SP>
__global__ void __launch_bounds__(256) unpack_kernel(FieldRef in, double2* __restrict__ ext, Geom g, int p, int ns,
                                                     int lg_ns, int ext_mode) {
    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = (int)(gi & (size_t)(ns - 1));
    const size_t h = gi >> lg_ns;
    if (h >= (size_t)g.Vh) return;
    size_t site;
    if (ext_mode == 0) {
        int c[4];
        site_coords(g, p, (int)h, c);
        site = (size_t)c[0] + (size_t)g.L[0] * (c[1] + (size_t)g.L[1] * (c[2] + (size_t)g.L[2] * c[3]));
    } else {
        site = h;
    }
    const size_t nsite = ext_mode == 0 ? 2 * (size_t)g.Vh : (size_t)g.Vh;
    double v[24];
    SpinorIO<SP, double>::load(in.d(0), in.n(0), h, s, ns, v);
    double2* dst = ext + ((size_t)s * nsite + site) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = make_double2(v[2 * k], v[2 * k + 1]);
}

// ---------------------------------------------------------------- vector kernels
// Generic per-system vector update on half fields (5D site per thread, no lane coupling):
//   kind 0: y = x                          (convert)
//   kind 1: p = r + beta p                 (beta from state; runs when status == need)
//   kind 2: X += x ; x = 0                 (fold the inner solution into the FP64 one)
//   kind 3: |x|^2 -> reduction (FIN_STORE into state.sum)
//   kind 4: y = a x + y  (a = coef)
//   kind 5: y = 0
//   kind 6: y = x / rscale                  (true residual -> inner units)
//   kind 7: X += rscale x ; x = 0           (fold the inner solution, inner -> true units)
template <class SPx, class SPy, class R>
__global__ void __launch_bounds__(256) vec_kernel(FieldRef x, FieldRef y, size_t n5, int ns, int kind, double coef,
                                                  SysState* st, int gate, int need, double* partials,
                                                  unsigned* counters, int part_stride, int sys_base,
                                                  unsigned long long* prof_count) {
    const int sys = blockIdx.y + sys_base;
    if (gate && st[sys].status != need) return;
    if (prof_count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof_count, 1ull);
    const size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gi < n5;
    const size_t h = valid ? gi / ns : 0;
    const int s = (int)(gi % ns);
    double nrm = 0.0;
    if (valid) {
        R a[24], b[24];
        if (kind != 5) SpinorIO<SPx, R>::load(x.d(sys), x.n(sys), h, s, ns, a);
        switch (kind) {
            case 0:
                SpinorIO<SPy, R>::store(y.d(sys), y.n(sys), h, s, ns, a);
                break;
            case 1: {
                const R beta = (R)st[sys].beta;
                SpinorIO<SPy, R>::load(y.d(sys), y.n(sys), h, s, ns, b);
#pragma unroll
                for (int k = 0; k < 24; ++k) b[k] = a[k] + beta * b[k];
                SpinorIO<SPy, R>::store(y.d(sys), y.n(sys), h, s, ns, b);
                break;
            }
            case 2: {
                SpinorIO<SPy, R>::load(y.d(sys), y.n(sys), h, s, ns, b);
#pragma unroll
                for (int k = 0; k < 24; ++k) { b[k] += a[k]; a[k] = 0; }
                SpinorIO<SPy, R>::store(y.d(sys), y.n(sys), h, s, ns, b);
                SpinorIO<SPx, R>::store(x.d(sys), x.n(sys), h, s, ns, a);
                break;
            }
            case 3:
#pragma unroll
                for (int k = 0; k < 24; ++k) nrm += (double)a[k] * (double)a[k];
                break;
            case 6: {
                const R inv = (R)(1.0 / st[sys].rscale);
#pragma unroll
                for (int k = 0; k < 24; ++k) a[k] *= inv;
                SpinorIO<SPy, R>::store(y.d(sys), y.n(sys), h, s, ns, a);
                break;
            }
            case 7: {
                const R sc = (R)st[sys].rscale;
                SpinorIO<SPy, R>::load(y.d(sys), y.n(sys), h, s, ns, b);
#pragma unroll
                for (int k = 0; k < 24; ++k) { b[k] += sc * a[k]; a[k] = 0; }
                SpinorIO<SPy, R>::store(y.d(sys), y.n(sys), h, s, ns, b);
                SpinorIO<SPx, R>::store(x.d(sys), x.n(sys), h, s, ns, a);
                break;
            }
            case 4: {
                SpinorIO<SPy, R>::load(y.d(sys), y.n(sys), h, s, ns, b);
#pragma unroll
                for (int k = 0; k < 24; ++k) b[k] += (R)coef * a[k];
                SpinorIO<SPy, R>::store(y.d(sys), y.n(sys), h, s, ns, b);
                break;
            }
            default: {
#pragma unroll
                for (int k = 0; k < 24; ++k) b[k] = 0;
                SpinorIO<SPy, R>::store(y.d(sys), y.n(sys), h, s, ns, b);
                break;
            }
        }
    }
    if (kind == 3) reduce_and_finalize<double>(nrm, partials, counters, st, sys, FIN_STORE, part_stride);
}

}  // namespace odwf
