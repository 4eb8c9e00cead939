// Wilson gauge action and force, and the molecular-dynamics updates of the HMC (Sec. 2: the
// Wilson plaquette gauge action at beta = 6/g0^2, the Omelyan integrator), in FP64 on the
// external gauge layout U[mu][t][z][y][x][a][b] (complex128) and momenta of the same shape.
//
//   gauge force   Pi_mu(x) = -(beta/3) ta(U_mu(x) Sigma_mu(x)), Sigma the sum of the six staples,
//                 so that dS_g/deps = tr(T Pi) for U_mu(x) -> exp(eps T) U_mu(x);
//   gauge action  S_g = beta sum_p (1 - Re tr P / 3) = beta (6 V - sum_links Re tr(U Sigma) / 12)
//                 (every plaquette has four links);
//   link update   U <- exp(a P) U, the exponential by Cayley-Hamilton (X^3 = s X + d 1 for
//                 traceless anti-Hermitian X) summed on the scalars to the last bit;
//   momentum update P <- P + c F.
#include "kernels.cuh"
#include "kernels.h"

namespace odwf {

namespace {
constexpr int kBSM = 128;

struct Z3 {
    double2 m[9];
};

__device__ __forceinline__ double2 zm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zmc(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a conj(b)
__device__ __forceinline__ double2 za(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ Z3 ld(const double2* __restrict__ U, size_t V, int mu, size_t s) {
    Z3 u;
    const double2* p = U + ((size_t)mu * V + s) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) u.m[k] = p[k];
    return u;
}
__device__ __forceinline__ Z3 mm(const Z3& a, const Z3& b) {  // a b
    Z3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.m[3 * i + j] = za(za(zm(a.m[3 * i], b.m[j]), zm(a.m[3 * i + 1], b.m[3 + j])), zm(a.m[3 * i + 2], b.m[6 + j]));
    return c;
}
__device__ __forceinline__ Z3 mmd(const Z3& a, const Z3& b) {  // a b^+
    Z3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.m[3 * i + j] =
                za(za(zmc(a.m[3 * i], b.m[3 * j]), zmc(a.m[3 * i + 1], b.m[3 * j + 1])), zmc(a.m[3 * i + 2], b.m[3 * j + 2]));
    return c;
}
__device__ __forceinline__ Z3 mdm(const Z3& a, const Z3& b) {  // a^+ b
    Z3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double2 s = make_double2(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) s = za(s, zm(make_double2(a.m[3 * k + i].x, -a.m[3 * k + i].y), b.m[3 * k + j]));
            c.m[3 * i + j] = s;
        }
    return c;
}

struct Lex {
    int L[4];
    size_t stride[4];
    size_t V;
};

__device__ __forceinline__ size_t shift(const Lex& g, const int c[4], size_t s, int mu, int dir) {
    const int x = c[mu];
    if (dir > 0) return x + 1 == g.L[mu] ? s - (size_t)(g.L[mu] - 1) * g.stride[mu] : s + g.stride[mu];
    return x == 0 ? s + (size_t)(g.L[mu] - 1) * g.stride[mu] : s - g.stride[mu];
}

// one thread per link (mu, s): Pi (optional) and per-block sums of Re tr(U Sigma)
__global__ void __launch_bounds__(kBSM) gauge_force_kernel(Lex g, const double2* __restrict__ U, double beta,
                                                           double2* __restrict__ F, double* __restrict__ part) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double retr = 0.0;
    if (i < 4 * g.V) {
        const int mu = (int)(i / g.V);
        const size_t s = i - (size_t)mu * g.V;
        int c[4];
        size_t r = s;
        for (int d = 0; d < 4; ++d) {
            c[d] = (int)(r % g.L[d]);
            r /= g.L[d];
        }
        Z3 S;
#pragma unroll
        for (int k = 0; k < 9; ++k) S.m[k] = make_double2(0.0, 0.0);
        const size_t xm = shift(g, c, s, mu, +1);
#pragma unroll 1
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            const size_t xn = shift(g, c, s, nu, +1), xb = shift(g, c, s, nu, -1);
            int cb[4] = {c[0], c[1], c[2], c[3]};
            cb[nu] = c[nu] == 0 ? g.L[nu] - 1 : c[nu] - 1;
            const size_t xmb = shift(g, cb, xb, mu, +1);  // x + mu - nu
            // upper: U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
            const Z3 up = mmd(mmd(ld(U, g.V, nu, xm), ld(U, g.V, mu, xn)), ld(U, g.V, nu, s));
            // lower: U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
            const Z3 lo = mdm(mm(ld(U, g.V, mu, xb), ld(U, g.V, nu, xmb)), ld(U, g.V, nu, xb));
#pragma unroll
            for (int k = 0; k < 9; ++k) S.m[k] = za(S.m[k], za(up.m[k], lo.m[k]));
        }
        const Z3 O = mm(ld(U, g.V, mu, s), S);
        retr = O.m[0].x + O.m[4].x + O.m[8].x;
        if (F) {
            // Pi = -(beta/3) ta(O)
            const double f = -beta / 3.0;
            double2 A[9];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const double2 x = O.m[3 * a + b], y = O.m[3 * b + a];
                    A[3 * a + b] = make_double2(0.5 * (x.x - y.x), 0.5 * (x.y + y.y));
                }
            const double im3 = (A[0].y + A[4].y + A[8].y) / 3.0;
            A[0].y -= im3;
            A[4].y -= im3;
            A[8].y -= im3;
            double2* o = F + ((size_t)mu * g.V + s) * 9;
#pragma unroll
            for (int k = 0; k < 9; ++k) o[k] = make_double2(f * A[k].x, f * A[k].y);
        }
    }
    __shared__ double sm[kBSM / 32];
    retr = warp_sum(retr);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = retr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kBSM / 32; ++k) t += sm[k];
        part[blockIdx.x] = t;
    }
}

// U <- exp(a P) U per link, exp by the Cayley-Hamilton series on the scalars
__global__ void __launch_bounds__(kBSM) link_update_kernel(size_t nlinks, double2* __restrict__ U,
                                                           const double2* __restrict__ P, double a) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nlinks) return;
    Z3 X;
#pragma unroll
    for (int k = 0; k < 9; ++k) X.m[k] = make_double2(a * P[i * 9 + k].x, a * P[i * 9 + k].y);
    const Z3 X2 = mm(X, X);
    const double s = 0.5 * (X2.m[0].x + X2.m[4].x + X2.m[8].x);
    double dim = 0.0;  // d = tr(X X^2) / 3 is i dim
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) dim += zm(X.m[3 * r + k], X2.m[3 * k + r]).y;
    dim /= 3.0;
    const double nrm = sqrt(fmax(-2.0 * s, 0.0));
    double2 ca = make_double2(0.0, 0.0), cb = make_double2(0.0, 0.0), cc = make_double2(1.0, 0.0);  // state of n = 2
    double2 f0 = make_double2(1.0, 0.0), f1 = make_double2(1.0, 0.0), f2 = make_double2(0.5, 0.0);
    double inv = 0.5, bound = 0.5 * nrm * nrm;
    for (int n = 3; n < 100; ++n) {
        const double2 na = make_double2(-cc.y * dim, cc.x * dim);
        const double2 nb = make_double2(cc.x * s + ca.x, cc.y * s + ca.y);
        ca = na;
        cc = cb;
        cb = nb;
        inv /= (double)n;
        f0 = make_double2(f0.x + ca.x * inv, f0.y + ca.y * inv);
        f1 = make_double2(f1.x + cb.x * inv, f1.y + cb.y * inv);
        f2 = make_double2(f2.x + cc.x * inv, f2.y + cc.y * inv);
        bound *= nrm / (double)n;
        if (bound < 1e-18 * fmax(nrm, 1e-300) || bound == 0.0) break;
    }
    Z3 E;
#pragma unroll
    for (int k = 0; k < 9; ++k) E.m[k] = za(zm(f1, X.m[k]), zm(f2, X2.m[k]));
    E.m[0] = za(E.m[0], f0);
    E.m[4] = za(E.m[4], f0);
    E.m[8] = za(E.m[8], f0);
    Z3 W;
#pragma unroll
    for (int k = 0; k < 9; ++k) W.m[k] = U[i * 9 + k];
    const Z3 R = mm(E, W);
#pragma unroll
    for (int k = 0; k < 9; ++k) U[i * 9 + k] = R.m[k];
}

__global__ void axpy_kernel(size_t n, double2* __restrict__ y, const double2* __restrict__ x, double c) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = make_double2(y[i].x + c * x[i].x, y[i].y + c * x[i].y);
}
}  // namespace

size_t gauge_force_blocks(size_t V) { return (4 * V + kBSM - 1) / kBSM; }

cudaError_t launch_gauge_force(const int dims[4], const double2* U, double beta, double2* F, double* partials,
                               double* retr_sum, cudaStream_t st) {
    Lex g;
    size_t stride = 1;
    for (int d = 0; d < 4; ++d) {
        g.L[d] = dims[d];
        g.stride[d] = stride;
        stride *= (size_t)dims[d];
    }
    g.V = stride;
    const size_t nb = gauge_force_blocks(g.V);
    note_launch();
    gauge_force_kernel<<<(unsigned)nb, kBSM, 0, st>>>(g, U, beta, F, partials);
    return launch_sum_partials(partials, (int)nb, retr_sum, st);
}

cudaError_t launch_link_update(size_t nlinks, double2* U, const double2* P, double a, cudaStream_t st) {
    note_launch();
    link_update_kernel<<<(unsigned)((nlinks + kBSM - 1) / kBSM), kBSM, 0, st>>>(nlinks, U, P, a);
    return cudaGetLastError();
}

cudaError_t launch_axpy(size_t n, double2* y, const double2* x, double c, cudaStream_t st) {
    note_launch();
    axpy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, y, x, c);
    return cudaGetLastError();
}

}  // namespace odwf
