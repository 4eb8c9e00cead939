// Fermion-force contraction of the two-flavour pseudofermion action (Sec. 2, the HMC's two-flavour
// parts), the Wilson gauge force and action, and the molecular-dynamics updates, in FP64.
//
// For full-lattice 5D fields L and R, the derivative of <L, W R> along U_mu(x) -> exp(eps T) U_mu(x)
// (W the Wilson hopping matrix, T traceless anti-Hermitian) is tr(T G_mu(x)) with
//     G_mu(x) = U_mu(x) K1 - K2 U_mu(x)^+,
//     K1 = sum_{s,spin} R_s(x+mu) conj((1 - gamma_mu) L_s(x)),
//     K2 = sum_{s,spin} R_s(x) conj((1 + gamma_mu) L_s(x+mu))
// (colour outer products; the first index from R), and -G on t-links across an antiperiodic
// boundary.  The pseudofermion force is a sum of such terms with L and R built from the solution
// by the site-local and hopping operators (see pf_force.cpp); the contraction kernel takes L and
// R as parity-split FP64 half fields and accumulates coef * G per link.
//
// One thread per link; the loop over s reads, per s, the four spinors L(x), R(x+mu), R(x),
// L(x+mu) once, projects the L's with (1 -+ gamma_mu) and accumulates the two 3x3 outer products.
// The algorithmic bytes per link are 4 * Ns * 192 (the four spinors) + 144 (the link) + 2 * 144
// (G in and out): the kernel is bound by the FP64 pipe on this part (about 2 Ns * 180 FMAs).
#include "kernels.cuh"
#include "kernels.h"

namespace odwf {

namespace {
constexpr int kBSF = 128;

struct C3 {
    double2 m[9];
};

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zmulc(double2 a, double2 b) {  // a conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// K_{ba} += sum_spin r[spin][b] conj(w[spin][a])
__device__ __forceinline__ void outer_acc(const double r[24], const double w[24], C3& K) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double2 acc = K.m[3 * b + a];
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) {
                const double2 rv = make_double2(r[(sp * 3 + b) * 2], r[(sp * 3 + b) * 2 + 1]);
                const double2 wv = make_double2(w[(sp * 3 + a) * 2], w[(sp * 3 + a) * 2 + 1]);
                acc = zadd(acc, zmulc(rv, wv));
            }
            K.m[3 * b + a] = acc;
        }
}

// w = (1 + sg gamma_mu) v
__device__ __forceinline__ void proj_full(int mu, double sg, const double v[24], double w[24]) {
    double h[12];
    project(mu, sg, v, h);
#pragma unroll
    for (int k = 0; k < 24; ++k) w[k] = 0.0;
    accumulate(mu, sg, h, w);
}

__global__ void __launch_bounds__(kBSF) force_contract_kernel(Geom g, int ns, const void* __restrict__ links, FieldRef Le,
                                                              FieldRef Lo, FieldRef Re, FieldRef Ro, double coef,
                                                              double2* __restrict__ G, int accumulate_into) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // ((p * Vh + h) * 4 + mu)
    if (i >= (size_t)8 * g.Vh) return;
    const int mu = (int)(i & 3);
    const size_t ph = i >> 2;
    const int p = (int)(ph / g.Vh), h = (int)(ph % g.Vh);
    int c[4];
    site_coords(g, p, h, c);
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[mu] = c[mu] + 1 == g.L[mu] ? 0 : c[mu] + 1;
    const int hn = half_index(g, cn);
    const FieldRef& Lx = p == 0 ? Le : Lo;  // L at x
    const FieldRef& Ln = p == 0 ? Lo : Le;  // L at x + mu
    const FieldRef& Rx = p == 0 ? Re : Ro;
    const FieldRef& Rn = p == 0 ? Ro : Re;
    C3 K1, K2;
#pragma unroll
    for (int k = 0; k < 9; ++k) K1.m[k] = K2.m[k] = make_double2(0.0, 0.0);
    double v[24], w[24];
#pragma unroll 1
    for (int s = 0; s < ns; ++s) {
        SpinorIO<SpF64, double>::load(Lx.d(0), nullptr, (size_t)h, s, ns, v);
        proj_full(mu, -1.0, v, w);  // (1 - gamma_mu) L(x)
        SpinorIO<SpF64, double>::load(Rn.d(0), nullptr, (size_t)hn, s, ns, v);
        outer_acc(v, w, K1);
        SpinorIO<SpF64, double>::load(Ln.d(0), nullptr, (size_t)hn, s, ns, v);
        proj_full(mu, 1.0, v, w);  // (1 + gamma_mu) L(x + mu)
        SpinorIO<SpF64, double>::load(Rx.d(0), nullptr, (size_t)h, s, ns, v);
        outer_acc(v, w, K2);
    }
    double u[18];
    LinkIO<LinkD18, double>::load(links, (size_t)(p * 4 + mu) * g.Vh + h, u);
    double sgn = coef;
    if (mu == 3 && g.tbc && c[3] == g.L[3] - 1) sgn = -sgn;
    double2* Gl = G + ((size_t)(p * 4 + mu) * g.Vh + h) * 9;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double2 uak = make_double2(u[2 * (3 * a + k)], u[2 * (3 * a + k) + 1]);
                const double2 ubk = make_double2(u[2 * (3 * b + k)], u[2 * (3 * b + k) + 1]);
                acc = zadd(acc, zmul(uak, K1.m[3 * k + b]));    // (U K1)_{ab}
                const double2 t = zmulc(K2.m[3 * a + k], ubk);  // K2_{ak} conj(U_{bk}) = (K2 U^+)_{ab}
                acc = make_double2(acc.x - t.x, acc.y - t.y);
            }
            acc = make_double2(sgn * acc.x, sgn * acc.y);
            Gl[3 * a + b] = accumulate_into ? zadd(Gl[3 * a + b], acc) : acc;
        }
}

// Pi = ta(G) (traceless anti-Hermitian part) into the external gauge layout U[mu][t][z][y][x][a][b]
__global__ void force_finalize_kernel(Geom g, const double2* __restrict__ G, double2* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)8 * g.Vh) return;
    const int mu = (int)(i & 3);
    const size_t ph = i >> 2;
    const int p = (int)(ph / g.Vh), h = (int)(ph % g.Vh);
    int c[4];
    site_coords(g, p, h, c);
    const size_t V = (size_t)2 * g.Vh;
    const size_t lex = (size_t)c[0] + (size_t)g.L[0] * (c[1] + (size_t)g.L[1] * (c[2] + (size_t)g.L[2] * c[3]));
    const double2* Gl = G + ((size_t)(p * 4 + mu) * g.Vh + h) * 9;
    double2 A[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const double2 x = Gl[3 * a + b], y = Gl[3 * b + a];
            A[3 * a + b] = make_double2(0.5 * (x.x - y.x), 0.5 * (x.y + y.y));  // (G - G^+)/2
        }
    const double im3 = (A[0].y + A[4].y + A[8].y) / 3.0;
    A[0].y -= im3;
    A[4].y -= im3;
    A[8].y -= im3;
    double2* o = out + ((size_t)mu * V + lex) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) o[k] = A[k];
}

// sum of squares of n doubles: per-block partials, then one block in a fixed order
__global__ void __launch_bounds__(256) sumsq_kernel(const double* __restrict__ a, size_t n, double* __restrict__ part) {
    double t = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        t = fma(a[i], a[i], t);
    __shared__ double sm[32];
    t = warp_sum(t);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = t;
    __syncthreads();
    if (wid == 0) {
        double s = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) part[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) sum_partials_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
    double t = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) t += part[i];
    __shared__ double sm[32];
    t = warp_sum(t);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sm[k];
        *out = s;
    }
}
}  // namespace

constexpr int kSumsqBlocks = 608;  // 4 blocks per SM of a 152-SM part

cudaError_t launch_force_contract(const Geom& g, int ns, const void* links_d18, const FieldRef& Le, const FieldRef& Lo,
                                  const FieldRef& Re, const FieldRef& Ro, double coef, double2* G, bool accumulate_into,
                                  cudaStream_t st) {
    const size_t n = (size_t)8 * g.Vh;
    note_launch();
    force_contract_kernel<<<(unsigned)((n + kBSF - 1) / kBSF), kBSF, 0, st>>>(g, ns, links_d18, Le, Lo, Re, Ro, coef, G,
                                                                             accumulate_into ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_force_finalize(const Geom& g, const double2* G, double2* out_ext, cudaStream_t st) {
    const size_t n = (size_t)8 * g.Vh;
    note_launch();
    force_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, G, out_ext);
    return cudaGetLastError();
}

size_t sumsq_partials() { return kSumsqBlocks; }

cudaError_t launch_sum_partials(const double* partials, int nb, double* out, cudaStream_t st) {
    note_launch();
    sum_partials_kernel<<<1, 256, 0, st>>>(partials, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_sumsq(const double* a, size_t n, double* partials, double* out, cudaStream_t st) {
    note_launch();
    sumsq_kernel<<<kSumsqBlocks, 256, 0, st>>>(a, n, partials);
    note_launch();
    sum_partials_kernel<<<1, 256, 0, st>>>(partials, kSumsqBlocks, out);
    return cudaGetLastError();
}

}  // namespace odwf
