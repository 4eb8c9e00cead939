// Float-float instances of the generic hopping and site-local kernels (kernels.cuh): the
// reliable-update residual b - S^dag S x of the mixed-precision CG in about 48-bit arithmetic
// built from FP32 operations (ff.cuh), with float-float fields and links.
#include "kernels.cuh"
#include "kernels.h"

namespace odwf {

namespace {
constexpr int kBS = 256;
// The float-float hops hold a float-float spinor accumulator, neighbour and link: at 256 threads
// per block they took ~250 registers and one block per SM (8 warps); at 128 threads and three
// blocks per SM (168 registers, 12 warps) they run 1.4x faster on 16^3x32x16 (K1 1.46 -> 1.03 ms).
constexpr int kBSH = 128;
constexpr int kMinBlocksFF = 3;
static_assert(kBSH >= kMinReduceBlock && kBSH % 32 == 0, "the reducing hops need blocks the partials fit");

template <int F>
__global__ void __launch_bounds__(kBSH, kMinBlocksFF) hop_ff_kernel(const HopParams<ff> P) {
    hop_body<SpFF, SpFF, SpFF, SpFF, LinkFF18, ff, F>(P);
}

template <int F>
cudaError_t hopff(const HopParams<ff>& P, int nsys, cudaStream_t st) {
    const size_t n = (size_t)P.g.Vh * P.ns;
    dim3 grid(blocks_for(n, kBSH), nsys);
    note_launch();
    hop_ff_kernel<F><<<grid, kBSH, 0, st>>>(P);
    return cudaGetLastError();
}

__global__ void links_ff18_kernel(const double* __restrict__ d18, float2* __restrict__ out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ff v(d18[i]);
    out[i] = make_float2(v.hi, v.lo);
}
}  // namespace

cudaError_t launch_hop_ff(const HopParams<ff>& P, Epi e, int nsys, cudaStream_t st) {
    switch (e) {
        case Epi::MINV: return hopff<EPI_MINV>(P, nsys, st);
        case Epi::SCHUR_MDINV: return hopff<EPI_SCHUR_NORM_MDINV_STORE>(P, nsys, st);
        case Epi::D_MINVDAG: return hopff<EPID_MINVDAG>(P, nsys, st);
        case Epi::D_NORMAL: return hopff<EPID_NORMAL>(P, nsys, st);
        case Epi::D_NORMAL_RESID: return hopff<EPID_NORMAL_RESID>(P, nsys, st);
        default: break;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_m5_ff(const FieldRef& in, const FieldRef& out, size_t n_sites, int ns, const double* r_sys,
                         int sys_base, int nsys, int op, const Coef5<ff>& cf, cudaStream_t st) {
    dim3 grid(blocks_for(n_sites * ns, kBS), nsys);
    note_launch();
    m5_kernel<SpFF, SpFF, ff><<<grid, kBS, 0, st>>>(in, out, n_sites, ns, lg2(ns), r_sys, sys_base, op, cf, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_links_ff18_from_d18(const void* d18, void* ff18, size_t n_links, cudaStream_t st) {
    const size_t n = n_links * 18;
    note_launch();
    links_ff18_kernel<<<blocks_for(n, 256), 256, 0, st>>>((const double*)d18, (float2*)ff18, n);
    return cudaGetLastError();
}

}  // namespace odwf
