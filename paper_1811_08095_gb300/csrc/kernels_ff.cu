// Float-float instances of the generic hopping and site-local kernels (kernels.cuh): the
// reliable-update residual b - S^dag S x of the mixed-precision CG in about 48-bit arithmetic
// built from FP32 operations (ff.cuh), with float-float fields and links.
#include "kernels.cuh"
#include "kernels.h"

namespace odwf {

namespace {
constexpr int kBS = 256;

template <int F>
cudaError_t hopff(const HopParams<ff>& P, int nsys, cudaStream_t st) {
    const size_t n = (size_t)P.g.Vh * P.ns;
    dim3 grid(blocks_for(n, kBS), nsys);
    note_launch();
    hop_kernel<SpFF, SpFF, SpFF, SpFF, LinkFF18, ff, F><<<grid, kBS, 0, st>>>(P);
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
