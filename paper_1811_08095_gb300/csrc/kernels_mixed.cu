// Mixed-precision kernels: FP32 arithmetic on FP16 / BF16 / FP32 operator fields with
// FP32 links (12 or 18 reals) and FP32 CG accumulators.
#include "kernels.cuh"
#include "kernels.h"

namespace odwf {

namespace {
constexpr int kBS = 256;

template <class SP, class LK, int F>
cudaError_t hopm(const HopParams<float>& P, int nsys, cudaStream_t st) {
    const size_t n = (size_t)P.g.Vh * P.ns;
    dim3 grid(blocks_for(n, kBS), nsys);
    note_launch(); hop_kernel<SP, SP, SP, SpF32, LK, float, F><<<grid, kBS, 0, st>>>(P);
    return cudaGetLastError();
}

template <class SP, class LK>
cudaError_t hopm_e(const HopParams<float>& P, Epi e, int nsys, cudaStream_t st) {
    switch (e) {
        case Epi::MINV: return hopm<SP, LK, EPI_MINV>(P, nsys, st);
        case Epi::SCHUR_NORM_MDINV: return hopm<SP, LK, EPI_SCHUR_NORM_MDINV>(P, nsys, st);
        case Epi::SCHUR_MDINV: return hopm<SP, LK, EPI_SCHUR_NORM_MDINV_STORE>(P, nsys, st);
        case Epi::D_MINVDAG: return hopm<SP, LK, EPID_MINVDAG>(P, nsys, st);
        case Epi::D_NORMAL: return hopm<SP, LK, EPID_NORMAL>(P, nsys, st);
        case Epi::D_NORMAL_CG: return hopm<SP, LK, EPID_NORMAL_CG>(P, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

template <class SP>
cudaError_t hopm_l(const HopParams<float>& P, Epi e, Lk lk, int nsys, cudaStream_t st) {
    switch (lk) {
        case Lk::F12: return hopm_e<SP, LinkF12>(P, e, nsys, st);
        case Lk::F18: return hopm_e<SP, LinkF18>(P, e, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_hop_mixed(const HopParams<float>& P, Epi e, Sp low, Lk lk, int nsys, cudaStream_t st) {
    switch (low) {
        case Sp::F32: return hopm_l<SpF32>(P, e, lk, nsys, st);
        case Sp::F16: return hopm_l<SpF16>(P, e, lk, nsys, st);
        case Sp::BF16: return hopm_l<SpBF16>(P, e, lk, nsys, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_m5_mixed(Sp low, const FieldRef& in, const FieldRef& out, size_t n_sites, int ns,
                            const double* r_sys, int sys_base, int nsys, int op, const Coef5<float>& cf,
                            cudaStream_t st) {
    dim3 grid(blocks_for(n_sites * ns, kBS), nsys);
    const int lg = lg2(ns);
    switch (low) {
        case Sp::F32: note_launch(); m5_kernel<SpF32, SpF32, float><<<grid, kBS, 0, st>>>(in, out, n_sites, ns, lg, r_sys, sys_base, op, cf, nullptr, 0); break;
        case Sp::F16: note_launch(); m5_kernel<SpF16, SpF16, float><<<grid, kBS, 0, st>>>(in, out, n_sites, ns, lg, r_sys, sys_base, op, cf, nullptr, 0); break;
        case Sp::BF16: note_launch(); m5_kernel<SpBF16, SpBF16, float><<<grid, kBS, 0, st>>>(in, out, n_sites, ns, lg, r_sys, sys_base, op, cf, nullptr, 0); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace odwf
