// Gradient flow (Sec. 2) and flow observables (Sec. 3): device-side types and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace odwf {
namespace flow {

// Lattice geometry of the flow kernels: extents, lexicographic strides and the height bt of the
// time slabs the sites are visited in (bt divides Lt).
struct FlowGeom {
    int L[4];
    size_t stride[4];
    size_t V;
    int bt;
};

// One measurement, written on the device by the reduction kernel (layout of odwf_flow_obs).
struct FlowObsDev {
    double t, e_plaq, e_clover, q_clover, plaq_min, plaq_mean;
};

size_t plaq_blocks(const FlowGeom& g);    // blocks of the plaquette kernel (its partial sums)
size_t update_blocks(const FlowGeom& g);  // blocks of the update kernel
size_t clover_blocks(const FlowGeom& g);  // blocks of the clover kernel (its partial sums)
cudaError_t launch_plaq(const FlowGeom& g, const float4* hi, float4* A, double* part_retr, float* part_min, bool measure,
                        cudaStream_t st);
cudaError_t launch_update(const FlowGeom& g, int stage, const float4* hi, const float4* lo, float4* hi_out,
                          float4* lo_out, const float4* A, float4* K, float eps, cudaStream_t st);
cudaError_t launch_clover(const FlowGeom& g, const float4* hi, const float4* A, double* part_e, double* part_q,
                          float* e_site, float* q_site, cudaStream_t st);
cudaError_t launch_reduce(const FlowGeom& g, const double* part_retr, const float* part_min, const double* part_e,
                          const double* part_q, double t, FlowObsDev* out, cudaStream_t st);
cudaError_t launch_split(const double2* U, float4* hi, float4* lo, size_t V, int mu, cudaStream_t st);
cudaError_t launch_join(const float4* hi, const float4* lo, double2* U, size_t V, int mu, cudaStream_t st);

}  // namespace flow
}  // namespace odwf
