// Host-side launchers of the ODWF kernels (definitions in kernels_f64.cu, kernels_mixed.cu).
#pragma once

#include <cuda_runtime.h>

#include "odwf_internal.h"

namespace odwf {

// Reducing kernels write one partial per block and system; the buffer is sized for blocks of at
// least this many threads, each thread one 5D site (or more).
constexpr int kMinReduceBlock = 64;


enum class Sp { F64 = 0, F32 = 1, F16 = 2, BF16 = 3, FF = 4 };  // FF: float-float pairs (ff.cuh)
enum class Lk { D18 = 0, F18 = 1, F12 = 2, H12 = 3, FF18 = 4 };

struct FieldRef;
template <class R>
struct HopParams;

// Named epilogues (see kernels.cuh)
enum class Epi {
    MINV,                 // M^-1 H p
    SCHUR,                // z - M^-1 H t
    SCHUR_NORM_MDINV,     // M^-dag (z - M^-1 H t), |z - M^-1 H t|^2 -> alpha
    SCHUR_MDINV,          // M^-dag (z - M^-1 H t)
    FULL,                 // M z + H p
    PLAIN,                // H p
    ZMINUS_POSTMINV,      // M^-1 (z - H p)
    ZMINUS,               // z - H p
    D_MINVDAG,            // M^-dag H^dag a
    D_NORMAL,             // M^dag z - H^dag c
    D_NORMAL_CG,          // fused CG update (r, x, |r|^2 -> beta)
    D_NORMAL_RESID,       // b - (M^dag z - H^dag c), |.|^2 -> sum
    D_ZMINUS,             // z - H^dag c
    D_FULL,               // M^dag z + H^dag p
    D_PLAIN,              // H^dag p
    D_SCHUR2,             // z - M^-dag H^dag t
    D_ZMINUS_POSTMINVDAG, // M^-dag (z - H^dag p)
};

// FP64 path (double spinors, 18-real double links, FP64 arithmetic)
cudaError_t launch_hop_f64(const HopParams<double>& P, Epi e, int nsys, cudaStream_t st);
// Float-float path (float-float fields and links, float-float arithmetic on the FP32 pipe): the
// reliable updates of the mixed-precision CG.  Epilogues MINV, SCHUR_MDINV, D_MINVDAG, D_NORMAL,
// D_NORMAL_RESID.
cudaError_t launch_hop_ff(const HopParams<ff>& P, Epi e, int nsys, cudaStream_t st);
cudaError_t launch_m5_ff(const FieldRef& in, const FieldRef& out, size_t n_sites, int ns, const double* r_sys,
                         int sys_base, int nsys, int op, const Coef5<ff>& cf, cudaStream_t st);
// Pseudofermion-force contraction (kernels_force.cu): G += coef * [U K1 - K2 U^+] per link from the
// parity-split FP64 fields L (Le, Lo) and R (Re, Ro); G in the internal link order
// ((p * 4 + mu) * Vh + h) * 9.  finalize: ta(G) into the external gauge layout.
cudaError_t launch_force_contract(const Geom& g, int ns, const void* links_d18, const FieldRef& Le, const FieldRef& Lo,
                                  const FieldRef& Re, const FieldRef& Ro, double coef, double2* G, bool accumulate_into,
                                  cudaStream_t st);
cudaError_t launch_force_finalize(const Geom& g, const double2* G, double2* out_ext, cudaStream_t st);
// sum of squares of n doubles into *out (deterministic two-pass; partials: sumsq_partials() doubles)
size_t sumsq_partials();
cudaError_t launch_sumsq(const double* a, size_t n, double* partials, double* out, cudaStream_t st);
cudaError_t launch_sum_partials(const double* partials, int nb, double* out, cudaStream_t st);  // one block, fixed order
// Wilson gauge force and action, MD updates (kernels_md.cu), FP64 on the external gauge layout.
// gauge force: F (may be null) = -(beta/3) ta(U Sigma) per link; *retr_sum = sum_links Re tr(U Sigma)
// (partials: gauge_force_blocks(V) doubles)
size_t gauge_force_blocks(size_t V);
cudaError_t launch_gauge_force(const int dims[4], const double2* U, double beta, double2* F, double* partials,
                               double* retr_sum, cudaStream_t st);
cudaError_t launch_link_update(size_t nlinks, double2* U, const double2* P, double a, cudaStream_t st);  // U <- exp(aP) U
cudaError_t launch_axpy(size_t n, double2* y, const double2* x, double c, cudaStream_t st);              // y += c x
// the FP64 links split into float-float pairs (same 144-byte records)
cudaError_t launch_links_ff18_from_d18(const void* d18, void* ff18, size_t n_links, cudaStream_t st);
// Mixed path (low-precision operator fields, FP32 accumulators r/x, float links, FP32 arithmetic)
cudaError_t launch_hop_mixed(const HopParams<float>& P, Epi e, Sp low, Lk lk, int nsys, cudaStream_t st);

// Second-generation mixed CG kernels (Ns = 8 or 16): kind 1..4 = K1..K4 of the iteration
// (see kernels_mixed2.cu); the non-dagger hops read chi = B psi fields.
bool hop2_supported(int ns, Sp low, size_t vh);
cudaError_t launch_hop2(const HopParams<float>& P, int kind, Sp low, Lk lk, int nsys, cudaStream_t st);
// The hops K1, K2, K3 with two adjacent s per lane (kernels_mixed3.cu): Ns = 8 or 16, FP16 / BF16.
bool hop3_supported(int ns, Sp low, int kind);
cudaError_t launch_hop3(const HopParams<float>& P, int kind, Sp low, Lk lk, int nsys, cudaStream_t st);
// the production hop for this configuration and kind (hop3 where supported, else hop2)
cudaError_t launch_hop_prod(const HopParams<float>& P, int kind, Sp low, Lk lk, int nsys, cudaStream_t st);
// p = r (mode 0) or p = r + beta p (mode 1), and chi = B p
cudaError_t launch_p_update2(Sp low, int ns, const FieldRef& r, const FieldRef& p, const FieldRef& chi,
                             size_t n_sites, int mode, const Coef5<float>& cf, const double* r_sys, SysState* st,
                             int gate, int need, int sys_base, int nsys, unsigned long long* prof,
                             cudaStream_t stream);

// Site-local M, M^dag, M^-1, M^-dag (op 0..3); op 4 = B (the chiral shift rho + sigma L)
// gate_st (optional): only systems whose status equals `need` are processed
cudaError_t launch_m5_f64(const FieldRef& in, const FieldRef& out, size_t n_sites, int ns, const double* r_sys,
                          int sys_base, int nsys, int op, const Coef5<double>& cf, cudaStream_t st,
                          const SysState* gate_st = nullptr, int need = 0);
cudaError_t launch_m5_mixed(Sp low, const FieldRef& in, const FieldRef& out, size_t n_sites, int ns,
                            const double* r_sys, int sys_base, int nsys, int op, const Coef5<float>& cf,
                            cudaStream_t st);

// Layout conversion between external complex128 fields and internal half fields
cudaError_t launch_pack(Sp sp, const double2* ext, const FieldRef& out, const Geom& g, int p, int ns, int ext_mode,
                        cudaStream_t st);
cudaError_t launch_unpack(Sp sp, const FieldRef& in, double2* ext, const Geom& g, int p, int ns, int ext_mode,
                          cudaStream_t st);

// Vector kernels (kinds as in kernels.cuh); x and y formats given separately
// part_stride: partials per system of a reducing launch (kind 3), 0 for the grid's block count
cudaError_t launch_vec(Sp spx, Sp spy, const FieldRef& x, const FieldRef& y, size_t n5, int ns, int kind,
                       double coef, SysState* st, int gate, int need, double* partials,
                       unsigned* counters, int sys_base, int nsys, cudaStream_t stream, int part_stride = 0);

// profiling counter for the next launch_vec (nullptr: none); single-threaded use per call site
void set_vec_prof(unsigned long long* c);

cudaError_t launch_state(SysState* st, int nsys, int mode, double tol2, cudaStream_t stream);

// Gauge packing from external complex128 U[mu][t][z][y][x][3][3] (device)
cudaError_t launch_pack_links(const double2* U, void* d18, void* f18, void* f12, const Geom& g, cudaStream_t st);

// FP32 links (18 reals padded to 20, or the first two rows) from the packed FP64 links
cudaError_t launch_links_from_d18(const void* d18, void* f18, void* f12, size_t n_links, cudaStream_t st);
// FP16 links of 12 reals (rows 0, 1, round to nearest) from the packed FP64 links
cudaError_t launch_links_h12_from_d18(const void* d18, void* h12, size_t n_links, cudaStream_t st);
// Site-major copy of a link array for the second-generation hops: for each parity p and half
// site h the eight links that site's hops multiply by, contiguous: out[(p * Vh + h) * 8 + j] =
// U_mu(x) (j = 2 mu, forward) or U_mu(x - mu) (j = 2 mu + 1, backward), `bytes` per link, gathered
// from the standard [p][mu][h] array `in` through the neighbour table (both parities).
cudaError_t launch_links_site_major(const void* in, void* out, int bytes, const int* nbr, const Geom& g,
                                    cudaStream_t st);
// Neighbour table: for each parity p and half site h, the half indices of the eight
// neighbours (x+, x-, y+, y-, z+, z-, t+, t-) in the other parity, bit 31 set where the hop
// crosses the antiperiodic time boundary.  nbr[(p * Vh + h) * 8 + j], 2 * Vh * 8 ints.
cudaError_t launch_build_neighbours(int* nbr, const Geom& g, cudaStream_t st);

int lg2(int v);

// process-wide count of kernel launches issued by the library
void note_launch();
long long launch_count();
void note_launches(long long n);  // adjusts the count (graph replays: kernels per graph)
inline int blocks_for(size_t n, int bs) { return (int)((n + bs - 1) / bs); }

}  // namespace odwf
