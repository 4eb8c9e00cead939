// Host engine behind the C ABI: one handle per (lattice, Ns, m0, weights).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/odwf.h"
#include "kernels.cuh"
#include "kernels.h"

namespace odwf {

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define ODWF_CK(call)                                           \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

bool is_device_ptr(const void* p);
// ODWF_EINVAL when p is device memory of a GPU other than `dev` (kernels on `dev` cannot read it
// without peer access); host, managed and unknown pointers pass.
int check_ptr_device(const void* p, int dev, const char* what);
int check_params(const odwf_solve_params* prm);  // ODWF_EINVAL with a message for bad solve parameters

// A device buffer owned by the engine.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// A half field for `nsys` systems (system slabs `stride` bytes apart) in format `sp`.
struct HalfField {
    Sp sp = Sp::F64;
    void* data = nullptr;
    float* norm = nullptr;
    size_t stride = 0;       // bytes per system
    size_t norm_stride = 0;  // floats per system
    FieldRef ref() const { return FieldRef{data, norm, stride, norm_stride}; }
    FieldRef ref_shared() const { return FieldRef{data, norm, 0, 0}; }  // same buffer for every system
    FieldRef ref_sys(int i) const {  // system i as a single-system field
        return FieldRef{(char*)data + i * stride, norm ? norm + i * norm_stride : nullptr, 0, 0};
    }
};

struct Engine {
    odwf_lattice lat{};
    Geom g{};
    int ns = 0;
    int lg_ns = 0;
    double m0 = 0, mq = 0;
    std::vector<double> omega;
    Coef5<double> cf64{};
    Coef5<float> cf32{};
    Coef5<ff> cfff{};  // the FP64 coefficients as float-float pairs (reliable updates)
    int device = 0;

    // packed links
    void* links_d18 = nullptr;
    void* links_f18 = nullptr;
    void* links_f12 = nullptr;
    void* links_h12 = nullptr;
    void* links_ff18 = nullptr;  // the FP64 links as float-float pairs (reliable updates)
    void* links_site[4] = {nullptr, nullptr, nullptr, nullptr};  // site-major copies by Lk (second-generation hops)
    bool have_site[4] = {false, false, false, false};
    int* nbr = nullptr;  // neighbour table of the second-generation hops (launch_build_neighbours)
    unsigned* bounds_flag = nullptr;  // device word for the debug build's index checks
    bool gauge_set = false;
    bool have_f12 = false, have_f18 = false, have_h12 = false;  // low-precision copies of the FP64 links
    bool have_ff18 = false;
    const void* links_of(Lk lk) const {
        return lk == Lk::F12 ? links_f12 : lk == Lk::F18 ? links_f18 : lk == Lk::H12 ? links_h12
             : lk == Lk::FF18 ? links_ff18 : links_d18;
    }

    // named workspaces (grow-only)
    std::map<std::string, DevBuf> ws;
    void* pinned = nullptr;
    size_t pinned_bytes = 0;

    ~Engine();
    int init(const odwf_lattice* l, int Ns, double m0_, double mq_, const double* w);
    int set_gauge(const void* U, cudaStream_t st);
    int ensure_links(Lk lk, cudaStream_t st);  // FP32 links in format lk, converted on first use
    int ensure_site_links(Lk lk, cudaStream_t st);  // site-major copy of format lk (after ensure_links)
    // debug builds: ODWF_ECUDA when a kernel recorded an out-of-range index (synchronizes st)
    int bounds_status(cudaStream_t st);

    size_t vh() const { return (size_t)g.Vh; }
    size_t sites5() const { return (size_t)g.Vh * ns; }
    size_t half_bytes(Sp sp) const;
    size_t norm_count() const { return sites5(); }
    size_t ext_bytes(int mode) const { return (mode == ODWF_MODE_FULL ? 2 : 1) * sites5() * 192; }

    void* get_ws(const std::string& name, size_t bytes, int* rc);
    int alloc_half(const std::string& name, Sp sp, int nsys, HalfField* f);
    void* host_stage(size_t bytes, int* rc);

    // parameters of one hop launch
    template <class R>
    HopParams<R> hop_params(int p_out, const double* r_dev) const;

    // FP64 operators on internal half fields (single system, r from r_dev[0])
    int apply_schur64(const HalfField& in, const HalfField& out, bool dag, const double* r_dev, cudaStream_t st);
    int apply_full64(const HalfField& in_e, const HalfField& in_o, const HalfField& out_e, const HalfField& out_o,
                     bool dag, const double* r_dev, cudaStream_t st);

    // C-ABI level operations
    int apply(void* out, const void* in, int mode, bool dag, cudaStream_t st);
    int apply_normal(void* out, const void* in, int system, cudaStream_t st);
    int apply_m5(void* out, const void* in, long n_sites, int op, cudaStream_t st);
    int gauge_force(const double2* U, double beta, double* action, double2* F, cudaStream_t st);
    int gauge_force_api(const void* U, double beta, double* action, void* force, cudaStream_t st);
    int md_trajectory(void* U, void* P, int nterms, const void* const* phi, const double* m1, const double* m2,
                      double beta, double tau, int nsteps, int integrator, int n_inner,
                      const odwf_solve_params* prm, double* energies, odwf_solve_stats* stats, cudaStream_t st);
    int pf_force(const void* phi, double m1, double m2, const odwf_solve_params* prm, double* action, void* force,
                 odwf_solve_stats* stats, cudaStream_t st);
    int pf_heatbath(const void* eta, double m1, double m2, const odwf_solve_params* prm, void* phi,
                    odwf_solve_stats* stats, cudaStream_t st);
    int apply_ff_normal(void* out, const void* in, cudaStream_t st);
    int apply_low_normal(void* out, const void* in, int prec, int recon, cudaStream_t st);
    int mixed_cg_step(int prec, int recon, int link_prec, double mq_step, const void* p_prev, const void* r, const void* x,
                      void* const* outs, odwf_cg_step_scalars* sc, cudaStream_t st);
    int effective_solve(void* x, const void* b, const odwf_solve_params* prm, odwf_solve_stats* stats,
                        cudaStream_t st);
    int residual_mass(const int32_t site[4], const odwf_solve_params* prm, double* mres, double* corr,
                      odwf_solve_stats* stats, cudaStream_t st);
    int time_kernel(int kind, int prec, int recon, int link_prec, int nsys, int reps, const void* fill,
                    odwf_kernel_prof* out, cudaStream_t st);
    int solve(int nsys, void* const* x, const void* const* b, const double* mq_arr, const odwf_solve_params* prm,
              odwf_solve_stats* stats, cudaStream_t st);
    int solve_on(int nsys, void* const* x, const void* const* b, const double* mq_arr,
                 const odwf_solve_params* prm, odwf_solve_stats* stats, cudaStream_t st);
    int solve_full(void* x, const void* b, const odwf_solve_params* prm, odwf_solve_stats* stats,
                   cudaStream_t st);
};

}  // namespace odwf

struct odwf_handle {
    odwf::Engine e;
};
