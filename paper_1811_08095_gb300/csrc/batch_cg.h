// Slot-based batched CG on the even-odd Schur normal equations S^dag S x = b.
//
// Every iteration is four fused hop launches plus one vector update, each covering all
// slots of the batch (grid.y = slot); a slot whose status is not "running" exits at its
// first instruction, so converged systems cost nothing and new systems can be admitted
// into free slots between iterations (continuous batching).
//   K1  t = M^-1 H_oe p
//   K2  a = M^-dag (p - M^-1 H_eo t),   |p - M^-1 H_eo t|^2 = p^dag S^dag S p  -> alpha
//   K3  c = M^-dag H_eo^dag a
//   K4  A p = M^dag a - H_oe^dag c;  r -= alpha A p;  x += alpha p;  |r|^2 -> beta, status
//   P   p = r + beta p
// Mixed precision: p, t, a, c are stored in FP16 / BF16 (per-site scale) or FP32, r and x
// in FP32, all arithmetic FP32.  A system whose inner residual falls below delta times its
// largest value since the last update (or below the target) is parked; the host then
// folds x into the FP64 solution, recomputes r = b - S^dag S x in FP64 on the GPU and
// restarts the inner iteration from it (reliable updates).
//
// Memory (mixed precision): per system the FP64 solution, the FP32 inner r and x and the
// five low-precision operator fields.  The FP64 right-hand side is not copied per system:
// the caller's b (external layout) is re-packed into one shared FP64 buffer at every
// reliable update, and the FP64 residual lives in a second shared buffer.  Updates run
// one after another on the update stream, and admissions / final checks on the iteration
// stream are ordered against that stream, so the shared buffers are never used by two
// systems at once.
#pragma once

#include <chrono>
#include <map>
#include <string>
#include <vector>

#include "engine.h"
#include "profile.h"

namespace odwf {

// inner link format of a mixed-precision solve (link_recon, link_prec of the parameters)
Lk link_format(const odwf_solve_params& prm);

struct BatchCG {
    Engine* E = nullptr;
    int cap = 0;
    bool mixed = false;
    Sp low = Sp::F16;
    Sp fsp = Sp::F64;  // X64, R64, B64 and the reliable-update temporaries: F64, or FF (float-float) when mixed
    Lk lk = Lk::F12;
    double delta = 0.1;
    double tol = 1e-10;
    int max_iter = 10000;

    // per-slot fields (slabs of `cap`); in mixed mode R64 and B64 are one shared system
    HalfField X64, R64, B64;       // FP64 solution, residual, right-hand side
    HalfField P64, T64, A64, C64;  // FP64 CG (mixed = false) operator fields
    HalfField Rin, Xin;            // mixed: FP32 inner residual / solution
    HalfField Pl, Tl, Al, Cl;      // mixed: low-precision operator fields
    HalfField Chil;                // mixed (second-generation kernels): chi_p = B p
    bool v2 = false;               // second-generation mixed kernels (Ns = 8, 16)
    HalfField A1, C1;              // mixed: FP64 temporaries for reliable updates (one system)

    SysState* st = nullptr;        // device [cap]
    SysState* st_host = nullptr;   // pinned mirror
    double* r_dev = nullptr;       // device [cap]
    double* partials = nullptr;    // device [cap * nblk]
    int nblk = 0;                  // partials per system (every reducing launch's grid fits)
    unsigned* counters = nullptr;  // device [cap]
    // reliable updates run on their own stream, overlapping the other systems' iterations
    cudaStream_t s_rel = nullptr;
    std::vector<cudaEvent_t> ev_rel;  // per slot: end of its update on s_rel
    std::vector<int> upd;             // per slot: an update is in flight
    std::vector<int> n_reliable;
    std::vector<int> active;       // host view: slot holds a system
    std::vector<const double2*> bsrc;  // mixed: the slot's right-hand side (device, external layout)
    double2* bstage = nullptr;         // mixed: per-slot device copies of host right-hand sides [cap]
    cudaEvent_t ev_sync = nullptr;     // orders the shared FP64 buffers between the two streams
    std::vector<double> mq;
    std::vector<double> slot_tol;
    // A chunk of k iterations over slots lo..lo+n-1 is captured once into a CUDA graph and
    // replayed (launch-bound small lattices; not while the kernel profiler is enabled).
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;
    };
    std::map<unsigned long long, GraphEntry> graphs;
    int pcls[5] = {-1, -1, -1, -1, -1};  // profiler classes: K1..K4, p update
    std::string kname[5];                 // (second-generation kernels) class names and
    double kbytes_sys[5] = {0}, kbytes_launch[5] = {0};  // algorithmic bytes per system / launch
    int pcls_rel[4] = {-1, -1, -1, -1};  // FP64 residual hops of the reliable update

    ~BatchCG();
    // update_prio_drop: priority levels of the update stream below the iteration stream s
    // (1 in a single batch, so that the other systems' iterations keep the SMs first; 0 in
    // the serving loop, where a group's updates must not fall below other groups' iterations)
    int init(Engine* e, int capacity, const odwf_solve_params& prm, cudaStream_t s, int update_prio_drop = 0);
    // b_ext: even-site external field (complex128).  A device pointer is read again at every
    // reliable update (mixed precision) and must stay valid until finalize(); a host pointer is
    // copied.  tol_slot / max_iter_slot <= 0 keep the batch defaults.
    int admit(int slot, const double2* b_ext, double mq_slot, cudaStream_t s, double tol_slot = 0,
              int max_iter_slot = 0);
    int admit_internal(int slot, cudaStream_t s, double tol_slot = 0, int max_iter_slot = 0);  // B64[slot] filled
    int release(int slot);  // slot free for the next admit
    // stop a running slot between chunks (its device status becomes idle, after any reliable
    // update in flight) and free it; its solution is not written out
    int cancel(int slot, cudaStream_t s);
    int run_iterations(int k, cudaStream_t s);
    int resume(cudaStream_t s, bool block);          // rejoin slots whose update finished
    int poll(cudaStream_t s);                      // refresh st_host (synchronizes s)
    int service(cudaStream_t s);                   // reliable updates for parked slots
    int finalize(int slot, double2* x_ext, cudaStream_t s, double* true_resid);
    // second-generation mixed iteration pieces (v2 only): K1..K4 hops, and the p update
    int launch_v2_hops(int lo, int n, cudaStream_t s);
    int launch_v2_pupdate(int mode, int lo, int n, int gate, int need, cudaStream_t s);
    int launch_v2_kernel(int kind, int lo, int n, cudaStream_t s);  // kind 1..4: K1..K4 alone, 5: P
    // write a slot's scalars (and r = m_q / (2 m0)) directly; synchronizes s
    int set_state(int slot, const SysState& init, double r, cudaStream_t s);
    bool slot_running(int i) const;
    bool slot_finished(int i) const;
    int any_running() const;

   private:
    template <class R>
    HopParams<R> params(int p_out) const;
    int ff_residual(int slot, cudaStream_t s);
    int fp64_residual(int slot, cudaStream_t s);
    int launch_iterations(int k, int lo, int n, cudaStream_t s);
    void drop_graphs();
    FieldRef Rref() const { return mixed ? R64.ref_shared() : R64.ref(); }
    FieldRef Bref() const { return mixed ? B64.ref_shared() : B64.ref(); }
    int load_b(int slot, cudaStream_t s);               // mixed: pack the slot's b into the shared B64
    int order_after(cudaStream_t first, cudaStream_t then);  // `then` waits for work queued on `first`
};

}  // namespace odwf
