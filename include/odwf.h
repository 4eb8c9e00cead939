/*
 * odwf.h -- C ABI of the GB300 optimal domain-wall fermion (ODWF) solver library.
 *
 * The library applies the 5D ODWF operator of Chiu, "Simulation of dynamical
 * (u,d,s,c) domain-wall/overlap quarks at the physical point" (LATTICE2018), Sec. 2,
 *
 *   (D psi)_s = (rho_s D_w + 1) psi_s + (sigma_s D_w - 1) (L psi)_s,   s = 1..Ns,
 *   D_w psi(x) = (4 - m0) psi(x) - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                             + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)],
 *   L = P_+ L_+ + P_- L_-,  (L_+ psi)_s = psi_{s-1} (s > 1), (L_+ psi)_1 = -r psi_Ns,
 *                           (L_- psi)_s = psi_{s+1} (s < Ns), (L_- psi)_Ns = -r psi_1,
 *   r = m_q / (2 m0),  P_+- = (1 +- gamma_5)/2,
 *
 * with the paper's c = 1, d = 0 (rho_s = sigma_s = omega_s, the optimal weights),
 * its adjoint D^dag, and even-odd preconditioned conjugate-gradient solves of the
 * Hermitian positive-definite normal equations that the pseudofermion forces of
 * Eq. (1)-(2) need (Sec. 2, "conjugate gradient").  Everything runs on one GPU.
 *
 * Conventions (all public fields are complex128, i.e. interleaved re/im doubles):
 *   lattice   dims = {Lx, Ly, Lz, Lt}, every extent even and >= 2; site index
 *             lex = x + Lx (y + Ly (z + Lz t)); a site is even when x+y+z+t is even.
 *   gauge     U[mu][t][z][y][x][a][b], mu = 0..3 <-> x, y, z, t, SU(3) row a, column b.
 *             t_antiperiodic != 0 gives hops across t = Lt-1 <-> 0 a factor -1.
 *   spinor    FULL:       psi[s][t][z][y][x][spin][colour]          (Ns * V * 12 complex)
 *             SCHUR_EVEN: psi[s][lex/2][spin][colour] over even sites (Ns * V/2 * 12 complex)
 *   gammas    chiral basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1..3 <-> mu = 0..2),
 *             gamma_4 = [[0, 1], [1, 0]] (mu = 3), gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 =
 *             diag(1, 1, -1, -1): spins 0, 1 are P_+, spins 2, 3 are P_-.
 *   Schur     S = 1 - M^-1 H_eo M^-1 H_oe on even sites, with M the site-local part of D
 *             (D_w -> 4 - m0) and H = D - M the parity-coupling hops.
 *
 * Pointers: every field argument may be device memory or host memory (pageable or
 * pinned); the library detects which and copies host data through its own device
 * staging buffers.  Device pointers are used in place.  The caller owns every buffer
 * it passes; the library owns its packed links, coefficients and workspaces, all
 * freed by odwf_destroy.  `stream` is a cudaStream_t (NULL = legacy default stream);
 * calls with device pointers are stream-ordered, calls with host pointers return
 * after the result is in host memory.
 *
 * Errors: every entry point returns an int status (ODWF_OK = 0); no exception
 * crosses the ABI.  odwf_last_error() gives a message for the calling thread's
 * last failure.
 *
 * Threads: a handle keeps workspaces and solver state, so calls on one handle must not
 * overlap (use one handle per thread, or serialise); different handles are independent.
 * The serving functions (serve_*) may be called from any number of threads.
 */
#ifndef ODWF_H
#define ODWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ODWF_OK = 0,
    ODWF_EINVAL = 1,      /* bad argument (sizes, modes, pointers) */
    ODWF_ENOMEM = 2,      /* device allocation failed / HBM budget exceeded */
    ODWF_ENOCONV = 3,     /* solver hit max_iter before the tolerance */
    ODWF_EBREAKDOWN = 4,  /* CG breakdown: p^dag A p <= 0 or a non-finite scalar */
    ODWF_ETIMEOUT = 5,    /* a bounded wait ran out */
    ODWF_ECUDA = 6,       /* a CUDA runtime call failed */
    ODWF_PENDING = 7,     /* serving: request still queued or running */
    ODWF_ENOTFOUND = 8,   /* serving: unknown ticket or field id */
    ODWF_ECANCELED = 9,   /* serving: the request was cancelled (serve_cancel) */
    ODWF_EBUSY = 10       /* serving: the queue is full (serve_set_policy); the request was not taken */
};

/* ODWF_FF: float-float, each real the unevaluated sum of two FP32 numbers (about 48 bits),
 * arithmetic built from FP32 operations: the reliable updates of the mixed-precision CG. */
typedef enum { ODWF_F64 = 0, ODWF_F32 = 1, ODWF_F16 = 2, ODWF_BF16 = 3, ODWF_FF = 4 } odwf_prec;

enum { ODWF_MODE_FULL = 0, ODWF_MODE_SCHUR_EVEN = 1 };

enum {
    ODWF_SYS_SCHUR_NORMAL = 0, /* S^dag S x_e = b_e,  SCHUR_EVEN fields */
    ODWF_SYS_FULL_NORMAL = 1,  /* D^dag D x = b,       FULL fields (two Schur solves) */
    ODWF_SYS_FULL_DIRAC = 2    /* D x = b,             FULL fields (Schur solve + reconstruction) */
};

enum { ODWF_OMEGA_SHIFTED_R5 = 0, ODWF_OMEGA_PLAIN = 1 };

enum { ODWF_UPDATES_AUTO = 0, ODWF_UPDATES_F64 = 1, ODWF_UPDATES_FF = 2 };

typedef struct {
    int32_t dims[4];        /* Lx, Ly, Lz, Lt */
    int32_t t_antiperiodic; /* 1: antiperiodic in time, 0: periodic */
} odwf_lattice;

typedef struct odwf_handle odwf_handle;

typedef struct {
    double tol;         /* target true relative residual ||b - A x|| / ||b|| (e.g. 1e-10) */
    int32_t max_iter;   /* cap on inner CG iterations (summed over restarts) */
    int32_t prec;       /* ODWF_F64: plain FP64 CG; ODWF_F32/F16/BF16: mixed precision with that
                           storage for the inner operator fields, FP32 arithmetic, reliable updates
                           (true residual b - A x) in FP64 or float-float (update_arith) */
    double delta;       /* reliable-update trigger: recompute the FP64 residual when the inner
                           residual drops below delta x its largest value since the last update
                           (<= 0 selects 0.01) */
    int32_t system;     /* ODWF_SYS_* */
    int32_t link_recon; /* mixed inner links: 12 (two rows, third reconstructed) or 18; 0 = 12 */
    double mq;          /* quark mass for this solve; NaN keeps the handle's m_q */
    int32_t check_every;/* host status poll interval in iterations (0 = 8) */
    int32_t link_prec;  /* mixed inner links: 0 or ODWF_F32 = FP32; ODWF_F16 = FP16 with 12 reals
                           (24 bytes per link, no scale: SU(3) entries have modulus <= 1; needs
                           Ns = 8 or 16 and link_recon 0 or 12) */
    int32_t update_arith; /* mixed: arithmetic of the reliable updates (true residual b - A x) and of
                           the accumulated solution.  ODWF_UPDATES_AUTO (0) and ODWF_UPDATES_FF:
                           float-float (pairs of FP32, about 48 bits, on the FP32 pipe);
                           ODWF_UPDATES_F64: FP64.  Both resolve the true residual far below 1e-10;
                           on GB300, whose FP64 rate is a small fraction of its FP32 rate,
                           float-float is faster for one system and for batches.  Full-lattice
                           systems (FULL_NORMAL, FULL_DIRAC) always update in FP64. */
} odwf_solve_params;

typedef struct {
    int32_t iters;          /* inner CG iterations */
    int32_t n_reliable;     /* FP64 residual recomputations */
    double true_resid;      /* final ||b - A x|| / ||b||, recomputed on the GPU (FP64, or float-float
                               for mixed solves that update in float-float) */
    double time_ms;         /* wall time of the solve inside the library */
    int32_t status;         /* ODWF_OK / ODWF_ENOCONV / ODWF_EBREAKDOWN for this system */
    int32_t reserved;
} odwf_solve_stats;

/* Last error message of the calling thread ("" if none). */
const char* odwf_last_error(void);

/* Library version string. */
const char* odwf_version(void);

/*
 * Optimal weights omega_s (Sec. 2): Zolotarev's optimal rational approximation
 * R_Z(x) of 1/sqrt(x), degree (n-1, n) for Ns = 2n, on x in [1, (lmax/lmin)^2].
 * variant ODWF_OMEGA_SHIFTED_R5 (the paper's choice): S(H) = sqrt(x) R_Z(x)/(1 + d_Z)
 *   with 0 <= 1 - S <= 2 d_Z; the weights are n distinct values, each twice, returned
 *   as w_1 < ... < w_n, w_n, ..., w_1 (R5 symmetric: omega_s = omega_{Ns+1-s}).
 * variant ODWF_OMEGA_PLAIN: S = sqrt(x) R_Z(x), |1 - S| <= d_Z, 2n distinct weights
 *   in increasing order.
 * omega_out: host array of Ns doubles; dz_out (may be NULL): d_Z.  Host-only, no GPU.
 * Returns ODWF_EINVAL for odd Ns, Ns < 2, Ns > 64 or 0 < lmin < lmax violated.
 */
int odwf_zolotarev_omega(int Ns, double lmin, double lmax, int variant, double* omega_out,
                         double* dz_out);

/*
 * Create a handle for one lattice, Ns, m0, default m_q and weights (Sec. 2).
 * omega: host array of Ns doubles (rho_s = sigma_s = omega_s).  Ns must divide 32
 * (2, 4, 8, 16 or 32).  Allocates nothing large; links come with odwf_set_gauge.
 * *out receives the handle; ODWF_EINVAL on bad sizes, ODWF_ECUDA without a device.
 */
int odwf_create(const odwf_lattice* lat, int Ns, double m0, double mq, const double* omega,
                odwf_handle** out);

/* Free the handle and everything the library allocated for it. */
int odwf_destroy(odwf_handle* h);

/*
 * Set the gauge field: U (host or device, complex128, layout above).  The library
 * packs it into its internal parity-split arrays: FP64 with 18 reals for the FP64
 * path and FP32 with 12 reals (third row rebuilt as conj(row1 x row2), exact for
 * SU(3)) plus 18 reals for the mixed path.  The time-boundary sign is applied in the
 * kernels, so the stored links stay in SU(3).  Stream-ordered on `stream`.
 */
int odwf_set_gauge(odwf_handle* h, const void* U, void* stream);

/*
 * out = D in (mode ODWF_MODE_FULL, full fields) or out = S in (ODWF_MODE_SCHUR_EVEN,
 * even-site fields), in FP64.  in and out must not overlap.
 */
int odwf_apply(odwf_handle* h, void* out, const void* in, int mode, void* stream);

/* out = D^dag in or out = S^dag in, as odwf_apply. */
int odwf_apply_dagger(odwf_handle* h, void* out, const void* in, int mode, void* stream);

/*
 * out = A in for the normal operator of `system`: S^dag S (SCHUR_NORMAL, even fields)
 * or D^dag D (FULL_NORMAL, full fields), FP64.
 */
int odwf_apply_normal(odwf_handle* h, void* out, const void* in, int system, void* stream);

/*
 * out = S^dag S in computed by the mixed-precision inner operator: in is rounded to
 * `prec` storage (ODWF_F32, ODWF_F16 or ODWF_BF16; FP16/BF16 with one FP32 scale per 5D
 * site), the four hops run in FP32 with FP32 links of `link_recon` (12 or 18) reals, and
 * every intermediate field is stored in `prec`.  Even-site fields, as odwf_apply_normal.
 * This is the operator the inner CG iterates with; it is exposed for accuracy checks.
 * prec = ODWF_FF gives the reliable updates' operator instead: float-float fields, links and
 * arithmetic throughout (link_recon is ignored).
 */
int odwf_apply_normal_prec(odwf_handle* h, void* out, const void* in, int prec, int link_recon, void* stream);

/*
 * Site-local part of D on a field of n_sites sites per s-slice (any sites, layout
 * [s][site][spin][colour]): op 0 = M, 1 = M^dag, 2 = M^-1, 3 = M^-dag, in FP64.
 * M = (4-m0) B + 1 - L with B = rho + sigma L; the inverse is an O(Ns) cyclic solve.
 */
int odwf_apply_m5(odwf_handle* h, void* out, const void* in, long n_sites, int op, void* stream);

/*
 * odwf_apply_m5 without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that must not let a library call cudaMalloc -- applications
 * whose own memory manager has already reserved the GPU's memory (a library-side
 * cudaMalloc would fail or fragment that pool) and latency-critical code that cannot
 * accept the device-wide synchronisation cudaMalloc and cudaFree imply.
 *
 * Computes out = op(in) for op 0 = M, 1 = M^dag, 2 = M^-1, 3 = M^-dag exactly as
 * odwf_apply_m5 does, for the operator with Ns, m0, mq and weights omega (host array of
 * Ns doubles; rho = sigma = omega), on n_sites sites in the layout
 * [s][site][spin][colour] (complex128).  No handle is needed.
 *   in, out   device memory, n_sites * Ns * 12 complex values each, not overlapping;
 *             host pointers are rejected with ODWF_EINVAL (staging them would allocate).
 *   limit     n_sites * Ns <= 65536; larger requests return ODWF_EINVAL.  The staging
 *             fields live in a fixed 24 MiB + 256 B device array that every GPU which
 *             loads the library keeps until the process exits.
 *   set-up    the first call on each device looks up that array's device address
 *             (cudaGetSymbolAddress) with the device current; make that first call
 *             before any stream capture begins.  Under CUDA's lazy module loading (the
 *             default) that first call is also when the device reserves the array's 24 MiB:
 *             a caller whose own pool will take most of the GPU's memory should make one
 *             small call (n_sites = 1) on each device before reserving its pool.  With
 *             CUDA_MODULE_LOADING=EAGER the array is reserved when the context is created.
 *             in and out must be memory of the current device (ODWF_EINVAL otherwise).
 *   sharing   every call uses the same array, which keeps the last call's contents
 *             (each call writes all it reads first); calls whose work overlaps on the
 *             GPU -- different streams, or host threads -- race on it and must be
 *             serialised by the caller.
 * Stream-ordered on `stream`; returns ODWF_OK, ODWF_EINVAL or ODWF_ECUDA.
 */
int odwf_apply_m5_noalloc(int Ns, double m0, double mq, const double* omega, void* out, const void* in,
                          long n_sites, int op, void* stream);

/*
 * Solve one system by conjugate gradient (Sec. 2).  x: initial guess ignored, result
 * written; b: right-hand side (layouts by system).  stats may be NULL.
 * The solve runs on an internal stream joined to `stream` at both ends and returns when it
 * has finished.  Chunks of iterations are replayed as CUDA graphs unless the kernel profiler
 * is enabled or the environment sets ODWF_GRAPHS=0.
 * Returns ODWF_OK on convergence to params->tol, ODWF_ENOCONV at max_iter (x holds the
 * last iterate), ODWF_EBREAKDOWN on a breakdown.
 */
int odwf_cg_solve(odwf_handle* h, void* x, const void* b, const odwf_solve_params* params,
                  odwf_solve_stats* stats, void* stream);

/*
 * Solve nsys systems that share the handle's gauge field, Ns, m0 and weights but
 * have their own right-hand side b[i] and mass mq[i] (mq may be NULL: the handle's
 * m_q), in one batched launch sequence: every hop launch covers all unconverged
 * systems and reuses each site's links across them; converged systems are masked
 * out.  stats: array of nsys entries (may be NULL).  Returns the first non-OK
 * per-system status, or ODWF_OK.  SCHUR_NORMAL only.
 */
int odwf_cg_solve_batched(odwf_handle* h, int nsys, void* const* x, const void* const* b,
                          const double* mq, const odwf_solve_params* params,
                          odwf_solve_stats* stats, void* stream);

/*
 * One iteration of the mixed-precision inner CG (Sec. 2's CG on the normal equations, with
 * the storage formats of odwf_cg_solve's mixed modes), through exactly the kernels the
 * batched solver launches every iteration, returning every field the iteration stores.  It
 * is exposed so that each stored field can be checked against an FP64 reference element by
 * element.  With W the hopping sum of D_w = (4 - m0) - W/2, B = rho + sigma L and
 * M = (4 - m0) B + 1 - L (so H = -1/2 W B and S = 1 - M^-1 H_eo M^-1 H_oe):
 *   p     = r + beta p_prev              (stored in `prec`)
 *   chi_p = B p                          (stored; the non-dagger hops read it)
 *   chi_t = B M^-1 (-1/2 W chi_p)        (odd sites; = B t with t = M^-1 H_oe p)
 *   s     = p - M^-1 (-1/2 W chi_t)      (= S p, not stored);  pAp = |s|^2;  alpha = rr / pAp
 *   a     = M^-dag s
 *   c     = M^-dag B^dag (-1/2 W^dag a)  (odd sites)
 *   Ap    = M^dag a - B^dag (-1/2 W^dag c)   (= S^dag S p, not stored)
 *   r_new = r - alpha Ap,  x_new = x + alpha p   (FP32);  rr_new = |r_new|^2
 * prec: ODWF_F32, ODWF_F16 or ODWF_BF16 (FP16/BF16 with one FP32 scale per 5D site);
 * link_recon: 12 or 18 (0 = 12); link_prec: as odwf_solve_params.link_prec (ODWF_F16 needs
 * link_recon 12); mq: the mass of this system (r = mq / (2 m0)).
 * p_prev, r, x: even-site fields (SCHUR_EVEN layout, host or device); r and x are rounded to
 * FP32 and p_prev to `prec` on entry.  outs: 8 pointers (host or device, each may be NULL),
 * receiving the stored fields in the SCHUR_EVEN layout of their parity (odd-site fields in
 * the same [s][lex/2][spin][colour] order over odd sites):
 *   0 p_prev as stored, 1 p, 2 chi_p, 3 chi_t (odd), 4 a, 5 c (odd), 6 r_new, 7 x_new.
 * sc: in: beta, rr (> 0); out: pAp, alpha, rr_new, status (ODWF_EBREAKDOWN when pAp <= 0 or
 * non-finite; the later fields are then not written by the kernels).  Needs Ns = 8 or 16.
 * Allocates its own workspaces (freed by odwf_destroy); returns when the outputs are written.
 */
typedef struct {
    double beta;    /* in */
    double rr;      /* in: |r|^2 of the incoming residual */
    double pAp;     /* out: |S p|^2 */
    double alpha;   /* out: rr / pAp */
    double rr_new;  /* out: |r_new|^2 */
    int32_t status; /* out */
    int32_t reserved;
} odwf_cg_step_scalars;

int odwf_mixed_cg_step(odwf_handle* h, int prec, int link_recon, int link_prec, double mq, const void* p_prev,
                       const void* r, const void* x, void* const* outs, odwf_cg_step_scalars* sc, void* stream);

/*
 * The 4D effective operator of Sec. 2 (the shifted-Zolotarev overlap that ODWF realizes):
 *   x = D_eff(m_q)^-1 b,   D_eff(m_q) = (1 + r)/2 + (1 - r)/2 gamma_5 S(H_w),  r = m_q / (2 m0),
 * computed through the 5D operator as [P^-1 D(m_q)^-1 D(2 m0) P (b (x) e_1)]_1 with
 * P_{s,s'} = P_- delta_{s,s'} + P_+ delta_{s+1,s'} (s + 1 cyclic): D(2 m0) is applied in FP64 and
 * D(m_q) y = eta is a FULL_DIRAC solve with `params` (prec, tol, max_iter, mq; system ignored).
 * b, x: 4D fields psi[t][z][y][x][spin][colour] (V * 12 complex128, host or device, not
 * overlapping).  Returns the D(m_q) solve's status; stats (may be NULL) describe that solve.
 */
int odwf_effective_solve(odwf_handle* h, void* x, const void* b, const odwf_solve_params* params,
                         odwf_solve_stats* stats, void* stream);

/*
 * Residual mass of the effective operator at a point source (Sec. 3, Table 1's quantity).  The
 * formula the paper uses is cited, not printed; the reading implemented is: with
 * G = (D_c + m_q)^-1 = (D_eff^-1 - 1) / (2 m0 - m_q) the propagator of the chirally symmetric
 * D_c = D (1 - D/(2 m0))^-1, D = (2 m0 D_eff - m_q) / (1 - m_q/(2 m0)),
 *   m_res = tr G_00 / sum_x tr (G_x0^dag G_x0) - m_q,
 * which vanishes for an exact sign function.  Twelve effective solves (one per spin-colour
 * component of the source at `site` = {x, y, z, t}).  params as odwf_effective_solve (the mass
 * is params->mq, NaN: the handle's).  *mres receives m_res; corr (Lt doubles, may be NULL)
 * the pseudoscalar correlator C(t) = sum over the time slice t0 + t of tr (G_x0^dag G_x0).
 * Returns the worst solve status (ODWF_OK when all converged).
 */
int odwf_residual_mass(odwf_handle* h, const int32_t* site, const odwf_solve_params* params, double* mres,
                       double* corr, odwf_solve_stats* stats, void* stream);

/* ----------------------------------------------------------------------------------
 * Kernel timing (no counterpart in the paper; used to place the kernels on the roofline).
 * ---------------------------------------------------------------------------------- */
typedef struct {
    char name[48];              /* kernel class, e.g. "mixed.f16.K4_normal_cg" */
    int64_t launches;           /* timed launches */
    int64_t system_launches;    /* (system, launch) pairs that ran (gated systems excluded) */
    double total_ms;            /* summed CUDA-event time of the launches, on their stream */
    double bytes_per_system;    /* algorithmic bytes per running system: each field read or
                                   written once */
    double bytes_per_launch;    /* algorithmic bytes per launch shared by all systems (links) */
} odwf_kernel_prof;

/* Start (on != 0, counters reset) or stop timing the solver's kernels.  Process-wide;
 * adds two event records per launch. */
int odwf_profile_enable(int on);

/* Synchronize the device and copy up to max_entries kernel classes with launches into
 * out; *n_out receives the count. */
int odwf_profile_read(odwf_kernel_prof* out, int max_entries, int* n_out);

/*
 * Two-flavour pseudofermion action and its force (Sec. 2: the two-flavour parts of the HMC, with
 * mass preconditioning by auxiliary heavy masses).  The action's formula is cited by the paper,
 * not printed; this is the ratio form: det D(m) = det(M(m))^2 det S(m) with M free of links, so
 *     S_pf = phi^+ S(m2)^+ (S(m1)^+ S(m1))^-1 S(m2) phi = |S(m1) X|^2,  X = (S(m1)^+ S(m1))^-1 S(m2) phi
 * represents det[D(m1)^+ D(m1)] / det[D(m2)^+ D(m2)]: m2 = 2 m0 (Pauli-Villars) is the plain
 * two-flavour factor, a chain m_q -> m_H1 -> m_H2 -> 2 m0 the mass-preconditioned product.
 * phi: even-site field (host or device, SCHUR_EVEN layout).  The solve for X runs with `params`
 * (tol, max_iter, prec, delta, ...; system and mq are set here) and its statistics go to stats
 * (may be NULL).  action (host): S_pf.  force (host or device, complex128, gauge layout
 * [mu][t][z][y][x][3][3], or NULL): per link the traceless anti-Hermitian Pi with
 * dS_pf/deps = tr(T Pi) for U_mu(x) -> exp(eps T) U_mu(x), T traceless anti-Hermitian.
 * Everything but the inner solve is FP64.  Allocates its FP64 workspaces on the handle (nine
 * even-site fields and the per-link sums).  Synchronises `stream`.
 */
int odwf_pf_force(odwf_handle* h, const void* phi, double m1, double m2, const odwf_solve_params* params,
                  double* action, void* force, odwf_solve_stats* stats, void* stream);

/*
 * Heat bath of the pseudofermion field of odwf_pf_force (Sec. 2's two-flavour parts): for a
 * Gaussian eta (even-site field, host or device, SCHUR_EVEN layout, components with
 * <|eta_i|^2> = 1), phi = S(m2)^-1 S(m1)^+ eta, so that S_pf(phi) = |eta|^2 and phi is distributed
 * as exp(-S_pf).  S(m2) phi = S(m1)^+ eta is solved as (S(m2)^+ S(m2)) phi = S(m2)^+ S(m1)^+ eta by
 * the library's CG with `params` (system and mq set here); its statistics go to stats (may be
 * NULL).  phi: output, host or device, SCHUR_EVEN layout.  Synchronises `stream`.
 */
int odwf_pf_heatbath(odwf_handle* h, const void* eta, double m1, double m2, const odwf_solve_params* params,
                     void* phi, odwf_solve_stats* stats, void* stream);

/*
 * Wilson plaquette gauge action and force (Sec. 2: the gauge action of the HMC at beta = 6/g0^2).
 * U: gauge field (host or device, complex128, [mu][t][z][y][x][3][3], the layout of
 * odwf_set_gauge; need not be the handle's field, which this call leaves unchanged).
 * action (host): S_g = beta sum_plaquettes (1 - Re tr P / 3).  force (host or device, the layout
 * of U, or NULL): per link Pi_mu(x) = -(beta/3) ta(U_mu(x) Sigma_mu(x)), Sigma the sum of the six
 * staples and ta the traceless anti-Hermitian part, so that dS_g/deps = tr(T Pi) for
 * U_mu(x) -> exp(eps T) U_mu(x).  FP64; the sum over links is in a fixed order (deterministic).
 * Synchronises `stream`.
 */
int odwf_gauge_force(odwf_handle* h, const void* U, double beta, double* action, void* force, void* stream);

/*
 * One molecular-dynamics trajectory of the HMC (Sec. 2: Wilson gauge action, two-flavour
 * pseudofermion terms with mass preconditioning, the Omelyan integrator) for
 *     H = K(P) + S_g(U) + sum_i S_pf(U; phi_i, m1[i], m2[i]),   K = -sum_links tr(P^2),
 * integrating dU/dt = P U, dP/dt = Pi / 2 (Pi the sum of the forces of odwf_gauge_force and
 * odwf_pf_force) over time tau in nsteps steps of eps = tau / nsteps.
 * integrator 0: leapfrog, P += eps/4 Pi, U <- exp(eps P) U, P += eps/4 Pi.
 * integrator 1: Omelyan (minimum norm, second order, lambda = 0.1931833275037836),
 *   P += lambda eps/2 Pi, U <- exp(eps/2 P) U, P += (1 - 2 lambda) eps/2 Pi, U <- exp(eps/2 P) U,
 *   P += lambda eps/2 Pi.
 * n_inner 0: one time scale, Pi the total force.  n_inner >= 1 (Sexton-Weingarten multiple time
 *   scales): the steps above kick with the pseudofermion forces alone, and each of their drifts
 *   U <- exp(h P) U is replaced by n_inner steps of the same integrator over time h under the
 *   gauge force alone (no solve on the inner scale).
 * U, P: device memory, complex128, gauge layout; updated in place.  P traceless anti-Hermitian.
 * phi[i] (host or device, SCHUR_EVEN layout), m1[i], m2[i] (host): 0 <= nterms <= 16 pseudofermion
 * terms; every solve runs with `params` (system and mq set per term).  energies (host, 2): H at
 * the start and at the end.  stats (may be NULL): iters and n_reliable summed over the
 * trajectory's solves, the largest true_resid, the summed time_ms, the first non-OK status.  The handle's gauge field is replaced by U at every force
 * evaluation and holds the final U on return.  FP64 except the inner solves.  No accept/reject
 * step and no momentum refresh: the caller draws P and phi and decides.  Synchronises `stream`.
 * Errors: ODWF_EINVAL for null or host U/P, nterms out of range, nsteps < 0, n_inner outside
 * [0, 1000], non-finite tau or beta, an unknown integrator or bad params; the solver's codes from the inner solves.
 */
int odwf_md_trajectory(odwf_handle* h, void* U, void* P, int nterms, const void* const* phi, const double* m1,
                       const double* m2, double beta, double tau, int nsteps, int integrator, int n_inner,
                       const odwf_solve_params* params, double* energies, odwf_solve_stats* stats,
                       void* stream);

/*
 * Time one kernel of the production mixed-precision iteration on its own: kind 1..4 = the
 * hops K1..K4 (see odwf_mixed_cg_step; K1 is the plain Dslash chi_t = B M^-1 (-1/2 W chi_p)),
 * 5 = the p update.  nsys systems (1..64) share the handle's links; every input field of every
 * system is filled from `fill` (an even-site field, host or device; any finite values) and
 * every system runs.  After one warm-up launch, `reps` launches are timed with two CUDA events
 * on `stream`; out receives the kernel class name, the launch counts, the total time and the
 * algorithmic bytes (each field read or written once per system, links once per launch).
 * Results are meaningful as bandwidth when one system's fields exceed the L2 cache.
 * Allocates its workspaces on the handle (freed by odwf_destroy).
 */
int odwf_time_kernel(odwf_handle* h, int kind, int prec, int link_recon, int link_prec, int nsys, int reps,
                     const void* fill, odwf_kernel_prof* out, void* stream);

/* Number of kernel launches the library has issued in this process (all kernels). */
long long odwf_launch_count(void);

/* ----------------------------------------------------------------------------------
 * Serving: a request loop that keeps gauge fields resident, admits solve requests by
 * an HBM budget into per-(field, Ns, m0, weights) batches, and solves them with
 * continuous batching (requests join a running batch between iterations as slots and
 * memory free up; batches of different fields run concurrently on separate streams).
 * ---------------------------------------------------------------------------------- */
typedef struct serve_handle serve_handle;

typedef struct {
    int32_t field_id;     /* a field registered with serve_register_gauge */
    int32_t Ns;
    double m0;
    double mq;
    const double* omega;  /* host, Ns doubles; copied at submit */
    int32_t nrhs;
    const void* const* b; /* nrhs host or device pointers, SCHUR_EVEN layout; a device b is
                             read again during the solve and must stay valid (and unchanged)
                             until the request completes; host data is copied at admission */
    void* const* x;       /* nrhs output pointers, same kind as b, written at completion */
    double tol;
    int32_t prec;         /* inner precision, as odwf_solve_params.prec */
    int32_t max_iter;
} odwf_request;

typedef struct {
    int32_t status;       /* ODWF_OK, ODWF_PENDING, or an error code */
    int32_t iters;        /* largest inner iteration count over the request's systems */
    double true_resid;    /* largest final true relative residual over its systems */
    double latency_ms;    /* submit -> completion */
    double queue_ms;      /* submit -> admission */
} odwf_result;

/* Create a server with a device-memory budget in bytes (0 = 90% of free memory). */
int serve_create(size_t hbm_budget_bytes, serve_handle** out);

/* Register (upload and pack) a resident gauge field under field_id. U host or device. */
int serve_register_gauge(serve_handle* s, int field_id, const odwf_lattice* lat, const void* U);

/* Queue a request; *ticket identifies it.  ODWF_ENOMEM if it can never fit the budget. */
int serve_submit(serve_handle* s, const odwf_request* req, uint64_t* ticket);

/*
 * Wait up to timeout_ms (0 = just look) for the request.  Returns ODWF_PENDING while it
 * is queued or running, otherwise its final status; res (may be NULL) gets the details.
 * A finished ticket can be polled again until serve_destroy.
 */
int serve_poll(serve_handle* s, uint64_t ticket, int timeout_ms, odwf_result* res);

/*
 * Admission and scheduling policy.  admit_deadline_ms > 0: a request still waiting for admission
 * after that long is shed, completing with ODWF_ETIMEOUT (its x is not written).  max_queued > 0:
 * at most that many requests wait; serve_submit then answers ODWF_EBUSY and takes no ticket.
 * Values <= 0 disable either (the default).  fair = 0 (default): batches of smaller lattices
 * get higher stream priorities (short requests finish first); fair = 1: every batch created
 * from now on runs at the same priority, so batches share the GPU in proportion to their work.
 * Applies to requests already queued from the next loop pass.
 */
int serve_set_policy(serve_handle* s, double admit_deadline_ms, int max_queued, int fair);

/*
 * Cancel a request.  A queued request completes at once with ODWF_ECANCELED; a running one
 * stops between two chunks of iterations (its systems' slots are freed, x is not written) and
 * then completes with ODWF_ECANCELED.  A finished request keeps its status.  ODWF_ENOTFOUND
 * for an unknown ticket.
 */
int serve_cancel(serve_handle* s, uint64_t ticket);

/*
 * Stop the loop after the running work, fail queued requests (ODWF_ETIMEOUT), finish pending
 * copies of results to host buffers, free everything.  Any CUDA or solver error inside a batch
 * fails every request with systems in that batch with the error's status (e.g. ODWF_ECUDA) and
 * frees the batch; other batches continue.
 */
int serve_destroy(serve_handle* s);

#ifdef __cplusplus
}
#endif

#endif /* ODWF_H */
