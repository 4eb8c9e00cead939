/*
 * odwf_flow.h -- C ABI of the gradient (Wilson) flow and the flow observables.
 *
 * The paper sets its lattice scale with the flow condition t^2 <E(t)> = 0.3 at t = t0 (Sec. 2)
 * and measures the topological charge on flowed fields (Sec. 3): the clover charge
 *
 *   Q_clover = sum_x eps_{mu nu rho sigma} tr[F_{mu nu}(x) F_{rho sigma}(x)] / (32 pi^2),
 *
 * F_{mu nu}(x) the field strength built from the four plaquettes around x in the (mu, nu) plane,
 * trusted once every plaquette satisfies Re tr U_plaq / 3 > 44/45 (Sec. 3, the admissibility
 * bound), after integrating the flow from t = 0 to t = 64 in steps of 0.01.
 *
 * Definitions used here (lattice spacing 1, mu = 0..3 <-> x, y, z, t):
 *   flow       dV/dt = Z(V) V with Z_mu(x) = -ta(U_mu(x) S_mu(x)), S_mu the sum of the six
 *              staples of the link and ta(X) = (X - X^+)/2 - tr(X - X^+)/6; i.e. the gradient
 *              flow of the Wilson plaquette action.  One step of size eps is the three-stage
 *              third-order Runge-Kutta scheme of Luscher (JHEP 2010) for this equation (the paper
 *              gives the step, 0.01, but not the integrator).
 *   F          (Q - Q^+)/(8i), made traceless, Q the sum of the four plaquette loops at x.
 *   E(x)       e_clover: sum_{mu<nu} tr F_{mu nu}(x)^2;  e_plaq: 2 sum_{mu<nu} Re tr(1 - P_{mu nu}(x)).
 *
 * Precision: the links are held as pairs of FP32 numbers (hi + lo, about 48 significant bits)
 * of their first two rows; the third row of an SU(3) matrix is conj(row0 x row1) and is rebuilt
 * where it is needed.  The force, the exponential and the observables are computed in FP32 and
 * every lattice sum is accumulated in FP64.  A flow of n steps agrees with an FP64 integration to
 * within n * eps * max|Z| * 64 * 2^-24 in each link entry (FP32 rounding of the force and of the
 * stage increments).
 *
 * Conventions as in odwf.h: the gauge field is complex128 U[mu][t][z][y][x][a][b]; pointers may
 * be host or device memory (the library detects which); calls that return observables to the
 * host synchronise `stream`; errors are int statuses with odwf_last_error() for the message.
 * Calls on one flow object must not overlap.  The object's kernels run on the GPU that was
 * current at odwf_flow_create, which must also be current at every later call.
 */
#ifndef ODWF_FLOW_H
#define ODWF_FLOW_H

#include <stdint.h>

#include "odwf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct odwf_flow odwf_flow;

/* One measurement on the field at flow time t. */
typedef struct {
    double t;          /* flow time */
    double e_plaq;     /* site average of 2 sum_{mu<nu} Re tr(1 - P_{mu nu}(x)) */
    double e_clover;   /* site average of sum_{mu<nu} tr F_{mu nu}(x)^2 */
    double q_clover;   /* clover topological charge (sum over sites) */
    double plaq_min;   /* min over all plaquettes of Re tr P / 3 (admissible when > 44/45) */
    double plaq_mean;  /* average over all plaquettes of Re tr P / 3 */
} odwf_flow_obs;

/*
 * Create a flow object for a periodic lattice dims = {Lx, Ly, Lz, Lt}, every extent >= 2 (no
 * parity requirement).  Allocates its device memory at once: 1088 bytes per site (two buffers of
 * float-float links, the six plaquette projections and the Runge-Kutta carry) plus per-block
 * partial sums.  ODWF_EINVAL on bad sizes, ODWF_ENOMEM when the allocation fails.
 */
int odwf_flow_create(const int32_t dims[4], odwf_flow** out);

/* Free the object and its device memory. */
int odwf_flow_destroy(odwf_flow* f);

/* Load the gauge field U (host or device, complex128, V * 36 entries) as the flow's field at t = 0.
 * U must be in SU(3): the third row of each link is not read but rebuilt from the first two.  With
 * a host U the copy goes through a device staging buffer of one direction (V * 144 bytes) that the
 * object keeps until odwf_flow_destroy; the call returns once U may be reused. */
int odwf_flow_set_gauge(odwf_flow* f, const void* U, void* stream);

/* Write the current (flowed) field to U (host or device, complex128, layout above). */
int odwf_flow_get_gauge(odwf_flow* f, void* U, void* stream);

/*
 * Measure the current field; obs->t is set to t.  obs is host memory.  e_site and q_site (each
 * V floats, lexicographic sites, host or device, or NULL) receive the per-site energy density
 * (clover) and charge density.  Synchronises `stream`.
 */
int odwf_flow_measure(odwf_flow* f, double t, odwf_flow_obs* obs, float* e_site, float* q_site, void* stream);

/*
 * Integrate nsteps steps of size eps (> 0) from flow time t_start.  With measure_every > 0 the
 * field is measured at t_start and after every measure_every steps (the measurement reuses the
 * plaquettes of the next step's first stage); the records go to obs[0 .. *n_obs) (host memory,
 * at most max_obs; ODWF_EINVAL before any work when more would be needed: that is
 * (nsteps - 1) / measure_every + 1, plus one when measure_every divides nsteps).
 * Synchronises `stream` when it measures; otherwise stream-ordered.
 */
int odwf_flow_run(odwf_flow* f, double eps, int nsteps, int measure_every, double t_start, odwf_flow_obs* obs,
                  int max_obs, int* n_obs, void* stream);

/*
 * Host only: the first flow time where t^2 e_clover(t) reaches `target` (0.3 for t0, Sec. 2),
 * by linear interpolation in t between the two measurements around the crossing.  Returns
 * ODWF_ENOTFOUND when no crossing occurs in obs[0 .. n).
 */
int odwf_flow_t0(const odwf_flow_obs* obs, int n, double target, double* t0);

#ifdef __cplusplus
}
#endif

#endif
