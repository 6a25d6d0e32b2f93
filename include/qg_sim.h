/*
 * qg_sim.h -- time integration on the GPU: the leapfrog integrator the paper
 * pairs with its tree code (Kodama & Ishiyama, arXiv:1812.07313, Sec. 5, the
 * cold-collapse runs: G = M = 1, fixed step Delta t), with every force
 * evaluation done by the GPU tree build, group walk and force kernel
 * (qg_gtree.h, qgrav.h).  State stays in device memory between steps.
 *
 * One step of length dt is kick-drift-kick:
 *     v += a(x) dt/2;   x += v dt;   a, phi = forces(x);   v += a dt/2
 * where forces(x) rebuilds the oct-tree, the sink groups and the
 * interaction lists from the current positions and evaluates Eq. 1 / Eq. 7
 * (quadrupole cells, or monopole-only cells) on them.
 *
 * Particles keep the caller's order (the tree's sorted order is internal).
 * Softening: params->eps2 for every particle, or a per-particle eps^2 given
 * with the state (each sink's own softening, as the force path's per-sink
 * eps2; e.g. one value per independent system).
 * Energies: K = 1/2 sum m v^2 and W = 1/2 sum m (phi + m / eps) -- the
 * self pair that the force path includes in phi (-m/eps for eps > 0) is
 * taken out again; with eps = 0 there is no self term.
 *
 * Streams: every step of a call runs on the given cuda_stream, or on the
 * simulation's own stream when it is NULL; calls that return results to the
 * host synchronise that stream.
 *
 * Every call returns a qg_status (QG_OK, QG_ERR_ARG, QG_ERR_CUDA,
 * QG_ERR_NOMEM, QG_ERR_STATE) and leaves the simulation valid; host arrays
 * are copied before returning and stay the caller's.  A step that fails
 * after the drift leaves the state without matching forces: further steps
 * return QG_ERR_STATE until qg_sim_set_state.
 */
#ifndef QG_SIM_H
#define QG_SIM_H

#include <stdint.h>

#include "qgrav.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qg_sim qg_sim;

typedef struct {
  double theta;   /* opening angle of the group walk (> 0) */
  double eps2;    /* Plummer softening squared, every particle */
  int n_crit;     /* sink group size bound (>= 1) */
  int leaf_max;   /* tree leaf size bound (>= 1) */
  int expansion;  /* QG_QUAD or QG_MONO */
  int autotune;   /* nonzero: qg_autotune the force launch on the first force
                     evaluation; afterwards, whenever the step's list entries
                     differ from those it was last tuned on by more than a
                     quarter, an online trial: each of the next (at most 6)
                     force evaluations runs one launch shape near the current
                     one (2, 4 or 8 warps per CTA; at 4 sinks per thread, fixed
                     or chosen per work item), timed by its own force kernel,
                     and the fastest is kept.  A trial adds no evaluations. */
} qg_sim_params;

/* Device time (CUDA events) of the parts of the last step, milliseconds,
 * and its wall-clock time (host clock, the step's own synchronisations
 * included). */
typedef struct {
  float build_ms, walk_ms, force_ms, integrate_ms;
  double wall_ms;
  int64_t groups, n_plist, n_clist, i_pp, i_pc;
  int64_t retunes;  /* force-launch tunings so far (autotune): the first
                       qg_autotune and every online trial started since */
  /* the force launch of the last step (qg_stats): sinks per thread (and 1
   * if chosen per item), warps per CTA, tile, FP32 form; trial_left: force
   * evaluations still to run in the current online trial (0 = none) */
  int32_t sinks_per_thread, sinks_adaptive, warps_per_group, tile_j, form, trial_left;
} qg_sim_times;

/* A simulation with the parameters of Sec. 5's runs (theta, eps, n_crit,
 * monopole or quadrupole cells).  force_opt may be NULL (defaults); its
 * expansion field is overridden by params->expansion. */
qg_status qg_sim_create(qg_sim **out, int device, const qg_sim_params *params, const qg_options *force_opt);
void qg_sim_destroy(qg_sim *sim);

/*
 * The initial conditions of a run (Sec. 5: a cold homogeneous sphere).
 * Initial state from HOST arrays x [n][3], v [n][3], m [n] (n < 2^31) and
 * sys_off [nsys+1] (independent systems, each with its own tree root;
 * sys_off = {0, n} for one system).  eps2 [n] (host, may be NULL): each
 * particle's squared softening, finite and >= 0, used instead of
 * params->eps2.  Evaluates the forces at x, so that the first step can kick.
 */
qg_status qg_sim_set_state(qg_sim *sim, int64_t n, const double *x, const double *v, const double *m,
                           const float *eps2, int64_t nsys, const int64_t *sys_off, void *cuda_stream);

/* The leapfrog of Sec. 5 with its fixed step: nsteps kick-drift-kick steps
 * of length dt (nsteps >= 0, dt finite). */
qg_status qg_sim_step(qg_sim *sim, double dt, int64_t nsteps, void *cuda_stream);

/* The particle data of List 4's particle class (positions, velocities and
 * the accelerations and potentials of the last force evaluation): copy the
 * state to HOST arrays (any pointer may be NULL); synchronises. */
qg_status qg_sim_get_state(qg_sim *sim, double *x, double *v, double *a, double *phi);

/* As qg_sim_get_state, on the device.
 * Device pointers to the state (the simulation owns them; valid until the
 * next qg_sim_set_state or qg_sim_destroy; any pointer may be NULL). */
qg_status qg_sim_state_dev(const qg_sim *sim, const double **x, const double **v, const double **a,
                           const double **phi, const double **m);

/* The energies that check a run (Sec. 5's cold collapse starts at virial
 * ratio 0.1): kinetic and potential energy, and total momentum p [3] (may be
 * NULL), of the current state: FP64 reductions on the device in a fixed
 * order. */
qg_status qg_sim_energy(qg_sim *sim, double *kinetic, double *potential, double *momentum, void *cuda_stream);

/* Seconds per step, the quantity the paper reports for its runs (Sec. 5),
 * split into its parts. */
qg_status qg_sim_last_times(const qg_sim *sim, qg_sim_times *out);

#ifdef __cplusplus
}
#endif
#endif
