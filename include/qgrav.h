/*
 * qgrav.h -- C-ABI of the GB300 (sm_103a) monopole + quadrupole tree-force
 * hot path.
 *
 * What it computes (Kodama & Ishiyama, arXiv:1812.07313):
 *   For every sink group g (the particles of one tree cell with at most
 *   n_crit particles, Sec. 3.4 "modified tree algorithm"), every sink i of g
 *   receives from the group's shared interaction list
 *     - each listed source particle p, a Plummer-softened point mass:
 *         phi_i -= m_p / rhat,  a_i += m_p r_ip / rhat^3          (Eq. 4)
 *     - each listed cell c (mass m_c at its centre of mass, quadrupole Q_c):
 *         phi_mono = m_c / rhat,  phi_quad = r.Q_c.r / (2 rhat^5)  (Eqs. 4-5)
 *         phi_i   -= phi_mono + phi_quad                            (Eq. 1)
 *         a_i     += (phi_mono + 5 phi_quad) / rhat^2 r - Q_c r / rhat^5
 *   with r = r_j - r_i and rhat^2 = |r|^2 + eps_i^2.  The acceleration is
 *   -grad of Eq. 1 (Eq. 6); the leading minus sign printed in Eq. 7 is a
 *   typesetting slip (it would make gravity repulsive) and is not applied.
 *   G = 1: masses carry G.  phi is the physical (negative) potential.
 *   A pair with rhat^2 == 0 exactly (zero softening, coincident points)
 *   contributes nothing.  The group's own particles are usually in its own
 *   particle list: with eps > 0 each such self pair adds -m/eps to phi and no
 *   force.
 *
 * Precision (QG_FP32_CENTRED, the default): positions are kept in FP64; on
 * the GPU each group's centre c_g (centre of the bounding box of its sinks)
 * is subtracted in FP64 from every sink and every staged list entry, and only
 * then is the offset cast to FP32.  The pairwise arithmetic is FP32 with the
 * SFU reciprocal square root; each thread's FP32 partial sums are folded,
 * after a bounded number of list entries, into float-float sums (an FP32
 * hi + lo pair, about 48 significant bits; FP64 sums in the sink-paired
 * form), and the partials of all threads of a group are merged the same way
 * in a fixed order and converted to FP64.  QG_FP32_RAW skips the centring
 * (absolute coordinates cast to FP32; an ablation).  QG_FP64 does everything
 * in FP64 (a comparison kernel, about 70x slower on this GPU).
 *
 * Expansion: QG_QUAD evaluates cells with Eq. 1; QG_MONO treats every cell
 * as a point mass at its centre of mass and ignores Q (the monopole-only
 * tree code the paper compares against).
 *
 * Memory and ownership.  Host-pointer calls (qg_set_sinks, qg_set_sources,
 * qg_set_cells, qg_get_forces) copy synchronously; the caller keeps its
 * arrays.  The *_dev variants take device pointers (e.g. torch tensor
 * storage) on the context's device, read them on the given stream before
 * returning, and do not keep them.  All arrays are row-major and densely
 * packed.  Index arrays are int32; offsets are int64.
 *
 * Errors.  Every call returns a qg_status; nothing aborts, throws or exits
 * across the ABI.  A call that fails leaves the previously set inputs in
 * place but marks the context not runnable until the failing input is set
 * again successfully; qg_last_error() returns a message for the last error.
 * Out-of-range offsets or indices are rejected (QG_ERR_ARG) before any
 * force kernel reads them: offsets on the host, list indices by a checking
 * kernel on the device copy.  qg_run is asynchronous: a CUDA error from it surfaces as
 * QG_ERR_CUDA from qg_run or from the next synchronising call.
 *
 * Threading.  A context is used by one host thread at a time.
 *
 * Correspondence with the paper's library (Sec. 3.4, Lists 3 and 4).  The
 * paper's tree code calls its force library once per group: g5_open and
 * g5_set_eps_to_all once, then per group g5_set_xmjMC / g5_set_nMC /
 * g5_calculate_force_on_xMC for the particle part of the list and
 * g5c_set_xmjMC / g5c_set_nMC / g5c_calculate_force_on_xMC for the cell part.
 * Here every group of a step is set at once (sinks, per-group lists as CSR
 * offsets) and evaluated in one call; each declaration below names the
 * paper's call or passage it stands for.
 */
#ifndef QGRAV_H
#define QGRAV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qg_ctx qg_ctx;

typedef enum {
  QG_OK = 0,
  QG_ERR_ARG = -1,     /* bad argument, size or index                      */
  QG_ERR_CUDA = -2,    /* a CUDA call failed                               */
  QG_ERR_NOMEM = -3,   /* device or host allocation failed                 */
  QG_ERR_STATE = -4,   /* inputs missing or inconsistent (e.g. ngroups)    */
  QG_ERR_TIMEOUT = -5, /* reserved: no call returns it (no kernel of this
                          library waits on another kernel or on the host) */
  QG_ERR_SIZE = -6     /* a size beyond a fixed maximum (qg_forces_noalloc) */
} qg_status;

enum { QG_FP32_CENTRED = 0, QG_FP32_RAW = 1, QG_FP64 = 2 };
enum { QG_QUAD = 0, QG_MONO = 1 };
enum { QG_ARITH_DEFAULT = 0, QG_ARITH_SCALAR = 1, QG_ARITH_PAIRED = 2, QG_ARITH_ENTRY_PAIRED = 3 };

/*
 * Options of a context.  A 0 in tile_j, warps_per_group, sinks_per_thread,
 * flush_j or arith selects a FIXED default, not a tuned one: tile 256, 4
 * sinks per thread, fold every 256 entries, and for QG_FP32_CENTRED the
 * entry-paired form with 2 warps (with 8 sinks per thread, and for the other
 * precisions, the scalar form with 4 warps) -- the shape the autotuner picks
 * on most of the workloads measured.  The tuning call is qg_autotune, which
 * times the supported shapes on the inputs set and stores the fastest in the
 * context.  The paper has no counterpart (its
 * kernel has one fixed shape, 4 i-particles x 2 j-cells per AVX2 iteration,
 * List 2); precision and expansion select the variants compared in Secs. 4-5.
 */
typedef struct {
  int precision;        /* QG_FP32_CENTRED | QG_FP32_RAW | QG_FP64          */
  int expansion;        /* QG_QUAD | QG_MONO                                 */
  int tile_j;           /* list entries staged per shared-memory tile;
                           0 = default (256); else 32..1024, multiple of 32 */
  int warps_per_group;  /* warps of the CTA that evaluates one group;
                           0 = default; supported: 1, 2, 4, 8               */
  int sinks_per_thread; /* sinks held in registers per thread;
                           0 = default; supported: 2, 4, 8                  */
  int flush_j;          /* FP32 partials are folded into the float-float
                           (or FP64) sums after at most this many list
                           entries per thread; 0 = 256                      */
  int arith;            /* QG_FP32_CENTRED only: QG_ARITH_SCALAR,
                           QG_ARITH_PAIRED (two sinks per float2 register,
                           f32x2 FMA instructions) or QG_ARITH_ENTRY_PAIRED
                           (two list entries per float2 register;
                           sinks_per_thread 2 or 4; the default, 0, up to 4
                           sinks per thread)                                 */
  int split_j;          /* long lists cut into work items (Sec. 3.4's group x
                           list, split for load balance): 0 = never (the
                           default); k > 0 = every list of more than k
                           entries is cut into parts of about k entries
                           (at most 64 parts); -1 = automatic: a group whose
                           FP32 work exceeds a quarter of one CTA's average
                           share of the step is cut into parts of about an
                           eighth of it.  Each part writes FP64 partial sums
                           per sink; the part that completes a group adds
                           them in a fixed order (bitwise repeatable).
                           qg_evaluate_host never splits.                   */
  int sinks_adaptive;   /* QG_FP32_CENTRED, scalar or entry-paired form: 1 =
                           every work item runs at the number of sinks per
                           thread from 1 to 4 that suits its group's size and
                           list length (sinks_per_thread then 0 or 4); 0 =
                           sinks_per_thread for every item (the default)   */
} qg_options;

typedef struct {
  int64_t n_sinks, n_groups, n_sources, n_cells;
  int64_t n_plist, n_clist;   /* total particle / cell list entries          */
  int64_t i_pp, i_pc;         /* particle-particle / particle-cell pairs     */
  int32_t grid, block;        /* launch shape of the force kernel            */
  int32_t sinks_per_thread;   /* the kernel variant chosen                   */
  int32_t tile_j;
  int32_t warps_per_group;
  int32_t flush_j;
  int32_t paired;             /* FP32 form: 0 scalar, 1 sink-paired,
                                 2 entry-paired                              */
  int32_t eval_in_place;      /* 1 if the last qg_evaluate_host read the
                                 lists and wrote the results in place       */
  int64_t n_items;            /* work items of the last qg_run's queue (the
                                 groups, or groups and parts of split lists) */
  int64_t n_split;            /* groups whose lists were split               */
  int32_t sinks_adaptive;     /* 1 if sinks per thread are chosen per item   */
  int32_t reserved;
} qg_stats;

/* Create a context on CUDA device `device`.  opt may be NULL (defaults).
 * Stands for g5_open (List 4); `device` replaces the paper's devid. */
qg_status qg_create(qg_ctx **out, int device, const qg_options *opt);
/* Release the context and its device memory.  Stands for g5_close (List 4). */
void qg_destroy(qg_ctx *ctx);
/* Change the options (see qg_options); the next qg_run uses them. */
qg_status qg_set_options(qg_ctx *ctx, const qg_options *opt);

/*
 * The i-particles of every group (Sec. 3.4: the particles of a cell with at
 * most n_crit particles share one interaction list; List 4's ilist holds
 * their positions xi and count ni) and their softening (g5_set_eps_to_all in
 * List 4 sets one eps for all; the i-particle structure of List 2 carries
 * eps^2 per i-particle, hence the optional per-sink array).
 * Sinks, grouped: group g owns sinks [group_off[g], group_off[g+1]).
 * x: [n][3] positions.  eps2: [n] per-sink squared softening (Phantom-GRAPE
 * keeps eps^2 per i-particle) or NULL to use eps2_all for every sink.
 * group_off: [ngroups+1], group_off[0] = 0, non-decreasing, last = n.
 */
qg_status qg_set_sinks(qg_ctx *ctx, int64_t n, const double *x, const float *eps2,
                       double eps2_all, int64_t ngroups, const int64_t *group_off);

/*
 * The j-particles of every group's list: what List 4 passes per group to
 * g5_set_xmjMC (positions xj, masses mj) and g5_set_nMC (their number),
 * evaluated as Plummer-softened point masses (the monopole term of Eq. 1).
 * Source particles and the particle part of every group's list.
 * x: [ns][3], m: [ns].  list_off: [ngroups+1] (same ngroups as the sinks),
 * list_off[0] = 0, non-decreasing; list_idx: [list_off[ngroups]] entries,
 * each in [0, ns).
 */
qg_status qg_set_sources(qg_ctx *ctx, int64_t ns, const double *x, const double *m,
                         const int64_t *list_off, const int32_t *list_idx);

/*
 * The j-cells of every group's list: what List 3's g5c_set_xmjMC (centres
 * of mass xj, masses mj, quadrupole tensors qj[6], Eq. 2) and g5c_set_nMC
 * (their number) pass per group, and the paper stores as floats in its
 * j-cell structure (List 1).
 * Tree cells and the cell part of every group's list.
 * com: [nc][3] centres of mass, m: [nc] masses, q: [nc][6] quadrupole
 * tensors about the centre of mass, q00 q01 q02 q11 q12 q22, unhalved as in
 * Eq. 2 (the 1/2 of Eq. 5 is applied by the kernel).  q22 is used as given
 * (not recomputed from the trace condition, as in the paper).
 * list_off / list_idx as for qg_set_sources, entries in [0, nc).
 */
qg_status qg_set_cells(qg_ctx *ctx, int64_t nc, const double *com, const double *m,
                       const double *q, const int64_t *list_off, const int32_t *list_idx);

/* Device-pointer variants (same layouts), read on `cuda_stream` (NULL = the
 * context's stream) before they return. */
qg_status qg_set_sinks_dev(qg_ctx *ctx, int64_t n, const double *x, const float *eps2,
                           double eps2_all, int64_t ngroups, const int64_t *group_off,
                           void *cuda_stream);
qg_status qg_set_sources_dev(qg_ctx *ctx, int64_t ns, const double *x, const double *m,
                             const int64_t *list_off, const int32_t *list_idx,
                             int64_t n_list, void *cuda_stream);
qg_status qg_set_cells_dev(qg_ctx *ctx, int64_t nc, const double *com, const double *m,
                           const double *q, const int64_t *list_off, const int32_t *list_idx,
                           int64_t n_list, void *cuda_stream);

/*
 * The force calls of every group at once: g5_calculate_force_on_xMC (the
 * j-particles) and g5c_calculate_force_on_xMC (the j-cells, Eqs. 1, 4-7) of
 * List 3 and the group loop of calc_force in List 4, accumulated into one
 * acceleration and potential per sink.
 * One evaluation of every group: work-queue build (groups ordered by
 * descending cost), then one persistent launch over all groups.  The
 * sequence is captured once in a CUDA graph and replayed.  Asynchronous on
 * `cuda_stream` (NULL = the context's stream).
 */
qg_status qg_run(qg_ctx *ctx, void *cuda_stream);

/*
 * No counterpart in the paper (its kernel has one fixed shape, List 2).
 * Autotuner: times every supported launch shape (sinks_per_thread x
 * warps_per_group x tile_j, in the scalar and the entry-paired FP32 forms for
 * QG_FP32_CENTRED, each at 4 sinks per thread also with sinks_adaptive) of
 * the current precision / expansion on the inputs
 * currently set -- each shape once (the force kernel's device time, CUDA
 * events), then the four fastest again with one warm-up and `reps` timed
 * runs each -- and keeps the fastest as the context's options.  The
 * sink-paired form (QG_ARITH_PAIRED) is not tried: it was slower at every
 * shape measured; it stays selectable through qg_options.  The sink grouping itself (n_crit) is an input and is
 * not tuned here.  best (may be NULL) receives the chosen options,
 * best_ms the chosen shape's mean force-kernel time.  Synchronous; the
 * outputs afterwards hold a valid result of the chosen shape.
 */
qg_status qg_autotune(qg_ctx *ctx, void *cuda_stream, int reps, qg_options *best, float *best_ms);

/* The results, as the arrays ai and pi that List 3's force call fills (the
 * kernel's output structure in List 2 holds ax, ay, az and phi): a [n][3]
 * and phi [n] (either may be NULL) copied to the host; synchronises.  phi is
 * the physical potential of Eq. 1 (negative), a = -grad phi (Eq. 6). */
qg_status qg_get_forces(qg_ctx *ctx, double *a, double *phi);

/* As qg_get_forces: device-to-device copy of the results into caller
 * buffers on `cuda_stream`. */
qg_status qg_get_forces_dev(qg_ctx *ctx, double *a, double *phi, void *cuda_stream);

/*
 * The force part of List 4's calc_force in one call (every group's
 * j-particle and j-cell calls, Lists 3 and 4), from host arrays as the
 * paper's library takes them.
 * One evaluation from HOST arrays: the inputs of qg_set_sinks, qg_set_sources
 * and qg_set_cells (same meaning, layout and checks), then the forces written
 * to a [n][3] and phi [n] (host).  The offsets, then the sinks and
 * sources, then the cells are copied first, in that order (one copy of x
 * when src_x is the same array as sink_x and ns == n); each set-up kernel
 * (work queue, group centres, packing) starts once the copies it reads
 * are done.  The lists then take one of two routes:
 *   - in place, when plist_idx, clist_idx, a and phi are all page-locked
 *     (cudaHostAlloc / cudaHostRegister), the GPU reads host memory
 *     through the host's page tables (a coherent CPU-GPU link, as on
 *     Grace-Blackwell) and the options select the FP32 centred precision in
 *     the scalar or entry-paired form: one persistent force launch reads every list index
 *     from host memory, checks it and keeps it in the context's device
 *     lists, and writes the results to the device and to a / phi; nothing
 *     is copied back;
 *   - otherwise copied in four chunks of groups while the force kernel runs
 *     over the chunks already there, each chunk's results copied back as
 *     soon as its kernel ends.
 * qg_stats.eval_in_place tells which.  Either way the results are bit for
 * bit those of the separate calls at the same options, and afterwards the
 * context holds these inputs and results (qg_run, qg_get_forces,
 * qg_autotune, qg_last_timing work on them).  Synchronous.  A list entry
 * outside [0, ns) or [0, nc) gives QG_ERR_ARG; the kernel reads entry 0 in
 * its place, so nothing is read out of bounds.
 */
qg_status qg_evaluate_host(qg_ctx *ctx, int64_t n, const double *sink_x, const float *sink_eps2, double eps2_all,
                           int64_t ngroups, const int64_t *group_off, int64_t ns, const double *src_x,
                           const double *src_m, const int64_t *plist_off, const int32_t *plist_idx, int64_t nc,
                           const double *cell_com, const double *cell_m, const double *cell_q,
                           const int64_t *clist_off, const int32_t *clist_idx, double *a, double *phi);

/* Sizes, launch shape and interaction counts of the inputs set.  The paper
 * reports cell interactions per second (Sec. 5.2, Fig. 4); i_pc counts those
 * pairs and i_pp the particle pairs. */
qg_status qg_get_stats(const qg_ctx *ctx, qg_stats *out);

/*
 * The force time of a step (T_force of Table 3, Sec. 5.1).
 * Device time of the last qg_run, from CUDA events recorded inside its
 * graph: step_ms = whole step (work-queue build + force kernel), force_ms =
 * the persistent force kernel alone.  Synchronises the run's stream.
 * Either pointer may be NULL.
 */
qg_status qg_last_timing(qg_ctx *ctx, float *step_ms, float *force_ms);
/* Message of the last failing call on this context (no counterpart in the
 * paper's library, whose calls return nothing). */
const char *qg_last_error(const qg_ctx *ctx);

/*
 * Direct summation on the GPU (the reference of the paper's force-error
 * measure, Eq. 8): every source acts on every sink as a Plummer point mass,
 * all in FP64.  Device pointers: sink_x [nsink][3], src_x [nsrc][3],
 * src_m [nsrc], outputs a [nsink][3], phi [nsink].  Pairs with rhat^2 == 0
 * are skipped.  Synchronous.  Used to measure the method's own error; it is
 * not part of the timed force step.
 */
qg_status qg_direct_dev(int device, int64_t nsink, const double *sink_x, double eps2,
                        int64_t nsrc, const double *src_x, const double *src_m,
                        double *a, double *phi, void *cuda_stream);

/*
 * The double -> float conversion that the paper's g5c_set_xmjMC applies when
 * it stores j-cells as floats (Sec. 3.4, List 1); here it is applied to
 * positions after the FP64 group centring.
 * Self-test of the rounding the FP32 kernels apply to FP64-centred offsets:
 * double -> float, nearest with ties to even, done with integer operations
 * (IEEE 754 binary64 -> binary32).  Magnitudes below the smallest normal
 * float give a signed zero.  qg_round_f32_host runs it on the CPU (host
 * arrays); qg_round_f32_dev runs it on the GPU (device arrays) and writes
 * the hardware conversion of the same inputs to out_hw for comparison.
 */
qg_status qg_round_f32_host(int64_t n, const double *in, float *out);
qg_status qg_round_f32_dev(int64_t n, const double *in, float *out, float *out_hw, void *cuda_stream);

/*
 * One force evaluation that allocates no memory, host or device.  The paper
 * has no counterpart: this is an entry point for callers that cannot call
 * cudaMalloc -- host codes whose device memory belongs to their own pool or
 * arena, and time-stepping loops that may not allocate (cudaMalloc and
 * cudaFree can block or synchronise the device) once they are running.
 *
 * Every input and output is a caller-owned device array on `device`, in the
 * layouts of qg_set_sinks_dev / qg_set_sources_dev / qg_set_cells_dev;
 * a [n][3] and phi [n] receive the result (FP32 pairwise arithmetic with FP64
 * centring and merges, QG_QUAD or QG_MONO as `expansion`; a fixed launch
 * shape).  The step's only scratch, its work queue, lives in one fixed
 * device array inside this library, sized for ngroups <= QG_NOALLOC_MAX_GROUPS
 * (about 5 MiB, held by every GPU that loads the library until the process
 * exits); a larger ngroups returns QG_ERR_SIZE before any GPU work.  Offsets
 * and list indices are checked on the GPU first (QG_ERR_ARG if invalid);
 * n_plist / n_clist are the list lengths, and every array must be at least
 * as long as the sizes say.
 *
 * All calls on a device share that scratch array and it keeps the last
 * call's contents (each call clears what it needs zeroed): calls whose work
 * overlaps on the GPU -- on different streams, or from racing host threads
 * -- corrupt each other.  The first call on a device looks up the array's
 * device address and caches it.  The call waits for the argument check on
 * `cuda_stream` (a device-to-host copy and a stream synchronisation), then
 * launches the step and returns; a and phi are complete when the stream
 * reaches that point.
 */
#define QG_NOALLOC_MAX_GROUPS (1 << 20)
qg_status qg_forces_noalloc(int device, int64_t n, const double *sink_x, const float *sink_eps2,
                            double eps2_all, int64_t ngroups, const int64_t *group_off,
                            int64_t ns, const double *src_x, const double *src_m,
                            const int64_t *plist_off, const int32_t *plist_idx, int64_t n_plist,
                            int64_t nc, const double *cell_com, const double *cell_m,
                            const double *cell_q, const int64_t *clist_off,
                            const int32_t *clist_idx, int64_t n_clist, int expansion,
                            double *a, double *phi, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
