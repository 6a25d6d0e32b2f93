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
 * SFU reciprocal square root; each thread's FP32 partial sums are folded into
 * FP64 after a bounded number of list entries, and the partials of all
 * threads of a group are merged in FP64.  QG_FP32_RAW skips the centring
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
  QG_ERR_TIMEOUT = -5, /* a bounded device-side wait gave up               */
  QG_ERR_SIZE = -6     /* a size beyond a fixed maximum (qg_forces_noalloc) */
} qg_status;

enum { QG_FP32_CENTRED = 0, QG_FP32_RAW = 1, QG_FP64 = 2 };
enum { QG_QUAD = 0, QG_MONO = 1 };
enum { QG_ARITH_DEFAULT = 0, QG_ARITH_SCALAR = 1, QG_ARITH_PAIRED = 2 };

typedef struct {
  int precision;        /* QG_FP32_CENTRED | QG_FP32_RAW | QG_FP64          */
  int expansion;        /* QG_QUAD | QG_MONO                                 */
  int tile_j;           /* list entries staged per shared-memory tile;
                           0 = default (256); else 32..1024, multiple of 32 */
  int warps_per_group;  /* warps of the CTA that evaluates one group;
                           0 = default; supported: 2, 4, 8                  */
  int sinks_per_thread; /* sinks held in registers per thread;
                           0 = default; supported: 2, 4, 8                  */
  int flush_j;          /* FP32 partials are folded into FP64 after at most
                           this many list entries per thread; 0 = 256       */
  int arith;            /* QG_FP32_CENTRED only: QG_ARITH_SCALAR (the
                           default, 0) or QG_ARITH_PAIRED (two sinks per
                           float2 register, f32x2 FMA instructions)          */
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
  int32_t paired;             /* 1 if the paired-FP32 form runs              */
  int32_t eval_in_place;      /* 1 if the last qg_evaluate_host read the
                                 lists and wrote the results in place       */
} qg_stats;

/* Create a context on CUDA device `device`.  opt may be NULL (defaults). */
qg_status qg_create(qg_ctx **out, int device, const qg_options *opt);
void qg_destroy(qg_ctx *ctx);
qg_status qg_set_options(qg_ctx *ctx, const qg_options *opt);

/*
 * Sinks, grouped: group g owns sinks [group_off[g], group_off[g+1]).
 * x: [n][3] positions.  eps2: [n] per-sink squared softening (Phantom-GRAPE
 * keeps eps^2 per i-particle) or NULL to use eps2_all for every sink.
 * group_off: [ngroups+1], group_off[0] = 0, non-decreasing, last = n.
 */
qg_status qg_set_sinks(qg_ctx *ctx, int64_t n, const double *x, const float *eps2,
                       double eps2_all, int64_t ngroups, const int64_t *group_off);

/*
 * Source particles and the particle part of every group's list.
 * x: [ns][3], m: [ns].  list_off: [ngroups+1] (same ngroups as the sinks),
 * list_off[0] = 0, non-decreasing; list_idx: [list_off[ngroups]] entries,
 * each in [0, ns).
 */
qg_status qg_set_sources(qg_ctx *ctx, int64_t ns, const double *x, const double *m,
                         const int64_t *list_off, const int32_t *list_idx);

/*
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
 * One evaluation of every group: work-queue build (groups ordered by
 * descending cost), then one persistent launch over all groups.  The
 * sequence is captured once in a CUDA graph and replayed.  Asynchronous on
 * `cuda_stream` (NULL = the context's stream).
 */
qg_status qg_run(qg_ctx *ctx, void *cuda_stream);

/*
 * Autotuner: times every supported launch shape (sinks_per_thread x
 * warps_per_group x tile_j, and scalar vs paired FP32 arithmetic for
 * QG_FP32_CENTRED) of the current precision / expansion on the
 * inputs currently set, `reps` timed runs each after one warm-up run (the
 * force kernel's device time, CUDA events), and keeps the fastest as the
 * context's options.  The sink grouping itself (n_crit) is an input and is
 * not tuned here.  best (may be NULL) receives the chosen options,
 * best_ms the chosen shape's mean force-kernel time.  Synchronous; the
 * outputs afterwards hold a valid result of the chosen shape.
 */
qg_status qg_autotune(qg_ctx *ctx, void *cuda_stream, int reps, qg_options *best, float *best_ms);

/* Copy a [n][3] and phi [n] (either may be NULL) to the host; synchronises. */
qg_status qg_get_forces(qg_ctx *ctx, double *a, double *phi);

/* Device-to-device copy of the results into caller buffers on `cuda_stream`. */
qg_status qg_get_forces_dev(qg_ctx *ctx, double *a, double *phi, void *cuda_stream);

/*
 * One evaluation from HOST arrays: the inputs of qg_set_sinks, qg_set_sources
 * and qg_set_cells (same meaning, layout and checks), then the forces written
 * to a [n][3] and phi [n] (host).  The sinks, sources and cells are copied
 * first (one copy of x when src_x is the same array as sink_x and ns == n).
 * The lists then take one of two routes:
 *   - in place, when plist_idx, clist_idx, a and phi are all page-locked
 *     (cudaHostAlloc / cudaHostRegister), the GPU reads host memory
 *     through the host's page tables (a coherent CPU-GPU link, as on
 *     Grace-Blackwell) and the options select the FP32 centred precision in
 *     the scalar form: one persistent force launch reads every list index
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

qg_status qg_get_stats(const qg_ctx *ctx, qg_stats *out);

/*
 * Device time of the last qg_run, from CUDA events recorded inside its
 * graph: step_ms = whole step (work-queue build + force kernel), force_ms =
 * the persistent force kernel alone.  Synchronises the run's stream.
 * Either pointer may be NULL.
 */
qg_status qg_last_timing(qg_ctx *ctx, float *step_ms, float *force_ms);
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
 * device address and caches it (make that first call before any stream
 * capture).  The call waits for the argument check on `cuda_stream`, then
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
