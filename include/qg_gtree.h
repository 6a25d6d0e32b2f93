/*
 * qg_gtree.h -- the oct-tree build, cell moments, sink groups and group walk
 * on the GPU (sm_103a), producing on the device the inputs the force path
 * (qgrav.h) consumes, so that a whole step stays on the GPU.
 *
 * Same method and the same results as the host builder (qg_tree.h), from
 * Kodama & Ishiyama, arXiv:1812.07313:
 *   - particles sorted along a 63-bit Morton curve of each system's bounding
 *     cube (21 levels), each system separately, equal keys in input order;
 *   - a node with at most leaf_max particles (or at level 21) is a leaf;
 *   - cell moments: mass, centre of mass and the quadrupole tensor about the
 *     centre of mass (Eq. 2), leaves from their particles, internal nodes
 *     from their children with the parallel-axis shift, all in FP64;
 *   - sink groups: maximal nodes with at most n_crit particles (Sec. 3.4);
 *   - the walk: for each group, a node becomes a j-cell iff its cube does not
 *     meet the group's particle bounding box, it holds none of the group's
 *     particles, and side^2 < theta^2 d^2 (d: distance from the node's centre
 *     of mass to the box; the test l/d < theta of Sec. 1); otherwise a leaf's
 *     particles join the j-particle list and an internal node is opened.
 *     One warp walks one group, testing up to 64 nodes at once; each group's
 *     lists hold the same entries as the host's depth-first walk, in the
 *     walk's own fixed order (deterministic from run to run).
 * Node numbering differs from the host builder's (level by level here); the
 * node set, the sorted particle order and the groups are the same.
 * qg_gtree_walk returns QG_ERR_STATE if a walk stack would overflow (not
 * reachable for trees of at most 21 levels, which is every tree built here).
 *
 * All arrays named *_dev are device memory on the tree's device; the tree
 * owns every array it exposes, valid until the next build / walk or destroy.
 * Every call returns a qg_status (QG_OK, QG_ERR_ARG, QG_ERR_CUDA,
 * QG_ERR_NOMEM, QG_ERR_STATE); calls are synchronous unless noted.
 */
#ifndef QG_GTREE_H
#define QG_GTREE_H

#include <stdint.h>

#include "qgrav.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qg_gtree qg_gtree;

/* A tree object on CUDA device `device` (no counterpart in the paper, whose
 * tree lives in the caller's node array, List 4); destroy frees it. */
qg_status qg_gtree_create(qg_gtree **out, int device);
void qg_gtree_destroy(qg_gtree *t);

/*
 * List 4's create_tree: the tree, its cell moments (Eq. 2) and the groups of
 * at most n_crit particles (Sec. 3.4); T_construct of Table 3.
 * Build from device arrays x [n][3], m [n] (n < 2^31).  sys_off [nsys+1] is a
 * HOST array: system s = particles [sys_off[s], sys_off[s+1]), sys_off[0] = 0,
 * sys_off[nsys] = n.  leaf_max >= 1, n_crit >= 1.
 */
qg_status qg_gtree_build(qg_gtree *t, int64_t n, const double *x_dev, const double *m_dev, int64_t nsys,
                         const int64_t *sys_off, int leaf_max, int n_crit, void *cuda_stream);

/* List 4's tree_traversal for every group at once (T_traverse of Table 3),
 * with the opening test of Sec. 1: group walk with opening angle theta
 * (theta <= 0 opens every node). */
qg_status qg_gtree_walk(qg_gtree *t, double theta, void *cuda_stream);

/* Sizes of the last build and walk (any pointer may be NULL). */
qg_status qg_gtree_sizes(const qg_gtree *t, int64_t *n, int64_t *nnodes, int64_t *ngroups, int64_t *n_plist,
                         int64_t *n_clist);

/*
 * Device arrays of the last build / walk (any pointer may be NULL):
 *   perm [n] int64 sorted -> input index; xs [n][3], ms [n] sorted particles;
 *   node_range [nnodes][2] int64 (sorted particle range), node_level [nnodes]
 *   int32, cell_com [nnodes][3], cell_m [nnodes], cell_q [nnodes][6] (q00 q01
 *   q02 q11 q12 q22), cell_side [nnodes]; group_off [ngroups+1] int64;
 *   plist_off / clist_off [ngroups+1] int64, plist_idx / clist_idx int32.
 * The walk leaves each group's lists where it finished them; the first call
 * that asks for a list array puts the lists in group (CSR) order, on the
 * walk's stream, and waits for it.
 */
qg_status qg_gtree_arrays(const qg_gtree *t, const int64_t **perm, const double **xs, const double **ms,
                          const int64_t **node_range, const int32_t **node_level, const double **cell_com,
                          const double **cell_m, const double **cell_q, const double **cell_side,
                          const int64_t **group_off, const int64_t **plist_off, const int32_t **plist_idx,
                          const int64_t **clist_off, const int32_t **clist_idx);

/*
 * Hands the groups and lists to the force calls, as List 4 passes each
 * group's i_list, j_list and j_cell to the g5_ / g5c_ calls:
 * set a force context's sinks (the sorted particles), sources and cells from
 * the last build and walk, device to device (the lists in CSR order, made
 * first if need be).  eps2_all as in qg_set_sinks.
 */
qg_status qg_gtree_attach(qg_gtree *t, qg_ctx *ctx, double eps2_all, void *cuda_stream);

/*
 * As qg_gtree_attach, without copies: the lists of the last walk move into
 * the context as the walk left them (each group's entries where the walk
 * finished them, with per-group begin / end offsets, so no CSR pass runs),
 * the context's former list buffers move into the tree, to be reused by the
 * next walk, their indices are not checked again (the walk produced them),
 * and the call synchronises `cuda_stream` once instead of once per input
 * set.  Positions, masses and moments are checked as qg_set_*_dev
 * check them.  Afterwards, until the next qg_gtree_walk, the tree holds no
 * lists: qg_gtree_arrays returns NULL for them and qg_gtree_attach /
 * qg_gtree_attach_move return QG_ERR_STATE (also after a failed call).  The
 * tree and the context must be on the same device (else QG_ERR_ARG).  The
 * time integrator (qg_sim.h) attaches this way every step.
 */
qg_status qg_gtree_attach_move(qg_gtree *t, qg_ctx *ctx, double eps2_all, void *cuda_stream);

/* List 4's assign_force_potential / add_force_potential: the per-sink
 * results returned to the particles.  out[perm[i]] = in[i] for k values per
 * particle (device arrays): results in sorted order back to input order. */
qg_status qg_gtree_unsort(const qg_gtree *t, const double *in_dev, double *out_dev, int k, void *cuda_stream);

/* T_construct and T_traverse of Table 3: device time of the last build and
 * walk (CUDA events), milliseconds. */
qg_status qg_gtree_timing(const qg_gtree *t, float *build_ms, float *walk_ms);

#ifdef __cplusplus
}
#endif
#endif
