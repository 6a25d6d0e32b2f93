/*
 * qg_tree.h -- host-side input generation for the tree-force hot path:
 * oct-tree build, cell moments, sink groups and the group walk that emits
 * the shared interaction lists (CSR) consumed by qg_set_sources /
 * qg_set_cells (see qgrav.h).
 *
 * Paper: Kodama & Ishiyama, arXiv:1812.07313.
 *   - tree method and its opening test l/d < theta: Sec. 1;
 *   - cell moments (mass, centre of mass, quadrupole tensor, Eq. 2);
 *   - modified tree algorithm: particles of a cell holding n_crit or fewer
 *     particles share one list of j-particles and j-cells: Sec. 3.4, the
 *     calc_force sample code (create_tree / traverse_tree).
 *
 * All arrays are host memory.  Every call returns 0 on success and a
 * negative value on bad arguments or allocation failure; no call aborts.
 * The handle owns every array it returns pointers to; they stay valid until
 * the next qgt_walk on the same handle (list arrays) or qgt_free (all).
 */
#ifndef QG_TREE_H
#define QG_TREE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qgt_tree qgt_tree;

/*
 * List 4's create_tree on the host: the tree and the groups of at most
 * n_crit particles (the modified tree algorithm, Sec. 3.4).
 * Build one oct-tree per system.  x: [n][3] positions, m: [n] masses.
 * sys_off: [nsys+1] offsets, system s = particles [sys_off[s], sys_off[s+1]).
 * leaf_max: a node with at most leaf_max particles is a leaf (>= 1).
 * n_crit: a group is a maximal node with at most n_crit particles (>= 1).
 * Particles are reordered along a Morton curve inside each system; the
 * permutation (sorted position -> input index) is qgt_perm().  Groups are
 * contiguous runs of sorted particles and never cross systems.
 */
int qgt_build(int64_t n, const double *x, const double *m,
              int64_t nsys, const int64_t *sys_off,
              int leaf_max, int n_crit, qgt_tree **out);

/* Frees a tree built by qgt_build. */
void qgt_free(qgt_tree *t);

/* Sizes: particles, nodes (= cells), groups. */
int qgt_sizes(const qgt_tree *t, int64_t *n, int64_t *nnodes, int64_t *ngroups);

/* perm[n]: sorted index -> input index (int64).  group_off[ngroups+1]. */
const int64_t *qgt_perm(const qgt_tree *t);
const int64_t *qgt_group_off(const qgt_tree *t);

/*
 * Per node (cell) j: com [3], mass, q [6] = q00 q01 q02 q11 q12 q22
 * (unhalved Eq. 2 about the centre of mass), geometric centre [3], side
 * length, sorted particle range [begin, end), system index.
 * The arrays are [nnodes][k] row-major.
 */
int qgt_nodes(const qgt_tree *t, const double **com, const double **mass,
              const double **q, const double **centre, const double **side,
              const int64_t **range /* [nnodes][2] */, const int32_t **sys);

/*
 * List 4's tree_traversal for every group, with the opening test l/d < theta
 * of Sec. 1 (theta, not theta^2 as List 4 passes it).
 * Group walk with opening angle theta.  For each group g with particle
 * bounding box B_g, a node n is accepted as a j-cell iff its cube does not
 * meet B_g, it holds none of g's particles, and side(n)^2 < theta^2 d^2
 * where d is the distance from n's centre of mass to B_g.  Otherwise it is
 * opened: a leaf's particles join the j-particle list (the group's own
 * particles included), an internal node's children are visited.
 * theta <= 0 opens everything (direct summation through the lists).
 * Particle list entries index the sorted particle array; cell entries index
 * the node arrays; both are int32 (so n and nnodes must be < 2^31).
 */
int qgt_walk(qgt_tree *t, double theta, int nthreads);

/* The lists of the last walk as CSR arrays: List 4's jlist (j-particles)
 * and jcell (j-cells) of every group, concatenated. */
int qgt_lists(const qgt_tree *t,
              const int64_t **plist_off, const int32_t **plist_idx, int64_t *np_total,
              const int64_t **clist_off, const int32_t **clist_idx, int64_t *nc_total);

#ifdef __cplusplus
}
#endif
#endif
