/*
 * qg_oracle.c -- plain FP64 CPU oracle for the monopole + quadrupole
 * tree-force evaluation of Kodama & Ishiyama, "Acceleration of the tree
 * method with SIMD instruction set" (arXiv:1812.07313).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, helper or
 * constant with the CUDA path (paper_1812_07313_gb300/csrc).
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: one sink at a time, one list entry at a time, all in double, no
 * blocking, no fusion, no reordering.
 *
 * Conventions fixed by the paper and by the readings of it:
 *   - G = 1 (the paper's kernel carries no G; its simulations set G = 1).
 *   - r_ij = r_j - r_i, rhat^2 = |r_ij|^2 + eps_i^2 (Plummer softening in
 *     every term, including the rhat^5 of the quadrupole term, Eq. 1).
 *   - phi is the physical potential, negative (Eq. 1).
 *   - a = -grad phi (Eq. 6).  Eq. 7 as printed carries a leading minus sign
 *     which, with r_ij = r_j - r_i, would make gravity repulsive; -grad of
 *     Eq. 1 worked out by hand (and the paper's own step list, which adds the
 *     first term and subtracts the second) gives
 *         a_i = + sum_j [ (phi_mono + 5 phi_quad) / rhat^2 * r_ij
 *                         - Q_j r_ij / rhat^5 ].
 *     The finite-difference test in tests/ pins this reading.
 *   - Q is unhalved (Eq. 2); the 1/2 sits in phi_quad (Eq. 5).
 *   - q22 is taken as supplied, not recomputed (Eq. 3 and the text after it).
 *   - A pair with rhat^2 == 0 exactly (zero softening, coincident points)
 *     contributes nothing.
 *
 * Parity of every function here is pinned by tests/test_oracle_pins.py
 * against closed forms, brute force and invariants; no function is
 * "parity unpinned".
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define QGO_OK 0
#define QGO_ERR_ARG -1

/* ------------------------------------------------------------------ */
/* Eq. 2: total mass, centre of mass and quadrupole tensor of a set of  */
/* point masses, straight from the definition.                          */
/*   Q = sum_k m_k (3 x_jk x_jk^T - r_jk^2 I),  x_jk = x_k - x_j (COM)   */
/* q is returned as q00 q01 q02 q11 q12 q22.                            */
/* ------------------------------------------------------------------ */
int qgo_cell_moments(int64_t n, const double *x, const double *m,
                     double *mass_out, double *com_out, double *q_out)
{
    if (n < 0 || (n > 0 && (!x || !m)) || !mass_out || !com_out || !q_out)
        return QGO_ERR_ARG;
    double mass = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    for (int64_t k = 0; k < n; k++) {
        mass += m[k];
        cx += m[k] * x[3 * k + 0];
        cy += m[k] * x[3 * k + 1];
        cz += m[k] * x[3 * k + 2];
    }
    if (mass > 0.0) { cx /= mass; cy /= mass; cz /= mass; }
    double q00 = 0, q01 = 0, q02 = 0, q11 = 0, q12 = 0, q22 = 0;
    for (int64_t k = 0; k < n; k++) {
        double xk = x[3 * k + 0] - cx;
        double yk = x[3 * k + 1] - cy;
        double zk = x[3 * k + 2] - cz;
        double r2 = xk * xk + yk * yk + zk * zk;
        q00 += m[k] * (3.0 * xk * xk - r2);
        q01 += m[k] * (3.0 * xk * yk);
        q02 += m[k] * (3.0 * xk * zk);
        q11 += m[k] * (3.0 * yk * yk - r2);
        q12 += m[k] * (3.0 * yk * zk);
        q22 += m[k] * (3.0 * zk * zk - r2);
    }
    *mass_out = mass;
    com_out[0] = cx; com_out[1] = cy; com_out[2] = cz;
    q_out[0] = q00; q_out[1] = q01; q_out[2] = q02;
    q_out[3] = q11; q_out[4] = q12; q_out[5] = q22;
    return QGO_OK;
}

/* Softening of sink i: per-sink eps^2 if given, else the global value. */
static double eps2_of(const double *eps2, double eps2_all, int64_t i)
{
    return eps2 ? eps2[i] : eps2_all;
}

/* ------------------------------------------------------------------ */
/* One source particle acting on one sink: the monopole (Plummer point  */
/* mass) term, Eq. 4 and its gradient.                                  */
/* ------------------------------------------------------------------ */
static void particle_term(const double xi[3], double eps2,
                          const double xj[3], double mj,
                          double acc[3], double *pot)
{
    double d0 = xj[0] - xi[0];
    double d1 = xj[1] - xi[1];
    double d2 = xj[2] - xi[2];
    double rhat2 = d0 * d0 + d1 * d1 + d2 * d2 + eps2;
    if (rhat2 == 0.0) return;
    double rhat = sqrt(rhat2);
    double phi_mono = mj / rhat;                 /* Eq. 4 */
    *pot -= phi_mono;                            /* Eq. 1, first term */
    double c = phi_mono / rhat2;                 /* m / rhat^3 */
    acc[0] += c * d0;
    acc[1] += c * d1;
    acc[2] += c * d2;
}

/* ------------------------------------------------------------------ */
/* One tree cell acting on one sink: Eq. 1 (potential), Eqs. 4-5 and the */
/* sign-corrected Eq. 7 (acceleration).  With use_quad == 0 the cell is  */
/* a point mass at its centre of mass (monopole-only tree code).         */
/* ------------------------------------------------------------------ */
static void cell_term(const double xi[3], double eps2,
                      const double com[3], double mj, const double q[6],
                      int use_quad, double acc[3], double *pot)
{
    /* r_ij = r_j - r_i */
    double d[3] = { com[0] - xi[0], com[1] - xi[1], com[2] - xi[2] };
    double rhat2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
    if (rhat2 == 0.0) return;
    double rhat = sqrt(rhat2);
    double rhat5 = rhat2 * rhat2 * rhat;

    /* The symmetric tensor Q_j of Eq. 2 written out in full. */
    double Q[3][3] = {
        { q[0], q[1], q[2] },
        { q[1], q[3], q[4] },
        { q[2], q[4], q[5] },
    };
    double Qd[3] = { 0.0, 0.0, 0.0 };
    double dQd = 0.0;
    if (use_quad) {
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                Qd[a] += Q[a][b] * d[b];
        for (int a = 0; a < 3; a++)
            dQd += d[a] * Qd[a];
    }

    double phi_mono = mj / rhat;                 /* Eq. 4 */
    double phi_quad = dQd / (2.0 * rhat5);       /* Eq. 5 */
    *pot -= phi_mono + phi_quad;                 /* Eq. 1 */
    for (int a = 0; a < 3; a++)                  /* Eq. 7, sign corrected */
        acc[a] += (phi_mono + 5.0 * phi_quad) / rhat2 * d[a] - Qd[a] / rhat5;
}

/* ------------------------------------------------------------------ */
/* Modified tree algorithm (Barnes 1990, Sec. 3.4 of the paper): the     */
/* sinks of group g, [group_off[g], group_off[g+1]), share one           */
/* interaction list of particles plist_idx[plist_off[g]..plist_off[g+1]) */
/* and cells clist_idx[clist_off[g]..clist_off[g+1]).                    */
/*                                                                      */
/* Positions are [n][3] doubles; cell_q is [nc][6] (q00 q01 q02 q11 q12  */
/* q22, unhalved Eq. 2).  sink_eps2 may be NULL (global eps2_all).        */
/* groups == NULL evaluates every group; otherwise only the ngroups_eval */
/* listed groups, whose sinks' a/phi are the only ones written.          */
/* a is [n][3], phi is [n].                                              */
/* ------------------------------------------------------------------ */
/* Host threads over which qgo_expansion_forces splits its groups (default 1:
 * the plain serial oracle).  A group is always evaluated by one thread, in
 * the order below, so the results do not depend on the thread count. */
static int qgo_threads = 1;

void qgo_set_threads(int n) { qgo_threads = n < 1 ? 1 : n; }

int qgo_expansion_forces(int64_t ngroups, const int64_t *group_off,
                         const double *sink_x, const double *sink_eps2,
                         double eps2_all,
                         const double *src_x, const double *src_m,
                         const int64_t *plist_off, const int32_t *plist_idx,
                         const double *cell_com, const double *cell_m,
                         const double *cell_q,
                         const int64_t *clist_off, const int32_t *clist_idx,
                         int use_quad,
                         const int64_t *groups, int64_t ngroups_eval,
                         double *a, double *phi)
{
    if (ngroups < 0 || !group_off || !a || !phi) return QGO_ERR_ARG;
    if (!plist_off || !clist_off) return QGO_ERR_ARG;
    int64_t nloop = groups ? ngroups_eval : ngroups;
    for (int64_t t = 0; t < nloop; t++) {
        int64_t g = groups ? groups[t] : t;
        if (g < 0 || g >= ngroups) return QGO_ERR_ARG;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(qgo_threads) if (qgo_threads > 1)
#endif
    for (int64_t t = 0; t < nloop; t++) {
        int64_t g = groups ? groups[t] : t;
        for (int64_t i = group_off[g]; i < group_off[g + 1]; i++) {
            const double *xi = &sink_x[3 * i];
            double eps2 = eps2_of(sink_eps2, eps2_all, i);
            double acc[3] = { 0.0, 0.0, 0.0 };
            double pot = 0.0;
            for (int64_t k = plist_off[g]; k < plist_off[g + 1]; k++) {
                int64_t j = plist_idx[k];
                particle_term(xi, eps2, &src_x[3 * j], src_m[j], acc, &pot);
            }
            for (int64_t k = clist_off[g]; k < clist_off[g + 1]; k++) {
                int64_t j = clist_idx[k];
                cell_term(xi, eps2, &cell_com[3 * j], cell_m[j], &cell_q[6 * j],
                          use_quad, acc, &pot);
            }
            a[3 * i + 0] = acc[0];
            a[3 * i + 1] = acc[1];
            a[3 * i + 2] = acc[2];
            phi[i] = pot;
        }
    }
    return QGO_OK;
}

/* ------------------------------------------------------------------ */
/* Direct O(N^2) summation (the "direct particle-particle method" that   */
/* Eq. 8 measures the tree force against): every source particle acts on */
/* every listed sink as a Plummer point mass.  sinks[k] (k < nsink) are  */
/* [3] positions; eps2 per sink or global.  Pairs with rhat^2 == 0 are   */
/* skipped, so a sink that is also a source with eps = 0 gets no self    */
/* term; with eps > 0 the self pair adds -m/eps to phi and nothing to a. */
/* ------------------------------------------------------------------ */
int qgo_direct_forces(int64_t nsink, const double *sink_x,
                      const double *sink_eps2, double eps2_all,
                      int64_t nsrc, const double *src_x, const double *src_m,
                      double *a, double *phi)
{
    if (nsink < 0 || nsrc < 0 || !a || !phi) return QGO_ERR_ARG;
    for (int64_t i = 0; i < nsink; i++) {
        const double *xi = &sink_x[3 * i];
        double eps2 = eps2_of(sink_eps2, eps2_all, i);
        double acc[3] = { 0.0, 0.0, 0.0 };
        double pot = 0.0;
        for (int64_t j = 0; j < nsrc; j++)
            particle_term(xi, eps2, &src_x[3 * j], src_m[j], acc, &pot);
        a[3 * i + 0] = acc[0];
        a[3 * i + 1] = acc[1];
        a[3 * i + 2] = acc[2];
        phi[i] = pot;
    }
    return QGO_OK;
}
