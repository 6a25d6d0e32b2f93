// qg_tree.cpp -- host oct-tree, cell moments, sink groups and group walk.
//
// This is input generation for the force hot path (the lists are the input
// of qg_set_sources / qg_set_cells).  It follows the modified tree algorithm
// of Sec. 3.4 of Kodama & Ishiyama (arXiv:1812.07313): the particles of a
// maximal cell with at most n_crit particles form one group and share one
// interaction list of j-particles and j-cells.  Cell moments follow Eq. 2
// (quadrupole about the centre of mass), accumulated bottom-up with the
// parallel-axis shift.  The opening test is l/d < theta (Sec. 1).
//
// Layout: per system, particles are sorted along a 63-bit Morton curve of
// the system's bounding cube, so every node (and every group) is a
// contiguous run of sorted particles.  Children of a node are stored
// contiguously after it.
#include "qg_tree.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int kMaxLevel = 21;  // 21 bits per axis -> 63-bit keys

struct Node {
  int64_t begin, end;   // sorted particle range
  int32_t first_child;  // index of first child, -1 for a leaf
  int32_t nchild;
  int32_t sys;
  int32_t level;
};

inline uint64_t spread3(uint64_t v) {
  // spread the low 21 bits of v so that bit b lands at bit 3b
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

// LSD radix sort of (key, index) pairs by the 63-bit key, 16 bits per pass.
void radix_sort(std::vector<uint64_t> &key, std::vector<int64_t> &idx) {
  const size_t n = key.size();
  std::vector<uint64_t> k2(n);
  std::vector<int64_t> i2(n);
  std::vector<int64_t> count(1 << 16);
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 16 * pass;
    std::fill(count.begin(), count.end(), 0);
    for (size_t i = 0; i < n; i++) count[(key[i] >> shift) & 0xffff]++;
    int64_t s = 0;
    for (auto &c : count) { int64_t t = c; c = s; s += t; }
    for (size_t i = 0; i < n; i++) {
      int64_t p = count[(key[i] >> shift) & 0xffff]++;
      k2[p] = key[i];
      i2[p] = idx[i];
    }
    key.swap(k2);
    idx.swap(i2);
  }
}

}  // namespace

struct qgt_tree {
  int64_t n = 0;
  int leaf_max = 8, n_crit = 64;
  std::vector<int64_t> perm;        // sorted -> input
  std::vector<double> xs, ms;       // sorted positions / masses
  std::vector<Node> nodes;
  std::vector<double> com, mass, q, centre, side;
  std::vector<int64_t> range;
  std::vector<int32_t> node_sys;
  std::vector<int64_t> group_off;
  std::vector<int32_t> group_node;
  std::vector<int32_t> sys_root;    // root node of each system (-1 if empty)
  // lists of the last walk
  std::vector<int64_t> plist_off, clist_off;
  std::vector<int32_t> plist_idx, clist_idx;
};

namespace {

// Build the tree of one system: particles [b, e) of the global sorted arrays
// (already sorted by key inside the system).  Appends nodes to local vectors.
struct SysTree {
  std::vector<Node> nodes;
  std::vector<double> centre, half;
};

void build_system(const std::vector<uint64_t> &key, int64_t b, int64_t e, int32_t sys,
                  const double lo[3], double width, int leaf_max, SysTree &st) {
  st.nodes.clear();
  st.centre.clear();
  st.half.clear();
  if (e <= b) return;
  Node root{b, e, -1, 0, sys, 0};
  st.nodes.push_back(root);
  st.centre.insert(st.centre.end(), {lo[0] + 0.5 * width, lo[1] + 0.5 * width, lo[2] + 0.5 * width});
  st.half.push_back(0.5 * width);
  std::vector<int32_t> stack{0};
  while (!stack.empty()) {
    int32_t k = stack.back();
    stack.pop_back();
    Node nd = st.nodes[k];
    int64_t cnt = nd.end - nd.begin;
    if (cnt <= leaf_max || nd.level >= kMaxLevel) continue;  // leaf
    const int shift = 3 * (kMaxLevel - 1 - nd.level);
    int64_t cut[9];
    cut[0] = nd.begin;
    cut[8] = nd.end;
    for (int o = 1; o < 8; o++) {
      // first particle in [nd.begin, nd.end) whose digit at this level >= o
      int64_t lo_i = cut[o - 1], hi_i = nd.end;
      while (lo_i < hi_i) {
        int64_t mid = (lo_i + hi_i) / 2;
        if ((int)((key[mid] >> shift) & 7) < o) lo_i = mid + 1; else hi_i = mid;
      }
      cut[o] = lo_i;
    }
    int32_t first = (int32_t)st.nodes.size();
    int32_t nchild = 0;
    const double h = st.half[k] * 0.5;
    const double cx = st.centre[3 * k], cy = st.centre[3 * k + 1], cz = st.centre[3 * k + 2];
    for (int o = 0; o < 8; o++) {
      if (cut[o + 1] <= cut[o]) continue;
      Node c{cut[o], cut[o + 1], -1, 0, sys, nd.level + 1};
      st.nodes.push_back(c);
      st.centre.push_back(cx + (((o >> 2) & 1) ? h : -h));
      st.centre.push_back(cy + (((o >> 1) & 1) ? h : -h));
      st.centre.push_back(cz + ((o & 1) ? h : -h));
      st.half.push_back(h);
      nchild++;
    }
    st.nodes[k].first_child = first;
    st.nodes[k].nchild = nchild;
    for (int c = nchild - 1; c >= 0; c--) stack.push_back(first + c);
  }
}

}  // namespace

extern "C" int qgt_build(int64_t n, const double *x, const double *m, int64_t nsys,
                         const int64_t *sys_off, int leaf_max, int n_crit, qgt_tree **out) {
  if (!out) return -1;
  *out = nullptr;
  if (n < 0 || nsys < 1 || !sys_off || leaf_max < 1 || n_crit < 1) return -1;
  if (n > 0 && (!x || !m)) return -1;
  if (sys_off[0] != 0 || sys_off[nsys] != n) return -1;
  for (int64_t s = 0; s < nsys; s++)
    if (sys_off[s + 1] < sys_off[s]) return -1;
  for (int64_t i = 0; i < 3 * n; i++)
    if (!std::isfinite(x[i])) return -1;
  qgt_tree *t = new (std::nothrow) qgt_tree;
  if (!t) return -3;
  try {
    t->n = n;
    t->leaf_max = leaf_max;
    t->n_crit = n_crit;
    std::vector<uint64_t> key(n);
    t->perm.resize(n);
    std::vector<double> lo(3 * nsys), width(nsys);
    // per system bounding cube and Morton keys
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < nsys; s++) {
      int64_t b = sys_off[s], e = sys_off[s + 1];
      double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int64_t i = b; i < e; i++)
        for (int d = 0; d < 3; d++) {
          mn[d] = std::min(mn[d], x[3 * i + d]);
          mx[d] = std::max(mx[d], x[3 * i + d]);
        }
      double w = 0.0;
      for (int d = 0; d < 3; d++) w = std::max(w, mx[d] - mn[d]);
      if (!(w > 0.0)) w = 1.0;
      // pad so that the largest coordinate maps strictly inside the cube
      w *= 1.0 + 1e-9;
      for (int d = 0; d < 3; d++) {
        double c = 0.5 * (mn[d] + mx[d]);
        lo[3 * s + d] = e > b ? c - 0.5 * w : 0.0;
      }
      width[s] = w;
      const double scale = (double)(1u << kMaxLevel) / w;
      for (int64_t i = b; i < e; i++) {
        uint64_t k = 0;
        for (int d = 0; d < 3; d++) {
          double f = (x[3 * i + d] - lo[3 * s + d]) * scale;
          int64_t c = (int64_t)std::floor(f);
          c = std::min<int64_t>(std::max<int64_t>(c, 0), (1 << kMaxLevel) - 1);
          k |= spread3((uint64_t)c) << (2 - d);
        }
        key[i] = k;
        t->perm[i] = i;
      }
    }
    // sort each system independently (systems are contiguous)
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < nsys; s++) {
      int64_t b = sys_off[s], e = sys_off[s + 1];
      std::vector<uint64_t> ks(key.begin() + b, key.begin() + e);
      std::vector<int64_t> is(t->perm.begin() + b, t->perm.begin() + e);
      radix_sort(ks, is);
      std::copy(ks.begin(), ks.end(), key.begin() + b);
      std::copy(is.begin(), is.end(), t->perm.begin() + b);
    }
    t->xs.resize(3 * n);
    t->ms.resize(n);
#pragma omp parallel for
    for (int64_t i = 0; i < n; i++) {
      int64_t p = t->perm[i];
      t->xs[3 * i] = x[3 * p];
      t->xs[3 * i + 1] = x[3 * p + 1];
      t->xs[3 * i + 2] = x[3 * p + 2];
      t->ms[i] = m[p];
    }
    // trees per system
    std::vector<SysTree> st(nsys);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < nsys; s++)
      build_system(key, sys_off[s], sys_off[s + 1], (int32_t)s, &lo[3 * s], width[s], leaf_max, st[s]);
    std::vector<int64_t> node_base(nsys + 1, 0);
    for (int64_t s = 0; s < nsys; s++) node_base[s + 1] = node_base[s] + (int64_t)st[s].nodes.size();
    const int64_t nn = node_base[nsys];
    if (nn >= INT32_MAX || n >= INT32_MAX) { delete t; return -1; }
    t->nodes.resize(nn);
    t->centre.resize(3 * nn);
    t->side.resize(nn);
    t->com.assign(3 * nn, 0.0);
    t->mass.assign(nn, 0.0);
    t->q.assign(6 * nn, 0.0);
    t->range.resize(2 * nn);
    t->node_sys.resize(nn);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < nsys; s++) {
      const int64_t base = node_base[s];
      SysTree &S = st[s];
      for (size_t k = 0; k < S.nodes.size(); k++) {
        Node nd = S.nodes[k];
        if (nd.first_child >= 0) nd.first_child += (int32_t)base;
        t->nodes[base + k] = nd;
        for (int d = 0; d < 3; d++) t->centre[3 * (base + k) + d] = S.centre[3 * k + d];
        t->side[base + k] = 2.0 * S.half[k];
        t->range[2 * (base + k)] = nd.begin;
        t->range[2 * (base + k) + 1] = nd.end;
        t->node_sys[base + k] = (int32_t)s;
      }
      // moments bottom-up: children are stored after their parent
      for (int64_t k = (int64_t)S.nodes.size() - 1; k >= 0; k--) {
        const int64_t j = base + k;
        const Node &nd = t->nodes[j];
        double *c = &t->com[3 * j], *qq = &t->q[6 * j];
        double M = 0.0;
        if (nd.first_child < 0) {
          // Eq. 2 directly over the leaf's particles
          for (int64_t i = nd.begin; i < nd.end; i++) {
            M += t->ms[i];
            for (int d = 0; d < 3; d++) c[d] = std::fma(t->ms[i], t->xs[3 * i + d], c[d]);
          }
          if (M > 0) {  // one division (the GPU builder evaluates the same expressions)
            const double inv = 1.0 / M;
            for (int d = 0; d < 3; d++) c[d] *= inv;
          }
          // Eq. 2 as Q = 3 S - tr(S) I with S = sum m r r^T (the same sum,
          // fewer operations; the GPU builder evaluates the same expressions,
          // with the same explicit fused multiply-adds)
          double sm[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
          for (int64_t i = nd.begin; i < nd.end; i++) {
            const double r[3] = {t->xs[3 * i] - c[0], t->xs[3 * i + 1] - c[1], t->xs[3 * i + 2] - c[2]};
            const double mi = t->ms[i];
            const double m0 = mi * r[0], m1 = mi * r[1], m2 = mi * r[2];
            sm[0] = std::fma(m0, r[0], sm[0]);
            sm[1] = std::fma(m0, r[1], sm[1]);
            sm[2] = std::fma(m0, r[2], sm[2]);
            sm[3] = std::fma(m1, r[1], sm[3]);
            sm[4] = std::fma(m1, r[2], sm[4]);
            sm[5] = std::fma(m2, r[2], sm[5]);
          }
          const double tr = sm[0] + sm[3] + sm[5];
          qq[0] = 3 * sm[0] - tr;
          qq[1] = 3 * sm[1];
          qq[2] = 3 * sm[2];
          qq[3] = 3 * sm[3] - tr;
          qq[4] = 3 * sm[4];
          qq[5] = 3 * sm[5] - tr;
        } else {
          for (int ch = 0; ch < nd.nchild; ch++) {
            const int64_t cj = nd.first_child + ch;
            M += t->mass[cj];
            for (int d = 0; d < 3; d++) c[d] = std::fma(t->mass[cj], t->com[3 * cj + d], c[d]);
          }
          if (M > 0) {  // one division (the GPU builder evaluates the same expressions)
            const double inv = 1.0 / M;
            for (int d = 0; d < 3; d++) c[d] *= inv;
          }
          // parallel-axis shift of each child's tensor to the parent's COM:
          // Q = sum Q_c + 3 S - tr(S) I with S = sum m_c d d^T
          double sm[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, qs[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
          for (int ch = 0; ch < nd.nchild; ch++) {
            const int64_t cj = nd.first_child + ch;
            const double mc = t->mass[cj];
            const double r[3] = {t->com[3 * cj] - c[0], t->com[3 * cj + 1] - c[1], t->com[3 * cj + 2] - c[2]};
            const double m0 = mc * r[0], m1 = mc * r[1], m2 = mc * r[2];
            sm[0] = std::fma(m0, r[0], sm[0]);
            sm[1] = std::fma(m0, r[1], sm[1]);
            sm[2] = std::fma(m0, r[2], sm[2]);
            sm[3] = std::fma(m1, r[1], sm[3]);
            sm[4] = std::fma(m1, r[2], sm[4]);
            sm[5] = std::fma(m2, r[2], sm[5]);
            const double *qc = &t->q[6 * cj];
            for (int k = 0; k < 6; k++) qs[k] += qc[k];
          }
          const double tr = sm[0] + sm[3] + sm[5];
          qq[0] = qs[0] + (3 * sm[0] - tr);
          qq[1] = qs[1] + 3 * sm[1];
          qq[2] = qs[2] + 3 * sm[2];
          qq[3] = qs[3] + (3 * sm[3] - tr);
          qq[4] = qs[4] + 3 * sm[4];
          qq[5] = qs[5] + (3 * sm[5] - tr);
        }
        t->mass[j] = M;
      }
    }
    // groups: maximal nodes with at most n_crit particles, in Morton order
    t->group_off.clear();
    t->group_node.clear();
    t->group_off.push_back(0);
    t->sys_root.assign(nsys, -1);
    for (int64_t s = 0; s < nsys; s++) {
      if (st[s].nodes.empty()) continue;
      t->sys_root[s] = (int32_t)node_base[s];
      std::vector<int64_t> stack{node_base[s]};
      while (!stack.empty()) {
        int64_t k = stack.back();
        stack.pop_back();
        const Node &nd = t->nodes[k];
        if (nd.end - nd.begin <= n_crit || nd.first_child < 0) {
          t->group_node.push_back((int32_t)k);
          t->group_off.push_back(nd.end);
        } else {
          for (int c = nd.nchild - 1; c >= 0; c--) stack.push_back(nd.first_child + c);
        }
      }
    }
  } catch (const std::bad_alloc &) {
    delete t;
    return -3;
  }
  *out = t;
  return 0;
}

extern "C" void qgt_free(qgt_tree *t) { delete t; }

extern "C" int qgt_sizes(const qgt_tree *t, int64_t *n, int64_t *nnodes, int64_t *ngroups) {
  if (!t) return -1;
  if (n) *n = t->n;
  if (nnodes) *nnodes = (int64_t)t->nodes.size();
  if (ngroups) *ngroups = (int64_t)t->group_off.size() - 1;
  return 0;
}

extern "C" const int64_t *qgt_perm(const qgt_tree *t) { return t ? t->perm.data() : nullptr; }
extern "C" const int64_t *qgt_group_off(const qgt_tree *t) { return t ? t->group_off.data() : nullptr; }

extern "C" int qgt_nodes(const qgt_tree *t, const double **com, const double **mass,
                         const double **q, const double **centre, const double **side,
                         const int64_t **range, const int32_t **sys) {
  if (!t) return -1;
  if (com) *com = t->com.data();
  if (mass) *mass = t->mass.data();
  if (q) *q = t->q.data();
  if (centre) *centre = t->centre.data();
  if (side) *side = t->side.data();
  if (range) *range = t->range.data();
  if (sys) *sys = t->node_sys.data();
  return 0;
}

extern "C" int qgt_walk(qgt_tree *t, double theta, int nthreads) {
  if (!t || !std::isfinite(theta)) return -1;
  const int64_t G = (int64_t)t->group_off.size() - 1;
  const double theta2 = theta > 0 ? theta * theta : 0.0;
  try {
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    (void)nthreads;
    std::vector<std::vector<int32_t>> pbuf(nt), cbuf(nt);
    std::vector<int64_t> pstart(G), pcnt(G), cstart(G), ccnt(G);
    std::vector<int32_t> owner(G);
#pragma omp parallel num_threads(nt)
    {
      int tid = 0;
#ifdef _OPENMP
      tid = omp_get_thread_num();
#endif
      std::vector<int32_t> &pb = pbuf[tid];
      std::vector<int32_t> &cb = cbuf[tid];
      std::vector<int32_t> stack;
#pragma omp for schedule(dynamic, 16)
      for (int64_t g = 0; g < G; g++) {
        const int64_t gb = t->group_off[g], ge = t->group_off[g + 1];
        const int32_t root = t->sys_root[t->node_sys[t->group_node[g]]];
        double bmin[3] = {INFINITY, INFINITY, INFINITY}, bmax[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = gb; i < ge; i++)
          for (int d = 0; d < 3; d++) {
            bmin[d] = std::min(bmin[d], t->xs[3 * i + d]);
            bmax[d] = std::max(bmax[d], t->xs[3 * i + d]);
          }
        owner[g] = tid;
        pstart[g] = (int64_t)pb.size();
        cstart[g] = (int64_t)cb.size();
        stack.clear();
        stack.push_back(root);
        while (!stack.empty()) {
          const int32_t k = stack.back();
          stack.pop_back();
          const Node &nd = t->nodes[k];
          bool open = true;
          if (theta2 > 0.0 && !(nd.begin < ge && nd.end > gb)) {
            const double h = 0.5 * t->side[k];
            const double *cc = &t->centre[3 * k];
            bool meets = true;
            for (int d = 0; d < 3; d++)
              if (cc[d] + h < bmin[d] || cc[d] - h > bmax[d]) meets = false;
            if (!meets) {
              double d2 = 0.0;
              for (int d = 0; d < 3; d++) {
                const double c = t->com[3 * k + d];
                const double e = c < bmin[d] ? bmin[d] - c : (c > bmax[d] ? c - bmax[d] : 0.0);
                d2 += e * e;
              }
              if (t->side[k] * t->side[k] < theta2 * d2) open = false;
            }
          }
          if (!open) {
            cb.push_back(k);
          } else if (nd.first_child < 0) {
            for (int64_t i = nd.begin; i < nd.end; i++) pb.push_back((int32_t)i);
          } else {
            for (int c = nd.nchild - 1; c >= 0; c--) stack.push_back(nd.first_child + c);
          }
        }
        pcnt[g] = (int64_t)pb.size() - pstart[g];
        ccnt[g] = (int64_t)cb.size() - cstart[g];
      }
    }
    t->plist_off.assign(G + 1, 0);
    t->clist_off.assign(G + 1, 0);
    for (int64_t g = 0; g < G; g++) {
      t->plist_off[g + 1] = t->plist_off[g] + pcnt[g];
      t->clist_off[g + 1] = t->clist_off[g] + ccnt[g];
    }
    t->plist_idx.resize(t->plist_off[G]);
    t->clist_idx.resize(t->clist_off[G]);
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t g = 0; g < G; g++) {
      const int o = owner[g];
      std::memcpy(&t->plist_idx[t->plist_off[g]], pbuf[o].data() + pstart[g], pcnt[g] * sizeof(int32_t));
      std::memcpy(&t->clist_idx[t->clist_off[g]], cbuf[o].data() + cstart[g], ccnt[g] * sizeof(int32_t));
    }
  } catch (const std::bad_alloc &) {
    return -3;
  }
  return 0;
}

extern "C" int qgt_lists(const qgt_tree *t, const int64_t **plist_off, const int32_t **plist_idx,
                         int64_t *np_total, const int64_t **clist_off, const int32_t **clist_idx,
                         int64_t *nc_total) {
  if (!t || t->plist_off.empty()) return -1;
  if (plist_off) *plist_off = t->plist_off.data();
  if (plist_idx) *plist_idx = t->plist_idx.data();
  if (np_total) *np_total = (int64_t)t->plist_idx.size();
  if (clist_off) *clist_off = t->clist_off.data();
  if (clist_idx) *clist_idx = t->clist_idx.data();
  if (nc_total) *nc_total = (int64_t)t->clist_idx.size();
  return 0;
}
