// qg_attach.h -- hand-over of a GPU-built tree's groups and lists to a force
// context inside the library (qg_gtree_attach_move): the force calls of List 4
// take each group's lists as the tree walk produced them.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qg_devbuf.h"
#include "qgrav.h"

namespace qg {

// The arrays of one build and walk of a qg_gtree, all on the context's
// device.  The list offsets and indices come from the library's own walk, so
// they are valid by construction; their buffers are exchanged with the
// context's (ownership moves both ways, nothing is copied or checked).
struct TreeLists {
  int device = -1;                                          // the tree's device
  int64_t n = 0, G = 0, nn = 0, np_list = 0, nc_list = 0;  // particles, groups, nodes, list entries
  const double *xs = nullptr, *ms = nullptr;                // sorted positions [n][3] and masses [n]
  const double *com = nullptr, *mass = nullptr, *q = nullptr;  // node moments (Eq. 2)
  const int64_t *goff = nullptr;                            // group offsets [G + 1]
  // the lists: CSR (poff, coff: offsets [G + 1]) or, when ranges, group g's
  // entries at [poff[g], pend[g]) of pidx (the walk's own order; likewise
  // for the cells)
  bool ranges = false;
  DevBuf<int64_t> *poff = nullptr, *coff = nullptr;
  DevBuf<int64_t> *pend = nullptr, *cend = nullptr;
  DevBuf<int32_t> *pidx = nullptr, *cidx = nullptr;
};

// Sets the context's sinks, sources and cells from t (eps2_all as in
// qg_set_sinks) on stream s with one host synchronisation; positions, masses
// and moments are checked as qg_set_*_dev check them.
qg_status attach_tree_lists(qg_ctx *c, TreeLists &t, double eps2_all, cudaStream_t s);

}  // namespace qg
