// qg_internal.h -- parameter block and kernel registry shared by the CUDA
// translation units of the qg_* library (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qg {

// Device pointers and sizes one force launch reads.  Layouts:
//   sink_x    [n][3] double           sink_eps2 [n] float or null
//   group_off [G+1]                   queue     [nitems] group ids
//   src       [ns] double4_32a (x, y, z, m)
//   cell_xm   [nc] double4_32a (x, y, z, m)
//   cell_q    [nc][2] float4 ((q00, q01, q02, q11), (q12, q22, 0, 0))
//   cell_q64  [nc][6] double (q00 q01 q02 q11 q12 q22)
//   a         [n][3] double           phi [n] double
struct ForceParams {
  const double *sink_x;
  const float *sink_eps2;
  double eps2_all;
  const int64_t *group_off;
  const double4_32a *src;
  const int64_t *plist_off;
  const int32_t *plist_idx;
  const double4_32a *cell_xm;
  const float4 *cell_q;
  const double *cell_q64;
  const int64_t *clist_off;
  const int32_t *clist_idx;
  const int32_t *queue;
  int32_t nitems;
  int32_t *head;
  double *a;
  double *phi;
  int32_t tile;     // list entries per shared-memory tile
  int32_t flush_j;  // entries per thread between FP32 -> FP64 folds
};

// Dynamic shared memory of one force CTA.
inline size_t force_smem_bytes(bool fp64, int R, int nthreads, int tile) {
  const size_t r4 = fp64 ? 32 : 16, r2 = fp64 ? 16 : 8;
  // FP64 accumulators [4R][nthreads]; the sink offsets (R * nthreads
  // 4-vectors of Real, never larger) alias them
  (void)r4;
  return (size_t)nthreads * 4 * R * 8
         + (size_t)tile * (2 * (fp64 ? 32 : 16) + r2);  // staged tile: A, B (4-vectors), C (2-vector)
}

// Kernel registry (one function per translation unit that instantiates it).
// Returns nullptr for an unsupported combination.
const void *force_kernel_f32(int R, bool quad, bool guard, bool centred);
const void *force_kernel_f64(int R, bool quad, bool guard);

}  // namespace qg
