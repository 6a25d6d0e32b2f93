// qg_internal.h -- parameter block and kernel registry shared by the CUDA
// translation units of the qg_* library (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qg {

// One gathered list entry's position (FP64, centred on the GPU) and its
// mass as the FP32 kernels use it: one aligned 32-byte sector.
struct __align__(32) PosMass {
  double x, y, z;
  float m;
  float pad;
};

// Largest magnitude of a position coordinate any entry point accepts (and of
// a mass, a quadrupole component or a softening in the allocation-free
// entry point): every value the kernels round with f64_to_f32_rn below,
// position offsets x_j - c_g included, then stays below 2^101, inside its
// domain.  Larger or non-finite inputs are rejected with QG_ERR_ARG.
constexpr double kMaxInput = 0x1p100;

// Round a double to the nearest float, ties to even, with integer
// operations only (IEEE 754 binary64 -> binary32: keep the sign, rebias the
// exponent from 1023 to 127, keep the top 23 of the 52 fraction bits and
// round on the 29 dropped ones).  Domain: finite |x| < 2^128 (a value that
// rounds up to 2^128 gives infinity, as it should); magnitudes below the
// smallest normal float give a signed zero (the FP32 kernels flush denormals
// anyway).  Outside the domain (|x| >= 2^128, infinities, NaN) the exponent
// wraps and the result is meaningless: callers pass only positions, position
// offsets, masses and quadrupole components of inputs checked against
// kMaxInput (a rejected input's values are rounded all the same, harmlessly,
// before the call reports it).  On
// this GPU the hardware double->float conversion issues on the narrow FP64
// pipe, which this keeps free for the FP64 centring itself.
__host__ __device__ inline float f64_to_f32_rn(double x) {
#ifdef __CUDA_ARCH__
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &x, sizeof b);
#endif
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  unsigned t = (hi << 3) | (lo >> 29);       // low 9 exponent bits | 23 fraction bits
  t -= 384u << 23;                           // exponent - 896 (mod 512): 1023 -> 127 bias
  const unsigned r = lo & 0x1fffffffu;       // the 29 dropped fraction bits
  t += (r + (t & 1u) + 0x0fffffffu) >> 29;   // round half to even (a carry bumps the exponent)
  t = ((hi & 0x7ff00000u) < (897u << 20)) ? 0u : t;  // below the smallest normal float
  t |= hi & 0x80000000u;                     // sign
#ifdef __CUDA_ARCH__
  return __uint_as_float(t);
#else
  float f;
  __builtin_memcpy(&f, &t, sizeof f);
  return f;
#endif
}

// The same entry for the centred FP32 kernels: every coordinate as a pair of
// floats, hi = the float nearest x and lo = the float nearest x - hi (about
// 48 bits of x together), and the mass as float: one aligned 32-byte sector.
// Centring on c = (hi_c, lo_c) is then (hi - hi_c) + (lo - lo_c): three FP32
// adds, exact in its first step wherever the entry is near the centre.
struct __align__(32) PosMassF {
  float hx, hy, hz, m;
  float lx, ly, lz, pad;
};

// x as hi + lo, both rounded to nearest with the integer rounding above (on
// the GPU the hardware double -> float conversion issues on the narrow FP64
// pipe; this needs one FP64 subtraction).  A result below the smallest normal
// float becomes 0, which the FP32 kernels (built to flush denormals) would
// make of it anyway.
__host__ __device__ inline void split_f32x2(double x, float &hi, float &lo) {
  hi = f64_to_f32_rn(x);
  lo = f64_to_f32_rn(x - (double)hi);
}

__host__ __device__ inline PosMassF make_posmassf(double x, double y, double z, float m) {
  PosMassF r;
  split_f32x2(x, r.hx, r.lx);
  split_f32x2(y, r.hy, r.ly);
  split_f32x2(z, r.hz, r.lz);
  r.m = m;
  r.pad = 0.f;
  return r;
}

// One work item of a step whose long lists are split (the modified tree
// algorithm's group x list, Sec. 3.4, cut into parts): group g, entries
// [e0, e1) of its list taken as its particle entries followed by its cell
// entries.  part = -1: the whole list (the group's results are written
// directly).  part = k of nparts: the item writes FP64 partial sums of its
// range for every sink of g to partial[slot + i] (slot = the group's first
// slot + k n_i), counts itself in done[ctr], and the item that completes the
// count adds the parts of every sink in the order k = 0, 1, ... and writes
// the results (bitwise repeatable whichever part finishes last).
struct Item {
  int32_t g;
  int32_t part;
  int32_t nparts;
  int32_t ctr;
  int64_t e0, e1;
  int64_t slot;
};

// Device pointers and sizes one force launch reads.  Layouts:
//   sink_x    [n][3] double           sink_eps2 [n] float or null
//   group_off [G+1]                   queue     [nitems] group ids
//   src       [ns] PosMass (x, y, z double; m float)   src_m64  [ns] double m
//   cell_pm   [nc] PosMass (x, y, z double; m float)   cell_m64 [nc] double m
//   cell_q    [nc][2] float4 ((q00, q01, q02, q11), (q12, q22, 0, 0))
//   cell_q64  [nc][6] double (q00 q01 q02 q11 q12 q22)
// The FP32 kernels read PosMass and cell_q (two 32-byte sectors per cell);
// the all-FP64 kernel reads the positions of PosMass and the *_m64 / q64
// arrays.
//   a         [n][3] double           phi [n] double
struct ForceParams {
  const double *sink_x;
  const float *sink_eps2;
  double eps2_all;
  float eps2_all_f;  // eps2_all rounded to float on the host (FP32 kernels)
  const int64_t *group_off;
  const double *gcentre;  // [G][3] centre of each group's bounding box (centred kernels)
  // the same centres, sinks, sources and cells as float pairs (centred FP32 kernels)
  const PosMassF *gcentre_f;
  const PosMassF *sink_f;
  const PosMassF *src_f;
  const PosMassF *cell_f;
  const PosMass *src;
  const double *src_m64;
  // group g's particle list is plist_idx[plist_off[g] .. plist_end[g]) (CSR
  // lists: plist_end = plist_off + 1); the same for its cell list
  const int64_t *plist_off;
  const int64_t *plist_end;
  const int32_t *plist_idx;
  const PosMass *cell_pm;
  const double *cell_m64;
  const float4 *cell_q;
  const double *cell_q64;
  const int64_t *clist_off;
  const int64_t *clist_end;
  const int32_t *clist_idx;
  const int32_t *queue;
  int32_t nitems;
  int32_t *head;
  // Split lists (null: every queue entry is a group id, whole lists): the
  // queue holds indices into items; partial [slots][4] FP64 (a, phi) per
  // sink and part; done [split groups] completion counts (zero at launch).
  const Item *items;
  double *partial;
  int *done;
  double *a;
  double *phi;
  // In-place kernels only (lists read from host memory): every index is
  // checked against n_src / n_cell as it is read (an entry outside its
  // array sets *bad and reads entry 0) and the checked index is written to
  // the keep array (device) at the same position, so the device ends up
  // holding the whole list.
  int32_t *plist_keep;
  int32_t *clist_keep;
  int32_t n_src, n_cell;
  int *bad;
  // In-place kernels only: the results' second copy, in host memory.
  double *a_host;
  double *phi_host;
  int32_t tile;     // list entries per shared-memory tile
  int32_t flush_j;  // entries per thread between FP32 -> FP64 folds
  float zero, one;  // 0 and 1, as runtime values (see Pair2 in qg_force.cuh)
};

// Dynamic shared memory of one force CTA: the FP64 accumulators [4R][nthreads]
// (the sink offsets, R * nthreads 4-vectors of Real, never larger, alias
// them) and one tile of staged list entries.
inline size_t force_smem_bytes(bool fp64, bool paired, int R, int nthreads, int tile) {
  const size_t per_entry = paired ? 5 * 16                   // (dx dx dy dy) (dz dz m m) + 3 for -Q
                                  : (fp64 ? 2 * 32 + 16 : 2 * 16 + 8);  // A, B 4-vectors, C 2-vector
  return (size_t)nthreads * 4 * R * 8 + (size_t)tile * per_entry;
}

// Kernel registry (one function per translation unit that instantiates it).
// Returns nullptr for an unsupported combination.
const void *force_kernel_f32(int R, bool quad, bool guard, bool centred);
const void *force_kernel_f32x2(int R, bool quad, bool guard);
const void *force_kernel_f32ep(int R, bool quad, bool guard);  // entry-paired FP32 centred
const void *force_kernel_f64(int R, bool quad, bool guard);
const void *force_kernel_inplace(int R, bool quad, bool guard, bool epaired);  // FP32 centred
// FP32 centred, sinks per thread chosen per work item (1 to 4); scalar or entry-paired
const void *force_kernel_adapt(bool epaired, bool quad, bool guard);
const void *force_kernel_inplace_adapt(bool epaired, bool quad, bool guard);

}  // namespace qg
