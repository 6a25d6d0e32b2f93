// qg_force.cuh -- the persistent group-force kernel (monopole particles +
// quadrupole cells, Kodama & Ishiyama arXiv:1812.07313, Eqs. 1, 4-7).
//
// One CTA evaluates one sink group at a time, taking group ids from a
// device work queue (ordered by descending cost) with an atomic counter.
// Inside the CTA:
//   1. c_g = centre of the bounding box of the group's sinks (FP64, computed
//      once per set of sinks by group_centre_kernel, and stored also as a
//      float-pair record).
//   2. sink offsets x_i - c_g are formed from the float-pair records (FP32
//      kernels) or in FP64 (the all-FP64 kernel), kept in shared memory;
//      each thread holds R sinks in registers.
//   3. the group's list is staged tile by tile into shared memory:
//      particles (x_j - c_g, m) and cells (x_j - c_g, m, Q) gathered through
//      the group's index range [off[g], end[g]) (CSR lists have end = off + 1)
//      and centred the same way.
//   4. the threads form S sink slots x K list streams (S = ceil(n_i / R),
//      K = blockDim / S); stream k walks entries k, k+K, ... of each tile,
//      so every staged entry is read from shared memory once per thread and
//      used for R sinks.
//   5. Real partial sums are folded into accumulators in shared memory
//      (float-float in the FP32 scalar and entry-paired forms, FP64 in the
//      others) after at most flush_j entries per thread; at the end the K
//      streams of each sink are merged in a fixed order (deterministic) and
//      written in FP64.
//
// Real = float is the production path; Real = double is the all-FP64
// comparison kernel (same structure, no casts).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qg_internal.h"

namespace qg {

template <typename Real> struct RT;
template <> struct RT<float> {
  using v4 = float4;
  using v2 = float2;
  static __device__ __forceinline__ v4 make4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
  static __device__ __forceinline__ v2 make2(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ float cvt(double x) { return f64_to_f32_rn(x); }
  // SFU approximate reciprocal square root (MUFU.RSQ)
  static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
};
template <> struct RT<double> {
  using v4 = double4_16a;  // shared memory only guarantees 16-byte alignment
  using v2 = double2;
  static __device__ __forceinline__ v4 make4(double a, double b, double c, double d) { return make_double4_16a(a, b, c, d); }
  static __device__ __forceinline__ v2 make2(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ double cvt(double x) { return x; }
  static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / sqrt(x); }
};

// Staging choices, fixed at compile time:
//   QG_CVT_HW  centred offsets rounded to FP32 by the hardware conversion for
//              the first QG_CVT_HW coordinates (it issues on the narrow FP64
//              pipe), by integer operations for the rest (ALU pipe);
//   QG_GATHER2 each thread keeps two list entries' gathers in flight before
//              converting either;
//   QG_EP_UNROLL unroll of the entry-paired pair loops.
#ifndef QG_CVT_HW
#define QG_CVT_HW 0
#endif
#ifndef QG_GATHER2
#define QG_GATHER2 1
#endif
#ifndef QG_EP_UNROLL
#define QG_EP_UNROLL 1
#endif
// #pragma unroll does not expand macros: the unroll count goes through _Pragma
#define QG_PRAGMA_(x) _Pragma(#x)
#define QG_UNROLL(n) QG_PRAGMA_(unroll n)

template <typename Real, int K>
__device__ __forceinline__ Real cvt_off(double v) {
  if constexpr (sizeof(Real) == 4) {
    if constexpr (K < QG_CVT_HW) return __double2float_rn(v);
    else return f64_to_f32_rn(v);
  } else {
    return v;
  }
}

// Group centre for the staging: FP64 (x, y, z) and, for the centred FP32
// kernels, the same centre as float pairs.
struct Centre {
  double x, y, z;
  float hx, hy, hz, lx, ly, lz;
};

// Centred offset of an entry: FP64 subtraction, then rounded to Real ...
template <typename Real>
__device__ __forceinline__ void centred(const PosMass &v, const Centre &c, Real &dx, Real &dy, Real &dz) {
  dx = cvt_off<Real, 0>(v.x - c.x);
  dy = cvt_off<Real, 1>(v.y - c.y);
  dz = cvt_off<Real, 2>(v.z - c.z);
}
// ... or from float pairs: (hi - hi_c) + (lo - lo_c), the same operations for
// a sink and for its own list entry, so that its self pair has offset 0
template <typename Real>
__device__ __forceinline__ void centred(const PosMassF &v, const Centre &c, Real &dx, Real &dy, Real &dz) {
  dx = (v.hx - c.hx) + (v.lx - c.lx);
  dy = (v.hy - c.hy) + (v.ly - c.ly);
  dz = (v.hz - c.hz) + (v.lz - c.lz);
}

// One source particle on one sink: Eq. 4 and its gradient.  13 Real ops + 1 rsqrt.
template <typename Real, bool GUARD>
__device__ __forceinline__ void mono_pair(Real dx, Real dy, Real dz, Real m, Real e2,
                                          Real &ax, Real &ay, Real &az, Real &pot) {
  const Real r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, e2)));
  Real ri = RT<Real>::rsqrt(r2);
  if (GUARD) ri = r2 > Real(0) ? ri : Real(0);
  const Real pm = m * ri;            // phi_mono = m / rhat
  pot += pm;
  const Real c = pm * (ri * ri);     // m / rhat^3
  ax = fma(c, dx, ax);
  ay = fma(c, dy, ay);
  az = fma(c, dz, az);
}

// One cell on one sink: Eqs. 1, 4-5 and -grad of Eq. 1.  33 Real ops + 1 rsqrt.
// q = (q00, q01, q02, q11), qq = (q12, q22).
template <typename Real, bool GUARD>
__device__ __forceinline__ void quad_pair(Real dx, Real dy, Real dz, Real m,
                                          Real q00, Real q01, Real q02, Real q11, Real q12, Real q22,
                                          Real e2, Real &ax, Real &ay, Real &az, Real &pot) {
  const Real r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, e2)));
  Real ri = RT<Real>::rsqrt(r2);
  if (GUARD) ri = r2 > Real(0) ? ri : Real(0);
  const Real ri2 = ri * ri;
  const Real pm = m * ri;                                  // phi_mono
  const Real qx = fma(q00, dx, fma(q01, dy, q02 * dz));    // (Q r)_x
  const Real qy = fma(q01, dx, fma(q11, dy, q12 * dz));    // (Q r)_y
  const Real qz = fma(q02, dx, fma(q12, dy, q22 * dz));    // (Q r)_z
  const Real rqr = fma(dx, qx, fma(dy, qy, dz * qz));      // r.Q.r
  const Real ri5 = ri2 * ri2 * ri;
  const Real u = rqr * ri5;                                // 2 phi_quad
  pot += pm;
  pot = fma(Real(0.5), u, pot);                            // + phi_quad
  const Real c = fma(Real(2.5), u, pm) * ri2;              // (phi_mono + 5 phi_quad) / rhat^2
  ax = fma(c, dx, ax);
  ax = fma(-ri5, qx, ax);
  ay = fma(c, dy, ay);
  ay = fma(-ri5, qy, ay);
  az = fma(c, dz, az);
  az = fma(-ri5, qz, az);
}

// Paired FP32 forms: two sinks per float2 and Blackwell's f32x2 instructions,
// one instruction issue per two lanes of work.  On this GPU the paired FMA
// runs at the full FP32 rate but the paired add and multiply at half of it,
// so every add and multiply is written as an FMA (a*b = fma(a, b, 0),
// a + b = fma(a, 1, b): the same single rounding).  Operands: j-entry values
// broadcast to both halves, (nx, ny, nz) the two sinks' offsets negated, so
// that every sign folds into the instructions.  13 and 33 paired FMAs per
// two pairs, as in the scalar forms.  The 0 and 1 operands come from the
// kernel's parameters (ForceParams::zero2, one2): as compile-time constants
// the compiler would fold the FMA back into the half-rate add or multiply.
// Position of the padding entry of the entry-paired form (an odd list tail):
// far enough that rhat^-5 underflows to zero, near enough that rhat^2 stays
// finite in FP32.
constexpr float kPadFar = 1.0e15f;

// Throughput of the pair loop at r = 1 ... 4 sinks per thread relative to the
// FP32 peak, measured on this GPU with the loop alone over a shared-memory
// tile (quadrupole, entry-paired, 64-thread CTAs, 8 per SM as for the R = 4
// kernel): the weights of choose_sinks_per_thread.
constexpr float kLoopEff1 = 0.746f, kLoopEff2 = 0.807f, kLoopEff3 = 0.824f, kLoopEff4 = 0.844f;

// Float-float running sums (hi, lo): hi holds the rounded sum and lo the
// rounding errors of every addition, each found exactly by Knuth's TwoSum
// (The Art of Computer Programming, vol. 2, 4.2.2), so hi + lo carries
// about 48 significant bits.  The FP32 kernels fold their partial sums into
// these instead of FP64 accumulators: six FP32 adds in place of a conversion
// and an add on the FP64 pipe, which issues at about 1/64 of the FP32 rate
// on this GPU.  The kernels are built with FTZ, so a sum below 2^-126 keeps
// FP32 precision only.
__device__ __forceinline__ float2 ff_add(float2 v, float x) {
  const float s = v.x + x;
  const float b = s - v.x;
  const float e = (v.x - (s - b)) + (x - b);
  return make_float2(s, v.y + e);
}
__device__ __forceinline__ float2 ff_add(float2 v, float2 w) {
  const float s = v.x + w.x;
  const float b = s - v.x;
  const float e = (v.x - (s - b)) + (w.x - b);
  return make_float2(s, (v.y + w.y) + e);
}
__device__ __forceinline__ double ff_value(float2 v) { return (double)v.x + (double)v.y; }

struct Pair2 {
  float2 zero, one, mone;
  __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) const { return __ffma2_rn(a, b, c); }
  __device__ __forceinline__ float2 mul2(float2 a, float2 b) const { return __ffma2_rn(a, b, zero); }
  __device__ __forceinline__ float2 add2(float2 a, float2 b) const { return __ffma2_rn(a, one, b); }
};

template <bool GUARD>
__device__ __forceinline__ void mono_pair2(const Pair2 &P, float2 jx, float2 jy, float2 jz, float2 jm, float2 nx,
                                           float2 ny, float2 nz, float2 e2, float2 &ax, float2 &ay, float2 &az,
                                           float2 &pot) {
  const float2 dx = P.add2(jx, nx), dy = P.add2(jy, ny), dz = P.add2(jz, nz);
  const float2 r2 = P.fma2(dx, dx, P.fma2(dy, dy, P.fma2(dz, dz, e2)));
  float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
  if (GUARD) {
    ri.x = r2.x > 0.f ? ri.x : 0.f;
    ri.y = r2.y > 0.f ? ri.y : 0.f;
  }
  const float2 pm = P.mul2(jm, ri);             // phi_mono
  pot = P.add2(pot, pm);
  const float2 c = P.mul2(pm, P.mul2(ri, ri));    // m / rhat^3
  ax = P.fma2(c, dx, ax);
  ay = P.fma2(c, dy, ay);
  az = P.fma2(c, dz, az);
}

// nq00..nq22 = -(q00, q01, q02, q11, q12, q22): with Q negated, nQ r = -(Q r)
// and r.nQ.r = -(r.Q.r), so a += c r + rhat^-5 nQ r needs no negation.
template <bool GUARD>
__device__ __forceinline__ void quad_pair2(const Pair2 &P, float2 jx, float2 jy, float2 jz, float2 jm,
                                           float2 nq00, float2 nq01,
                                           float2 nq02, float2 nq11, float2 nq12, float2 nq22, float2 nx,
                                           float2 ny, float2 nz, float2 e2, float2 &ax, float2 &ay, float2 &az,
                                           float2 &pot) {
  const float2 dx = P.add2(jx, nx), dy = P.add2(jy, ny), dz = P.add2(jz, nz);
  const float2 r2 = P.fma2(dx, dx, P.fma2(dy, dy, P.fma2(dz, dz, e2)));
  float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
  if (GUARD) {
    ri.x = r2.x > 0.f ? ri.x : 0.f;
    ri.y = r2.y > 0.f ? ri.y : 0.f;
  }
  const float2 ri2 = P.mul2(ri, ri);
  const float2 pm = P.mul2(jm, ri);                                     // phi_mono
  const float2 qx = P.fma2(nq00, dx, P.fma2(nq01, dy, P.mul2(nq02, dz)));   // -(Q r)_x
  const float2 qy = P.fma2(nq01, dx, P.fma2(nq11, dy, P.mul2(nq12, dz)));   // -(Q r)_y
  const float2 qz = P.fma2(nq02, dx, P.fma2(nq12, dy, P.mul2(nq22, dz)));   // -(Q r)_z
  const float2 rqr = P.fma2(dx, qx, P.fma2(dy, qy, P.mul2(dz, qz)));        // -(r.Q.r)
  const float2 ri5 = P.mul2(P.mul2(ri2, ri2), ri);
  const float2 u = P.mul2(rqr, ri5);                                    // -2 phi_quad
  pot = P.add2(pot, pm);
  pot = P.fma2(make_float2(-0.5f, -0.5f), u, pot);                      // + phi_quad
  const float2 c = P.mul2(P.fma2(make_float2(-2.5f, -2.5f), u, pm), ri2); // (phi_mono + 5 phi_quad)/rhat^2
  ax = P.fma2(c, dx, ax);
  ax = P.fma2(ri5, qx, ax);
  ay = P.fma2(c, dy, ay);
  ay = P.fma2(ri5, qy, ay);
  az = P.fma2(c, dz, az);
  az = P.fma2(ri5, qz, az);
}

// Entry-paired FP32 forms: two list entries per float2 (the halves of every
// j-value are two different entries, read as they were staged), each sink's
// values broadcast to both halves once per group.  The offset is taken the
// other way round, d = x_i - x_j = -r, and the staged mass is negated,
// nm = -m: then Q d = -(Q r), d.Q.d = r.Q.r, and every sign of Eq. 7 folds
// into an FMA with no negation in the loop.  pot accumulates the physical
// potential, -(phi_mono + phi_quad), directly.  13 and 33 paired FMAs (and two
// rsqrt) per two pairs, as in the scalar forms; the -1, 0 and 1 operands are
// runtime values (see Pair2).
template <bool GUARD>
__device__ __forceinline__ void mono_pairE(const Pair2 &P, float2 jx, float2 jy, float2 jz, float2 nm, float2 sx,
                                           float2 sy, float2 sz, float2 e2, float2 &ax, float2 &ay, float2 &az,
                                           float2 &pot) {
  const float2 dx = P.fma2(jx, P.mone, sx), dy = P.fma2(jy, P.mone, sy), dz = P.fma2(jz, P.mone, sz);  // -r
  const float2 r2 = P.fma2(dx, dx, P.fma2(dy, dy, P.fma2(dz, dz, e2)));
  float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
  if (GUARD) {
    ri.x = r2.x > 0.f ? ri.x : 0.f;
    ri.y = r2.y > 0.f ? ri.y : 0.f;
  }
  const float2 npm = P.mul2(nm, ri);             // -phi_mono
  pot = P.add2(pot, npm);
  const float2 c = P.mul2(npm, P.mul2(ri, ri));  // -m / rhat^3
  ax = P.fma2(c, dx, ax);
  ay = P.fma2(c, dy, ay);
  az = P.fma2(c, dz, az);
}

template <bool GUARD>
__device__ __forceinline__ void quad_pairE(const Pair2 &P, float2 jx, float2 jy, float2 jz, float2 nm, float2 q00,
                                           float2 q01, float2 q02, float2 q11, float2 q12, float2 q22, float2 sx,
                                           float2 sy, float2 sz, float2 e2, float2 &ax, float2 &ay, float2 &az,
                                           float2 &pot) {
  const float2 dx = P.fma2(jx, P.mone, sx), dy = P.fma2(jy, P.mone, sy), dz = P.fma2(jz, P.mone, sz);  // -r
  const float2 r2 = P.fma2(dx, dx, P.fma2(dy, dy, P.fma2(dz, dz, e2)));
  float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
  if (GUARD) {
    ri.x = r2.x > 0.f ? ri.x : 0.f;
    ri.y = r2.y > 0.f ? ri.y : 0.f;
  }
  const float2 ri2 = P.mul2(ri, ri);
  const float2 npm = P.mul2(nm, ri);                                       // -phi_mono
  const float2 qx = P.fma2(q00, dx, P.fma2(q01, dy, P.mul2(q02, dz)));    // -(Q r)_x
  const float2 qy = P.fma2(q01, dx, P.fma2(q11, dy, P.mul2(q12, dz)));    // -(Q r)_y
  const float2 qz = P.fma2(q02, dx, P.fma2(q12, dy, P.mul2(q22, dz)));    // -(Q r)_z
  const float2 rqr = P.fma2(dx, qx, P.fma2(dy, qy, P.mul2(dz, qz)));       // r.Q.r
  const float2 ri5 = P.mul2(P.mul2(ri2, ri2), ri);
  const float2 u = P.mul2(rqr, ri5);                                       // 2 phi_quad
  pot = P.add2(pot, npm);
  pot = P.fma2(make_float2(-0.5f, -0.5f), u, pot);                         // - phi_quad
  const float2 c = P.mul2(P.fma2(make_float2(-2.5f, -2.5f), u, npm), ri2); // -(phi_mono + 5 phi_quad)/rhat^2
  ax = P.fma2(c, dx, ax);
  ax = P.fma2(ri5, qx, ax);
  ay = P.fma2(c, dy, ay);
  ay = P.fma2(ri5, qy, ay);
  az = P.fma2(c, dz, az);
  az = P.fma2(ri5, qz, az);
}

// A list index is read once per launch: the streaming (evict-first) load keeps
// the index stream from pushing the gathered records out of L2.  Likewise the
// results, written once, go out with streaming stores.
__device__ __forceinline__ int ld_index(const int32_t *q) { return __ldcs(q); }
__device__ __forceinline__ void st_result(double *q, double v) { __stcs(q, v); }

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// A list index read in place from host memory: checked against its array
// (an entry outside it counts in *bad and becomes 0, a valid record) and
// kept on the device at its list position.
__device__ __forceinline__ int keep_index(int j, int lim, int32_t *keep, int *bad) {
  if ((unsigned)j >= (unsigned)lim) {
    atomicOr(bad, 1);
    j = 0;
  }
  *keep = j;
  return j;
}

// Arithmetic forms of the FP32 kernel: scalar, sink-paired (two sinks per
// float2, j-values broadcast) and entry-paired (two list entries per float2,
// sink values broadcast).
enum : int { kScalar = 0, kSinkPaired = 1, kEntryPaired = 2 };

// Launch bounds per variant: the largest block it is launched with and the
// CTAs per SM the register budget must allow.  Scalar R <= 4: 3 blocks of 256
// threads leaves 80 registers a thread (72 used at R = 2), which still fits
// the six 128-thread CTAs that shared memory allows per SM (64 registers
// measured 2-3 % slower); the paired R = 4 forms carry twice the registers per
// sink (or per j-entry) and get up to 128; R = 8 keeps 8 sinks x 4 sums in
// registers and is limited to 128 threads; the all-FP64 comparison form gets
// up to 128.
template <typename Real, int R, int FORM> struct Bounds {
  static constexpr int threads = R >= 8 ? 128 : 256;
  static constexpr int min_blocks = (R >= 8 || sizeof(Real) == 8 || (FORM != kScalar && R >= 4)) ? 2 : 3;
};

// The sink chunks of one work item (group g's sinks [s0, s0 + ni), its list
// entries [p0, p1) and [c0, c1)) at R sinks per thread: sink staging, list
// tiles, pair loops, folds, the fixed-order merge of the K streams and the outputs
// (or, for a part of a split list, its partial sums at slot).  Rtile is the R
// the shared memory was laid out for (the tile follows the 8-byte
// accumulators of Rtile sinks per thread).
template <typename Real, int R, bool QUAD, bool GUARD, bool CENTRED, int FORM, bool INPLACE>
__device__ __forceinline__ void evaluate_chunks(const ForceParams &p, unsigned char *smem_raw, const int Rtile,
                                                const Centre &cc, const int64_t s0, const int ni, const int64_t p0,
                                                const int64_t p1, const int64_t c0, const int64_t c1, const int part,
                                                const int64_t slot) {
  constexpr bool PAIRED = FORM == kSinkPaired;
  constexpr bool EPAIR = FORM == kEntryPaired;
  constexpr bool FF = sizeof(Real) == 4 && CENTRED;
  constexpr int H = R / 2;               // sink pairs per thread (sink-paired form)
  constexpr int NE = EPAIR ? R : 1;      // broadcast sinks per thread (entry-paired form)
  constexpr bool keep = INPLACE;
  const Pair2 P2{make_float2(p.zero, p.zero), make_float2(p.one, p.one), make_float2(-p.one, -p.one)};
  using V4 = typename RT<Real>::v4;
  using V2 = typename RT<Real>::v2;
  const int NT = blockDim.x;
  const int tid = threadIdx.x;
  const int T = p.tile;
  // acc64 [4R][NT] (value-major, so that a warp's accesses are consecutive);
  // sink_s aliases it: the sink offsets are read into registers before the
  // accumulators are zeroed.  The FP32 scalar and entry-paired forms keep
  // float-float sums there (accF, 8 bytes each like a double); the
  // sink-paired and all-FP64 forms keep FP64 sums.
  constexpr bool FFACC = sizeof(Real) == 4 && !PAIRED;
  double *acc64 = reinterpret_cast<double *>(smem_raw);
  float2 *accF = reinterpret_cast<float2 *>(smem_raw);
  V4 *sink_s = reinterpret_cast<V4 *>(smem_raw);
  // Staged tile.  Scalar form: A (dx dy dz m), B (q00 q01 q02 q11), C (q12 q22).
  // Sink-paired form: every value twice, (dx dx dy dy) (dz dz m m) and the
  // negated quadrupole (q00 q00 q01 q01) (q02 q02 q11 q11) (q12 q12 q22 q22).
  // Entry-paired form: entries 2u and 2u+1 side by side in pair u,
  // (dx dx' dy dy') (dz dz' -m -m') (q00 q00' q01 q01') (q02 q02' q11 q11')
  // (q12 q12' q22 q22'): 40 bytes per entry, as in the scalar form.
  double *tile = acc64 + 4 * Rtile * NT;
  V4 *tA = reinterpret_cast<V4 *>(tile);
  V4 *tB = tA + T;
  V2 *tC = reinterpret_cast<V2 *>(tB + T);
  float4 *tP0 = reinterpret_cast<float4 *>(tile);
  float4 *tP1 = tP0 + T;
  float4 *tQ0 = tP1 + T;
  float4 *tQ1 = tQ0 + T;
  float4 *tQ2 = tQ1 + T;
  float4 *tE0 = reinterpret_cast<float4 *>(tile);
  float4 *tE1 = tE0 + T / 2;
  float4 *tE2 = tE1 + T / 2;
  float4 *tE3 = tE2 + T / 2;
  float4 *tE4 = tE3 + T / 2;

    // ---- sink chunks of at most R * NT sinks --------------------------------
    for (int sb = 0; sb < ni; sb += R * NT) {
      const int nch = min(ni - sb, R * NT);
      __syncthreads();  // previous chunk's readers of sink_s / acc64 are done
      for (int i = tid; i < nch; i += NT) {
        const int64_t si = s0 + sb + i;
        // softening: the per-sink array is float already; the global value
        // was rounded to float on the host (FP32) or is used as given (FP64)
        Real e2;
        if constexpr (sizeof(Real) == 4) e2 = p.sink_eps2 ? p.sink_eps2[si] : p.eps2_all_f;
        else e2 = p.sink_eps2 ? (double)p.sink_eps2[si] : p.eps2_all;
        Real dx, dy, dz;
        if constexpr (FF) {
          centred<Real>(p.sink_f[si], cc, dx, dy, dz);
        } else {
          const double *xi = p.sink_x + 3 * si;
          dx = RT<Real>::cvt(xi[0] - cc.x);
          dy = RT<Real>::cvt(xi[1] - cc.y);
          dz = RT<Real>::cvt(xi[2] - cc.z);
        }
        sink_s[i] = RT<Real>::make4(dx, dy, dz, e2);
      }
      __syncthreads();

      const int S = (nch + R - 1) / R;  // sink slots
      const int K = NT / S;             // list streams
      // tiles hold a whole number of passes of the K streams, so that no
      // tile ends in a partly filled pass (only the list's last tile may);
      // in the entry-paired form a stream takes two entries per pass
      const int TK = EPAIR ? 2 * (T / 2 >= K ? (T / 2 / K) * K : T / 2) : (T >= K ? (T / K) * K : T);
      const int s = tid % S;
      const int k = tid / S;
      const bool active = k < K;

      Real sx[R], sy[R], sz[R], se[R];
      Real ax[R], ay[R], az[R], pt[R];
      float2 nx2[H > 0 ? H : 1], ny2[H > 0 ? H : 1], nz2[H > 0 ? H : 1], e22[H > 0 ? H : 1];
      float2 ax2[H > 0 ? H : 1], ay2[H > 0 ? H : 1], az2[H > 0 ? H : 1], pt2[H > 0 ? H : 1];
      float2 bsx[NE], bsy[NE], bsz[NE], bse[NE], bax[NE], bay[NE], baz[NE], bpt[NE];
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int i = s + S * r;
        const V4 v = sink_s[i < nch ? i : 0];
        sx[r] = v.x; sy[r] = v.y; sz[r] = v.z; se[r] = v.w;
        ax[r] = ay[r] = az[r] = pt[r] = Real(0);
      }
      if constexpr (PAIRED) {
#pragma unroll
        for (int h = 0; h < H; h++) {
          nx2[h] = make_float2(-sx[2 * h], -sx[2 * h + 1]);
          ny2[h] = make_float2(-sy[2 * h], -sy[2 * h + 1]);
          nz2[h] = make_float2(-sz[2 * h], -sz[2 * h + 1]);
          e22[h] = make_float2(se[2 * h], se[2 * h + 1]);
          ax2[h] = ay2[h] = az2[h] = pt2[h] = make_float2(0.f, 0.f);
        }
      }
      if constexpr (EPAIR) {
#pragma unroll
        for (int r = 0; r < R; r++) {
          bsx[r] = make_float2(sx[r], sx[r]);
          bsy[r] = make_float2(sy[r], sy[r]);
          bsz[r] = make_float2(sz[r], sz[r]);
          bse[r] = make_float2(se[r], se[r]);
          bax[r] = bay[r] = baz[r] = bpt[r] = make_float2(0.f, 0.f);
        }
      }
      __syncthreads();  // every thread holds its sinks: sink_s becomes acc64
#pragma unroll
      for (int v = 0; v < 4 * R; v++) {
        if constexpr (FFACC) accF[v * NT + tid] = make_float2(0.f, 0.f);
        else acc64[v * NT + tid] = 0.0;
      }
      int nproc = 0;

      auto fold = [&]() {
        if constexpr (PAIRED) {
#pragma unroll
          for (int h = 0; h < H; h++) {
            double *a = acc64 + 8 * h * NT + tid;  // sinks 2h and 2h + 1
            a[0] += (double)ax2[h].x;
            a[NT] += (double)ay2[h].x;
            a[2 * NT] += (double)az2[h].x;
            a[3 * NT] += (double)pt2[h].x;
            a[4 * NT] += (double)ax2[h].y;
            a[5 * NT] += (double)ay2[h].y;
            a[6 * NT] += (double)az2[h].y;
            a[7 * NT] += (double)pt2[h].y;
            ax2[h] = ay2[h] = az2[h] = pt2[h] = make_float2(0.f, 0.f);
          }
        } else if constexpr (EPAIR) {
          // the two halves (even and odd entries) of each sum added in FP32
          // -- together they cover at most flush_j entries, as one scalar
          // FP32 sum does -- then folded; the potential was accumulated with
          // the physical sign
#pragma unroll
          for (int r = 0; r < R; r++) {
            float2 *a = accF + 4 * r * NT + tid;
            a[0] = ff_add(a[0], bax[r].x + bax[r].y);
            a[NT] = ff_add(a[NT], bay[r].x + bay[r].y);
            a[2 * NT] = ff_add(a[2 * NT], baz[r].x + baz[r].y);
            a[3 * NT] = ff_add(a[3 * NT], -(bpt[r].x + bpt[r].y));
            bax[r] = bay[r] = baz[r] = bpt[r] = make_float2(0.f, 0.f);
          }
        } else if constexpr (FFACC) {
#pragma unroll
          for (int r = 0; r < R; r++) {
            float2 *a = accF + 4 * r * NT + tid;
            a[0] = ff_add(a[0], ax[r]);
            a[NT] = ff_add(a[NT], ay[r]);
            a[2 * NT] = ff_add(a[2 * NT], az[r]);
            a[3 * NT] = ff_add(a[3 * NT], pt[r]);
            ax[r] = ay[r] = az[r] = pt[r] = Real(0);
          }
        } else {
#pragma unroll
          for (int r = 0; r < R; r++) {
            double *a = acc64 + 4 * r * NT + tid;
            a[0] += (double)ax[r];
            a[NT] += (double)ay[r];
            a[2 * NT] += (double)az[r];
            a[3 * NT] += (double)pt[r];
            ax[r] = ay[r] = az[r] = pt[r] = Real(0);
          }
        }
        nproc = 0;
      };

      // The first two list indices this thread stages from the next tile are
      // loaded one tile ahead (during the current tile's arithmetic), so the
      // gather of a tile waits for one memory round trip instead of two.  The
      // in-place form, whose lists are in host memory (a round trip several
      // times longer), loads the first four ahead.
      int pf0 = -1, pf1 = -1, pf2 = -1, pf3 = -1;
      auto prefetch = [&](const int32_t *idx, int64_t b, int64_t end) {
        const int c = (int)min((int64_t)TK, end - b);
        // the entry-paired form stages entries 2 tid and 2 tid + 1 first
        // (then 2 tid + 2 NT and 2 tid + 2 NT + 1)
        const int e0 = EPAIR ? 2 * tid : tid, e1 = EPAIR ? 2 * tid + 1 : tid + NT;
        pf0 = e0 < c ? (INPLACE ? __ldg(idx + b + e0) : ld_index(idx + b + e0)) : -1;
        pf1 = e1 < c ? (INPLACE ? __ldg(idx + b + e1) : ld_index(idx + b + e1)) : -1;
        if constexpr (INPLACE) {
          const int e2 = EPAIR ? 2 * tid + 2 * NT : tid + 2 * NT, e3 = EPAIR ? 2 * tid + 2 * NT + 1 : tid + 3 * NT;
          pf2 = e2 < c ? __ldg(idx + b + e2) : -1;
          pf3 = e3 < c ? __ldg(idx + b + e3) : -1;
        }
      };
      // in-place forms: index of entry t of the tile at base, from the
      // registers loaded ahead where there is one
      auto ahead = [&](const int32_t *idx, int64_t base, int t) -> int {
        const int u = t - (EPAIR ? 2 * tid : tid);
        const int o1 = EPAIR ? 1 : NT, o2 = 2 * NT, o3 = EPAIR ? 2 * NT + 1 : 3 * NT;
        return u == 0 ? pf0 : u == o1 ? pf1 : u == o2 ? pf2 : u == o3 ? pf3 : idx[base + t];
      };
      if (p0 < p1) prefetch(p.plist_idx, p0, p1);
      else if (c0 < c1) prefetch(p.clist_idx, c0, c1);

      // ---- 3-4. particle part of the list (monopole, Eq. 4) ----------------
      for (int64_t base = p0; base < p1; base += TK) {
        const int cnt = (int)min((int64_t)TK, p1 - base);
        __syncthreads();  // the previous tile's readers are done
        auto put_p = [&](int t, const auto &v, int j) {
          const Real m = sizeof(Real) == 4 ? (Real)v.m : (Real)p.src_m64[j];
          Real dx, dy, dz;
          centred<Real>(v, cc, dx, dy, dz);
          if constexpr (PAIRED) {
            tP0[t] = make_float4(dx, dx, dy, dy);
            tP1[t] = make_float4(dz, dz, m, m);
          } else {
            tA[t] = RT<Real>::make4(dx, dy, dz, m);
          }
        };
        if constexpr (EPAIR) {
          // pair u = entries 2u and 2u + 1, both gathers in flight; an odd
          // last entry is paired with a massless entry far away (it adds
          // exactly zero: every term carries its mass, or rhat^-5 which
          // underflows to zero there)
          const int npair = (cnt + 1) >> 1;
          for (int u = tid; u < npair; u += NT) {
            const int t0 = 2 * u, t1 = t0 + 1;
            const bool first = u == tid;
            int j0, j1;
            if constexpr (INPLACE) {
              j0 = keep_index(ahead(p.plist_idx, base, t0), p.n_src, p.plist_keep + base + t0, p.bad);
              j1 = t1 < cnt ? keep_index(ahead(p.plist_idx, base, t1), p.n_src, p.plist_keep + base + t1, p.bad) : j0;
            } else {
              j0 = first ? pf0 : ld_index(p.plist_idx + base + t0);
              j1 = t1 < cnt ? (first ? pf1 : ld_index(p.plist_idx + base + t1)) : j0;
            }
            const PosMassF v0 = p.src_f[j0];
            const PosMassF v1 = p.src_f[j1];
            float dx0, dy0, dz0;
            centred<float>(v0, cc, dx0, dy0, dz0);
            float dx1 = kPadFar, dy1 = kPadFar, dz1 = kPadFar, m1 = 0.f;
            if (t1 < cnt) {
              centred<float>(v1, cc, dx1, dy1, dz1);
              m1 = v1.m;
            }
            tE0[u] = make_float4(dx0, dx1, dy0, dy1);
            tE1[u] = make_float4(dz0, dz1, -v0.m, -m1);
          }
        } else if constexpr (QG_GATHER2 != 0) {
          for (int t = tid; t < cnt; t += 2 * NT) {
            const int t1 = t + NT;
            [[maybe_unused]] const bool first = t == tid;
            int j0, j1;
            if constexpr (INPLACE) {
              j0 = ahead(p.plist_idx, base, t);
              j1 = t1 < cnt ? ahead(p.plist_idx, base, t1) : j0;
            } else {
              j0 = first ? pf0 : ld_index(p.plist_idx + base + t);
              j1 = t1 < cnt ? (first ? pf1 : ld_index(p.plist_idx + base + t1)) : j0;
            }
            if (keep) {
              j0 = keep_index(j0, p.n_src, p.plist_keep + base + t, p.bad);
              j1 = t1 < cnt ? keep_index(j1, p.n_src, p.plist_keep + base + t1, p.bad) : j0;
            }
            if constexpr (FF) {
              const PosMassF v0 = p.src_f[j0];
              const PosMassF v1 = p.src_f[j1];
              put_p(t, v0, j0);
              if (t1 < cnt) put_p(t1, v1, j1);
            } else {
              const PosMass v0 = p.src[j0];
              const PosMass v1 = p.src[j1];
              put_p(t, v0, j0);
              if (t1 < cnt) put_p(t1, v1, j1);
            }
          }
        } else {
          for (int t = tid; t < cnt; t += NT) {
            int j = INPLACE ? ahead(p.plist_idx, base, t) : t == tid ? pf0 : (t == tid + NT ? pf1 : ld_index(p.plist_idx + base + t));
            if (keep) j = keep_index(j, p.n_src, p.plist_keep + base + t, p.bad);
            if constexpr (FF) put_p(t, p.src_f[j], j);
            else put_p(t, p.src[j], j);
          }
        }
        if (base + TK < p1) prefetch(p.plist_idx, base + TK, p1);
        else if (c0 < c1) prefetch(p.clist_idx, c0, c1);
        __syncthreads();
        if (active) {
          if constexpr (PAIRED) {
#pragma unroll 2
            for (int jj = k; jj < cnt; jj += K) {
              const float4 P0 = tP0[jj], P1 = tP1[jj];
#pragma unroll
              for (int h = 0; h < H; h++)
                mono_pair2<GUARD>(P2, make_float2(P0.x, P0.y), make_float2(P0.z, P0.w), make_float2(P1.x, P1.y),
                                  make_float2(P1.z, P1.w), nx2[h], ny2[h], nz2[h], e22[h], ax2[h], ay2[h],
                                  az2[h], pt2[h]);
            }
            nproc += (cnt - k + K - 1) / K;
          } else if constexpr (EPAIR) {
            const int npair = (cnt + 1) >> 1;
QG_UNROLL(QG_EP_UNROLL)
            for (int uu = k; uu < npair; uu += K) {
              const float4 E0 = tE0[uu], E1 = tE1[uu];
#pragma unroll
              for (int r = 0; r < R; r++)
                mono_pairE<GUARD>(P2, make_float2(E0.x, E0.y), make_float2(E0.z, E0.w), make_float2(E1.x, E1.y),
                                  make_float2(E1.z, E1.w), bsx[r], bsy[r], bsz[r], bse[r], bax[r], bay[r],
                                  baz[r], bpt[r]);
            }
            nproc += 2 * ((npair - k + K - 1) / K);
          } else {
#pragma unroll 2
            for (int jj = k; jj < cnt; jj += K) {
              const V4 A = tA[jj];
#pragma unroll
              for (int r = 0; r < R; r++)
                mono_pair<Real, GUARD>(A.x - sx[r], A.y - sy[r], A.z - sz[r], A.w, se[r],
                                       ax[r], ay[r], az[r], pt[r]);
            }
            nproc += (cnt - k + K - 1) / K;
          }
          if (nproc >= p.flush_j) fold();
        }
      }

      // ---- 3-4. cell part of the list (Eq. 1 / Eq. 7, or monopole) --------
      for (int64_t base = c0; base < c1; base += TK) {
        const int cnt = (int)min((int64_t)TK, c1 - base);
        __syncthreads();  // the previous tile's readers are done
        auto put_c = [&](int t, const auto &v, int j, float4 q0, float4 q1) {
          const Real m = sizeof(Real) == 4 ? (Real)v.m : (Real)p.cell_m64[j];
          Real dx, dy, dz;
          centred<Real>(v, cc, dx, dy, dz);
          if constexpr (PAIRED) {
            tP0[t] = make_float4(dx, dx, dy, dy);
            tP1[t] = make_float4(dz, dz, m, m);
            if (QUAD) {
              tQ0[t] = make_float4(-q0.x, -q0.x, -q0.y, -q0.y);
              tQ1[t] = make_float4(-q0.z, -q0.z, -q0.w, -q0.w);
              tQ2[t] = make_float4(-q1.x, -q1.x, -q1.y, -q1.y);
            }
          } else {
            tA[t] = RT<Real>::make4(dx, dy, dz, m);
            if (QUAD) {
              if (sizeof(Real) == 4) {
                tB[t] = RT<Real>::make4(q0.x, q0.y, q0.z, q0.w);
                tC[t] = RT<Real>::make2(q1.x, q1.y);
              } else {
                const double *q = p.cell_q64 + 6 * (int64_t)j;
                tB[t] = RT<Real>::make4((Real)q[0], (Real)q[1], (Real)q[2], (Real)q[3]);
                tC[t] = RT<Real>::make2((Real)q[4], (Real)q[5]);
              }
            }
          }
        };
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (EPAIR) {
          // as for the particles: pair u = entries 2u and 2u + 1, an odd last
          // entry paired with a massless, quadrupole-free entry far away
          const int npair = (cnt + 1) >> 1;
          for (int u = tid; u < npair; u += NT) {
            const int t0 = 2 * u, t1 = t0 + 1;
            const bool first = u == tid;
            int j0, j1;
            if constexpr (INPLACE) {
              j0 = keep_index(ahead(p.clist_idx, base, t0), p.n_cell, p.clist_keep + base + t0, p.bad);
              j1 = t1 < cnt ? keep_index(ahead(p.clist_idx, base, t1), p.n_cell, p.clist_keep + base + t1, p.bad) : j0;
            } else {
              j0 = first ? pf0 : ld_index(p.clist_idx + base + t0);
              j1 = t1 < cnt ? (first ? pf1 : ld_index(p.clist_idx + base + t1)) : j0;
            }
            const PosMassF v0 = p.cell_f[j0];
            const PosMassF v1 = p.cell_f[j1];
            float4 a0 = zero4, b0 = zero4, a1 = zero4, b1 = zero4;
            if (QUAD) {
              a0 = p.cell_q[2 * j0];
              b0 = p.cell_q[2 * j0 + 1];
              a1 = p.cell_q[2 * j1];
              b1 = p.cell_q[2 * j1 + 1];
            }
            float dx0, dy0, dz0;
            centred<float>(v0, cc, dx0, dy0, dz0);
            float dx1 = kPadFar, dy1 = kPadFar, dz1 = kPadFar, m1 = 0.f;
            if (t1 < cnt) {
              centred<float>(v1, cc, dx1, dy1, dz1);
              m1 = v1.m;
            } else {
              a1 = b1 = zero4;
            }
            tE0[u] = make_float4(dx0, dx1, dy0, dy1);
            tE1[u] = make_float4(dz0, dz1, -v0.m, -m1);
            if (QUAD) {
              tE2[u] = make_float4(a0.x, a1.x, a0.y, a1.y);
              tE3[u] = make_float4(a0.z, a1.z, a0.w, a1.w);
              tE4[u] = make_float4(b0.x, b1.x, b0.y, b1.y);
            }
          }
        } else if constexpr (QG_GATHER2 != 0) {
          for (int t = tid; t < cnt; t += 2 * NT) {
            const int t1 = t + NT;
            [[maybe_unused]] const bool first = t == tid;
            int j0, j1;
            if constexpr (INPLACE) {
              j0 = ahead(p.clist_idx, base, t);
              j1 = t1 < cnt ? ahead(p.clist_idx, base, t1) : j0;
            } else {
              j0 = first ? pf0 : ld_index(p.clist_idx + base + t);
              j1 = t1 < cnt ? (first ? pf1 : ld_index(p.clist_idx + base + t1)) : j0;
            }
            if (keep) {
              j0 = keep_index(j0, p.n_cell, p.clist_keep + base + t, p.bad);
              j1 = t1 < cnt ? keep_index(j1, p.n_cell, p.clist_keep + base + t1, p.bad) : j0;
            }
            const bool fq = QUAD && sizeof(Real) == 4;
            const float4 a0 = fq ? p.cell_q[2 * j0] : zero4, b0 = fq ? p.cell_q[2 * j0 + 1] : zero4;
            const float4 a1 = fq ? p.cell_q[2 * j1] : zero4, b1 = fq ? p.cell_q[2 * j1 + 1] : zero4;
            if constexpr (FF) {
              const PosMassF v0 = p.cell_f[j0];
              const PosMassF v1 = p.cell_f[j1];
              put_c(t, v0, j0, a0, b0);
              if (t1 < cnt) put_c(t1, v1, j1, a1, b1);
            } else {
              const PosMass v0 = p.cell_pm[j0];
              const PosMass v1 = p.cell_pm[j1];
              put_c(t, v0, j0, a0, b0);
              if (t1 < cnt) put_c(t1, v1, j1, a1, b1);
            }
          }
        } else {
          for (int t = tid; t < cnt; t += NT) {
            int j = INPLACE ? ahead(p.clist_idx, base, t) : t == tid ? pf0 : (t == tid + NT ? pf1 : ld_index(p.clist_idx + base + t));
            if (keep) j = keep_index(j, p.n_cell, p.clist_keep + base + t, p.bad);
            const bool fq = QUAD && sizeof(Real) == 4;
            const float4 qa = fq ? p.cell_q[2 * j] : zero4, qb = fq ? p.cell_q[2 * j + 1] : zero4;
            if constexpr (FF) put_c(t, p.cell_f[j], j, qa, qb);
            else put_c(t, p.cell_pm[j], j, qa, qb);
          }
        }
        if (base + TK < c1) prefetch(p.clist_idx, base + TK, c1);
        __syncthreads();
        if (active) {
          if constexpr (PAIRED) {
            if (QUAD) {
#pragma unroll 2
              for (int jj = k; jj < cnt; jj += K) {
                const float4 P0 = tP0[jj], P1 = tP1[jj], Q0 = tQ0[jj], Q1 = tQ1[jj], Q2 = tQ2[jj];
#pragma unroll
                for (int h = 0; h < H; h++)
                  quad_pair2<GUARD>(P2, make_float2(P0.x, P0.y), make_float2(P0.z, P0.w), make_float2(P1.x, P1.y),
                                    make_float2(P1.z, P1.w), make_float2(Q0.x, Q0.y), make_float2(Q0.z, Q0.w),
                                    make_float2(Q1.x, Q1.y), make_float2(Q1.z, Q1.w), make_float2(Q2.x, Q2.y),
                                    make_float2(Q2.z, Q2.w), nx2[h], ny2[h], nz2[h], e22[h], ax2[h], ay2[h],
                                    az2[h], pt2[h]);
              }
            } else {
#pragma unroll 2
              for (int jj = k; jj < cnt; jj += K) {
                const float4 P0 = tP0[jj], P1 = tP1[jj];
#pragma unroll
                for (int h = 0; h < H; h++)
                  mono_pair2<GUARD>(P2, make_float2(P0.x, P0.y), make_float2(P0.z, P0.w), make_float2(P1.x, P1.y),
                                    make_float2(P1.z, P1.w), nx2[h], ny2[h], nz2[h], e22[h], ax2[h], ay2[h],
                                    az2[h], pt2[h]);
              }
            }
          } else if constexpr (EPAIR) {
            const int npair = (cnt + 1) >> 1;
            if (QUAD) {
QG_UNROLL(QG_EP_UNROLL)
              for (int uu = k; uu < npair; uu += K) {
                const float4 E0 = tE0[uu], E1 = tE1[uu], E2 = tE2[uu], E3 = tE3[uu], E4 = tE4[uu];
#pragma unroll
                for (int r = 0; r < R; r++)
                  quad_pairE<GUARD>(P2, make_float2(E0.x, E0.y), make_float2(E0.z, E0.w), make_float2(E1.x, E1.y),
                                    make_float2(E1.z, E1.w), make_float2(E2.x, E2.y), make_float2(E2.z, E2.w),
                                    make_float2(E3.x, E3.y), make_float2(E3.z, E3.w), make_float2(E4.x, E4.y),
                                    make_float2(E4.z, E4.w), bsx[r], bsy[r], bsz[r], bse[r], bax[r], bay[r],
                                    baz[r], bpt[r]);
              }
            } else {
QG_UNROLL(QG_EP_UNROLL)
              for (int uu = k; uu < npair; uu += K) {
                const float4 E0 = tE0[uu], E1 = tE1[uu];
#pragma unroll
                for (int r = 0; r < R; r++)
                  mono_pairE<GUARD>(P2, make_float2(E0.x, E0.y), make_float2(E0.z, E0.w), make_float2(E1.x, E1.y),
                                    make_float2(E1.z, E1.w), bsx[r], bsy[r], bsz[r], bse[r], bax[r], bay[r],
                                    baz[r], bpt[r]);
              }
            }
          } else if (QUAD) {
#pragma unroll 2
            for (int jj = k; jj < cnt; jj += K) {
              const V4 A = tA[jj];
              const V4 B = tB[jj];
              const V2 C = tC[jj];
#pragma unroll
              for (int r = 0; r < R; r++)
                quad_pair<Real, GUARD>(A.x - sx[r], A.y - sy[r], A.z - sz[r], A.w,
                                       B.x, B.y, B.z, B.w, C.x, C.y, se[r],
                                       ax[r], ay[r], az[r], pt[r]);
            }
          } else {
#pragma unroll 2
            for (int jj = k; jj < cnt; jj += K) {
              const V4 A = tA[jj];
#pragma unroll
              for (int r = 0; r < R; r++)
                mono_pair<Real, GUARD>(A.x - sx[r], A.y - sy[r], A.z - sz[r], A.w, se[r],
                                       ax[r], ay[r], az[r], pt[r]);
            }
          }
          // list entries this thread has added since its last fold (two per pass when entry-paired)
          nproc += EPAIR ? 2 * ((((cnt + 1) >> 1) - k + K - 1) / K) : (cnt - k + K - 1) / K;
          if (nproc >= p.flush_j) fold();
        }
      }

      // ---- 5. merge of the K streams, fixed order --------------------------
      // (float-float in the FP32 scalar and entry-paired forms, then one
      // conversion to FP64; FP64 in the others)
      if (active) fold();
      __syncthreads();
      auto merged = [&](int si, int ri, double &m0, double &m1, double &m2, double &m3) {
        if constexpr (FFACC) {
          float2 f0 = make_float2(0.f, 0.f), f1 = f0, f2 = f0, f3 = f0;
          for (int kk = 0; kk < K; kk++) {
            const float2 *a = accF + 4 * ri * NT + kk * S + si;
            f0 = ff_add(f0, a[0]); f1 = ff_add(f1, a[NT]); f2 = ff_add(f2, a[2 * NT]); f3 = ff_add(f3, a[3 * NT]);
          }
          m0 = ff_value(f0); m1 = ff_value(f1); m2 = ff_value(f2); m3 = ff_value(f3);
        } else {
          m0 = m1 = m2 = m3 = 0.0;
          for (int kk = 0; kk < K; kk++) {
            const double *a = acc64 + 4 * ri * NT + kk * S + si;
            m0 += a[0]; m1 += a[NT]; m2 += a[2 * NT]; m3 += a[3 * NT];
          }
        }
      };
      if constexpr (!INPLACE) {
        for (int i = tid; i < nch; i += NT) {
          const int si = i % S, ri = i / S;
          double m0, m1, m2, m3;
          merged(si, ri, m0, m1, m2, m3);
          const int64_t o = s0 + sb + i;
          if (part < 0) {
            st_result(p.a + 3 * o, m0);
            st_result(p.a + 3 * o + 1, m1);
            st_result(p.a + 3 * o + 2, m2);
            st_result(p.phi + o, -m3);  // physical potential, Eq. 1
          } else {            // this part's sums, merged below by the group's last part
            double *w = p.partial + 4 * (slot + sb + i);
            w[0] = m0;
            w[1] = m1;
            w[2] = m2;
            w[3] = m3;
          }
        }
      } else {
        // the same sums, written to the device and to host memory
        double m[R][3];  // sink i = tid + r NT
#pragma unroll
        for (int r = 0; r < R; r++) {
          const int i = tid + r * NT;
          m[r][0] = m[r][1] = m[r][2] = 0.0;
          if (i < nch) {
            const int si = i % S, ri = i / S;
            double m3;
            merged(si, ri, m[r][0], m[r][1], m[r][2], m3);
            const int64_t o = s0 + sb + i;
            p.phi[o] = -m3;
            p.phi_host[o] = -m3;
          }
        }
        // a[3o + c] through shared memory, so that consecutive threads write
        // consecutive words (host memory takes scattered 8-byte words at a
        // third of the rate of whole lines)
        __syncthreads();  // every thread has read acc64
        double *out = acc64;
#pragma unroll
        for (int r = 0; r < R; r++) {
          const int i = tid + r * NT;
          if (i < nch) {
            out[3 * i] = m[r][0];
            out[3 * i + 1] = m[r][1];
            out[3 * i + 2] = m[r][2];
          }
        }
        __syncthreads();
        double *ag = p.a + 3 * (s0 + sb), *ah = p.a_host + 3 * (s0 + sb);
        for (int t = tid; t < 3 * nch; t += NT) {
          const double v = out[t];
          ag[t] = v;
          ah[t] = v;
        }
      }
    }

}

// Sinks per thread for a work item when the kernel chooses it per item (1 to
// RMAX): the choice that keeps the FMA pipe busiest with useful pairs.  For
// each r, S = ceil(n/r) sink slots and K = NT/S streams leave S K threads
// active (whole warps of them issue), each running ceil(L/K) list entries
// (rounded up to pairs in the entry-paired form) of r sinks; the lane-cycles
// spent are weighed by the pair loop's throughput at r sinks per thread
// (isolated-loop measurements on this GPU).  Uniform across the CTA.
template <int RMAX, bool EPAIR>
__device__ __forceinline__ int choose_sinks_per_thread(int n, int64_t L, int NT) {
  constexpr float eff[5] = {1.f, kLoopEff1, kLoopEff2, kLoopEff3, kLoopEff4};
  int best = RMAX;
  float best_cost = 0.f;
  for (int r = RMAX; r >= 1; r--) {
    const int S = (n + r - 1) / r;
    if (S > NT && r < RMAX) continue;  // would need more sink chunks than the largest r
    const int Sc = min(S, NT);
    const int K = max(NT / Sc, 1);
    int64_t it = (L + K - 1) / K;
    if (EPAIR) it = (it + 1) & ~(int64_t)1;
    const int warps = (min(Sc * K, NT) + 31) / 32;
    const int chunks = (S + NT - 1) / NT;
    const float cost = (float)chunks * (float)warps * 32.f * (float)r * (float)it / eff[r];
    if (r == RMAX || cost < best_cost) {  // ties keep the larger r
      best = r;
      best_cost = cost;
    }
  }
  return best;
}

// INPLACE: the lists are read from host memory (checked and kept as they
// are read, ForceParams::plist_keep) and the results also written to host
// memory (ForceParams::a_host), a[] through shared memory so that a warp
// writes consecutive words.  A separate instantiation, so that the kernel
// the graph replays carries none of it.
// ADAPT: R is the largest number of sinks per thread, and every work item
// runs at the number from 1 to R that suits its group's size and list length
// (choose_sinks_per_thread); shared memory is laid out for R.
template <typename Real, int R, bool QUAD, bool GUARD, bool CENTRED, int FORM, bool INPLACE = false,
          bool ADAPT = false>
__global__ void __launch_bounds__(Bounds<Real, R, FORM>::threads, Bounds<Real, R, FORM>::min_blocks)
    force_kernel(const ForceParams p) {
  constexpr bool PAIRED = FORM == kSinkPaired;
  constexpr bool EPAIR = FORM == kEntryPaired;
  // centred FP32 kernels centre sinks and entries from their float-pair
  // records; the all-FP64 kernel from the FP64 positions
  constexpr bool FF = sizeof(Real) == 4 && CENTRED;
  static_assert(!PAIRED || (sizeof(Real) == 4 && R % 2 == 0), "paired arithmetic: FP32, even R");
  static_assert(!EPAIR || (sizeof(Real) == 4 && CENTRED), "entry-paired arithmetic: FP32 centred");
  static_assert(!INPLACE || !PAIRED, "in place: scalar or entry-paired form");
  static_assert(!ADAPT || (!PAIRED && R == 4), "sinks per thread chosen per item: up to 4, not sink-paired");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  __shared__ int s_last;  // split lists: this item completed its group's parts

  const int NT = blockDim.x;
  const int tid = threadIdx.x;

  for (;;) {
    __syncthreads();  // the previous group is finished with shared memory
    if (tid == 0) s_item = atomicAdd(p.head, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= p.nitems) break;
    const int q = p.queue[item];
    // the work item: a whole group, or one part of a split group's list
    // (entries [e0, e1) of its particle entries followed by its cell entries)
    int g = q, part = -1, nparts = 1, ctr = 0;
    int64_t e0 = 0, e1 = -1, slot = 0;
    if (p.items) {
      const Item it = p.items[q];
      g = it.g;
      part = it.part;
      nparts = it.nparts;
      ctr = it.ctr;
      e0 = it.e0;
      e1 = it.e1;
      slot = it.slot;
    }
    const int64_t s0 = p.group_off[g];
    const int ni = (int)(p.group_off[g + 1] - s0);
    constexpr bool keep = INPLACE;
    if (ni <= 0) {
      if (keep) {  // no sinks: the lists are only checked and kept
        for (int64_t e = p.plist_off[g] + tid; e < p.plist_end[g]; e += NT)
          keep_index(p.plist_idx[e], p.n_src, p.plist_keep + e, p.bad);
        for (int64_t e = p.clist_off[g] + tid; e < p.clist_end[g]; e += NT)
          keep_index(p.clist_idx[e], p.n_cell, p.clist_keep + e, p.bad);
      }
      continue;
    }

    // ---- 1. group centre: the bounding-box centre of the sinks, computed
    // once when the sinks were set (group_centre_kernel)
    Centre cc{};
    if constexpr (FF) {
      const PosMassF cf = p.gcentre_f[g];
      cc.hx = cf.hx; cc.hy = cf.hy; cc.hz = cf.hz;
      cc.lx = cf.lx; cc.ly = cf.ly; cc.lz = cf.lz;
    } else if (CENTRED) {
      cc.x = p.gcentre[3 * g];
      cc.y = p.gcentre[3 * g + 1];
      cc.z = p.gcentre[3 * g + 2];
    }

    const int64_t gp0 = p.plist_off[g], np_g = p.plist_end[g] - gp0;
    const int64_t gc0 = p.clist_off[g], nc_g = p.clist_end[g] - gc0;
    if (e1 < 0) e1 = np_g + nc_g;
    const int64_t p0 = gp0 + min(e0, np_g), p1 = gp0 + min(e1, np_g);
    const int64_t c0 = gc0 + max(e0 - np_g, (int64_t)0), c1 = gc0 + max(e1 - np_g, (int64_t)0);

    // ---- sink chunks: the staging, pair loops, folds, merges and outputs
    if constexpr (ADAPT) {
      const int r = choose_sinks_per_thread<R, EPAIR>(ni, (p1 - p0) + (c1 - c0), NT);
      if (r == 1)
        evaluate_chunks<Real, 1, QUAD, GUARD, CENTRED, FORM, INPLACE>(p, smem_raw, R, cc, s0, ni, p0, p1, c0, c1,
                                                                      part, slot);
      else if (r == 2)
        evaluate_chunks<Real, 2, QUAD, GUARD, CENTRED, FORM, INPLACE>(p, smem_raw, R, cc, s0, ni, p0, p1, c0, c1,
                                                                      part, slot);
      else if (r == 3)
        evaluate_chunks<Real, 3, QUAD, GUARD, CENTRED, FORM, INPLACE>(p, smem_raw, R, cc, s0, ni, p0, p1, c0, c1,
                                                                      part, slot);
      else
        evaluate_chunks<Real, R, QUAD, GUARD, CENTRED, FORM, INPLACE>(p, smem_raw, R, cc, s0, ni, p0, p1, c0, c1,
                                                                      part, slot);
    } else {
      evaluate_chunks<Real, R, QUAD, GUARD, CENTRED, FORM, INPLACE>(p, smem_raw, R, cc, s0, ni, p0, p1, c0, c1, part,
                                                                    slot);
    }

    // ---- a6. split lists: the part that completes its group's count adds
    // the parts' sums of every sink in the fixed order k = 0, 1, ... (no
    // part waits for another; the partial sums of other CTAs are read past
    // the L1, after the count that follows their writes)
    if constexpr (!INPLACE) {
      if (part >= 0) {
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = atomicAdd(p.done + ctr, 1) == nparts - 1;
        __syncthreads();
        if (s_last) {
          __threadfence();
          const int64_t base = slot - (int64_t)part * ni;  // the group's first slot
          for (int i = tid; i < ni; i += NT) {
            double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
            for (int k = 0; k < nparts; k++) {
              const double *w = p.partial + 4 * (base + (int64_t)k * ni + i);
              m0 += __ldcg(w);
              m1 += __ldcg(w + 1);
              m2 += __ldcg(w + 2);
              m3 += __ldcg(w + 3);
            }
            const int64_t o = s0 + i;
            st_result(p.a + 3 * o, m0);
            st_result(p.a + 3 * o + 1, m1);
            st_result(p.a + 3 * o + 2, m2);
            st_result(p.phi + o, -m3);
          }
        }
      }
    }
  }
}

}  // namespace qg
