// qg_api.cu -- the qg_* C-ABI (include/qgrav.h): context, input upload and
// packing, argument validation, the device work queue and the CUDA graph
// that one qg_run replays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qg_attach.h"
#include "qg_devbuf.h"
#include "qg_internal.h"
#include "qg_queue.cuh"
#include "qgrav.h"

namespace {

using qg::kBuckets;
using qg::queue_hist_items_kernel;
using qg::queue_hist_kernel;
using qg::queue_scatter_kernel;

// ------------------------------------------------------------------ kernels

// |v| <= kMaxInput and finite (false for NaN)
__device__ __forceinline__ bool in_range(double v) { return fabs(v) <= qg::kMaxInput; }

// sources: [ns][3] + [ns] -> PosMass (x, y, z, float m); the FP64 masses
// stay in their own array (m is that array).  A position or mass that is not
// finite or exceeds kMaxInput in magnitude sets *bad.
__global__ void pack_src_kernel(int64_t ns, const double *__restrict__ x, const double *__restrict__ m,
                                qg::PosMass *__restrict__ out, qg::PosMassF *__restrict__ outf, int *bad) {
  bool ok = true;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
    qg::PosMass v;
    v.x = x[3 * i];
    v.y = x[3 * i + 1];
    v.z = x[3 * i + 2];
    v.m = (float)m[i];
    v.pad = 0.f;
    out[i] = v;
    outf[i] = qg::make_posmassf(v.x, v.y, v.z, v.m);
    ok = ok && in_range(v.x) && in_range(v.y) && in_range(v.z) && in_range(m[i]);
  }
  if (!ok) atomicOr(bad, 1);
}

// cells: com [nc][3], m [nc], q [nc][6] -> PosMass, float4 x 2 (Q), and a
// dense FP64 copy of Q for the all-FP64 kernel (skipped when q already is it).
// A value that is not finite or exceeds kMaxInput in magnitude sets *bad.
__global__ void pack_cells_kernel(int64_t nc, const double *__restrict__ com, const double *__restrict__ m,
                                  const double *q, qg::PosMass *__restrict__ pm, qg::PosMassF *__restrict__ pmf,
                                  float4 *__restrict__ qf, double *q64, int *bad) {
  bool ok = true;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
    qg::PosMass v;
    v.x = com[3 * i];
    v.y = com[3 * i + 1];
    v.z = com[3 * i + 2];
    v.m = (float)m[i];
    v.pad = 0.f;
    pm[i] = v;
    pmf[i] = qg::make_posmassf(v.x, v.y, v.z, v.m);
    const double *qi = q + 6 * i;
    qf[2 * i] = make_float4((float)qi[0], (float)qi[1], (float)qi[2], (float)qi[3]);
    qf[2 * i + 1] = make_float4((float)qi[4], (float)qi[5], 0.f, 0.f);
    if (q64 != q)
      for (int c = 0; c < 6; c++) q64[6 * i + c] = qi[c];
    ok = ok && in_range(v.x) && in_range(v.y) && in_range(v.z) && in_range(m[i]);
    for (int c = 0; c < 6; c++) ok = ok && in_range(qi[c]);
  }
  if (!ok) atomicOr(bad, 1);
}

// Sink checks of group_centre_kernel (bits of *flags).
constexpr int kBadPosition = 1;  // a position not finite or beyond kMaxInput
constexpr int kBadEps2 = 2;      // a per-sink eps^2 negative, not finite or beyond kMaxInput
constexpr int kZeroEps2 = 4;     // a per-sink eps^2 below the smallest normal float (0 to the FP32 kernels)

// c_g for every group: the centre of the bounding box of its sinks, one warp
// per group.  Offsets from the group's first sink are rounded to float, their
// extremes found (exact, so in any order), and the centre formed in FP64:
// c = x_first + (lo + hi) / 2.  The force kernels centre sinks and list
// entries on it.  Every sink's position (and per-sink eps^2, when given) is
// checked on the way (the kBad* / kZeroEps2 bits of *flags).
__global__ void group_centre_kernel(int64_t G, const int64_t *__restrict__ goff, const double *__restrict__ x,
                                    const float *__restrict__ eps2, double *__restrict__ centre,
                                    qg::PosMassF *__restrict__ centre_f, qg::PosMassF *__restrict__ sink_f,
                                    int *flags) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (gridDim.x * (int64_t)blockDim.x) >> 5;
  int f = 0;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
    const int64_t s0 = goff[g], ni = goff[g + 1] - s0;
    double c = 0.0;
    if (ni > 0) {
      const double b0 = x[3 * s0], b1 = x[3 * s0 + 1], b2 = x[3 * s0 + 2];
      float mn0 = 0.f, mn1 = 0.f, mn2 = 0.f, mx0 = 0.f, mx1 = 0.f, mx2 = 0.f;
      for (int64_t i = lane; i < ni; i += 32) {
        const double *xi = x + 3 * (s0 + i);
        sink_f[s0 + i] = qg::make_posmassf(xi[0], xi[1], xi[2], 0.f);
        if (!(in_range(xi[0]) && in_range(xi[1]) && in_range(xi[2]))) f |= kBadPosition;
        if (eps2) {
          const float e = eps2[s0 + i];
          if (!(e >= 0.f && (double)e <= qg::kMaxInput)) f |= kBadEps2;
          else if (e < 0x1p-126f) f |= kZeroEps2;
        }
        const float o0 = qg::f64_to_f32_rn(xi[0] - b0);
        const float o1 = qg::f64_to_f32_rn(xi[1] - b1);
        const float o2 = qg::f64_to_f32_rn(xi[2] - b2);
        mn0 = fminf(mn0, o0); mn1 = fminf(mn1, o1); mn2 = fminf(mn2, o2);
        mx0 = fmaxf(mx0, o0); mx1 = fmaxf(mx1, o1); mx2 = fmaxf(mx2, o2);
      }
      for (int o = 16; o > 0; o >>= 1) {
        mn0 = fminf(mn0, __shfl_xor_sync(0xffffffffu, mn0, o));
        mn1 = fminf(mn1, __shfl_xor_sync(0xffffffffu, mn1, o));
        mn2 = fminf(mn2, __shfl_xor_sync(0xffffffffu, mn2, o));
        mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
        mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
        mx2 = fmaxf(mx2, __shfl_xor_sync(0xffffffffu, mx2, o));
      }
      const float lo = lane == 0 ? mn0 : lane == 1 ? mn1 : mn2, hi = lane == 0 ? mx0 : lane == 1 ? mx1 : mx2;
      const double base = lane == 0 ? b0 : lane == 1 ? b1 : b2;
      c = base + 0.5 * ((double)lo + (double)hi);
    }
    if (lane < 3) centre[3 * g + lane] = c;
    // the centre as float pairs, for the centred FP32 kernels
    const double c0 = __shfl_sync(0xffffffffu, c, 0), c1 = __shfl_sync(0xffffffffu, c, 1),
                 c2 = __shfl_sync(0xffffffffu, c, 2);
    if (lane == 0) centre_f[g] = qg::make_posmassf(c0, c1, c2, 0.f);
  }
  if (f) atomicOr(flags, f);
}

// Index check that also makes the list safe to read: an entry outside
// [0, n) is counted in *bad and replaced by 0 (a kernel already queued behind
// this one then reads a valid record, and its caller fails with QG_ERR_ARG).
__global__ void sanitize_index_kernel(int64_t cnt, int32_t *__restrict__ idx, int64_t n, int *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = idx[i];
    if (v < 0 || (int64_t)v >= n) {
      atomicOr(bad, 1);
      idx[i] = 0;
    }
  }
}

// Index check of a device list: sets *bad when an entry is outside [0, n).
__global__ void check_index_kernel(int64_t cnt, const int32_t *__restrict__ idx, int64_t n, int *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = idx[i];
    if (v < 0 || (int64_t)v >= n) atomicOr(bad, 1);
  }
}

// ------------------------------------------------------------------ buffers

using qg::DevBuf;

// Context scratch (int): queue histogram [kBuckets], cursors [kBuckets], the
// queue head, the list-index check flag and the input-value check flags of
// the qg_set_* calls.
constexpr int kScratchInts = 2 * kBuckets + 3;
constexpr int kValueFlagSlot = 2 * kBuckets + 2;

}  // namespace

struct qg_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t last_stream = nullptr;
  qg_options opt{};
  std::string err;

  // sinks
  int64_t n = 0, G = -1;
  bool sinks_ok = false;
  bool eps_positive = true;  // every sink's eps^2 > 0
  bool has_eps2 = false;
  double eps2_all = 0.0;
  DevBuf<double> sink_x;
  DevBuf<float> sink_eps2;
  DevBuf<int64_t> goff;
  DevBuf<double> gcentre;  // [G][3] bounding-box centre of each group
  DevBuf<qg::PosMassF> gcentre_f, sink_f;  // the centres and sinks as float pairs
  std::vector<int64_t> h_goff;
  // sources
  int64_t ns = 0, G_src = -1, np_list = 0;
  bool src_ok = false;
  DevBuf<qg::PosMass> src;
  DevBuf<qg::PosMassF> src_f;
  DevBuf<double> src_m64;
  DevBuf<double> stage_x;  // device staging of host positions
  // group g's list: pidx[poff[g] .. poff[g + 1]) (CSR, the qg_set_* layout)
  // or, when p_ranges, pidx[poff[g] .. pend[g]) (a GPU tree's lists in the
  // order its walk produced them, qg_gtree_attach_move)
  DevBuf<int64_t> poff, pend;
  DevBuf<int32_t> pidx;
  std::vector<int64_t> h_poff, h_pend;
  bool p_ranges = false;
  // cells
  int64_t nc = 0, G_cell = -1, nc_list = 0;
  bool cells_ok = false;
  DevBuf<qg::PosMass> cell_pm;
  DevBuf<qg::PosMassF> cell_f;
  DevBuf<double> cell_m64;
  DevBuf<float4> cell_q;
  DevBuf<double> cell_q64;
  DevBuf<int64_t> coff, cend;  // as poff / pend
  DevBuf<int32_t> cidx;
  std::vector<int64_t> h_coff, h_cend;
  bool c_ranges = false;
  // outputs and queue
  DevBuf<double> a, phi;
  DevBuf<int> scratch;  // hist[kBuckets], cursor[kBuckets], head, bad
  DevBuf<unsigned char> bucket;
  DevBuf<int32_t> queue;
  // split lists (qg_options.split_j): the step's work items, the FP64
  // partial sums of the split groups' parts, their completion counts
  int64_t n_items = 0;  // 0: no split, one item per group
  int n_split = 0;
  int64_t n_slots = 0;
  DevBuf<qg::Item> items;
  DevBuf<double> partial;
  DevBuf<int> done;
  bool ran = false;  // outputs hold the result of a qg_run for the current sinks
  // graph, and events recorded inside it (step start, force start/end)
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool graph_valid = false;
  bool timed = false;  // ev[] hold the last run's step / force times
  // qg_evaluate_host: streams for the copies in and out, events per chunk
  cudaStream_t copy_in = nullptr, copy_out = nullptr, chunk_stream[4] = {};
  cudaEvent_t chunk_in[8] = {}, chunk_done[8] = {}, inputs_ready = nullptr, packed = nullptr;
  cudaEvent_t offsets_ready = nullptr, sinks_ready = nullptr;  // the first two groups of input copies
  DevBuf<double> stage_src;  // source positions when they are not the sinks' array
  int coherent_host = -1;    // device reads host memory through the host's page tables (-1: not asked yet)
  int *hbad = nullptr;       // page-locked [4]: bad-entry flags read back per chunk
  qg_stats stats{};
  // chosen launch (kernel_inplace: the same variant reading its lists from
  // host memory, or null where none is built)
  const void *kernel = nullptr, *kernel_inplace = nullptr;
  int grid_inplace = 0;
  int R = 4, nthreads = 128, tile = 256, flush = 128, grid = 0;
  size_t smem = 0;
};

namespace {

qg_status fail(qg_ctx *c, qg_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define QG_CUDA(ctx, call)                                                                       \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? QG_ERR_NOMEM : QG_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

cudaStream_t pick_stream(qg_ctx *c, void *s) { return s ? (cudaStream_t)s : c->stream; }

void invalidate(qg_ctx *c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  c->exec = nullptr;
  c->graph_valid = false;
  c->timed = false;
}

bool valid_options(const qg_options &o, std::string &why) {
  if (o.precision < QG_FP32_CENTRED || o.precision > QG_FP64) { why = "precision"; return false; }
  if (o.expansion != QG_QUAD && o.expansion != QG_MONO) { why = "expansion"; return false; }
  if (o.tile_j && (o.tile_j < 32 || o.tile_j > 1024 || o.tile_j % 32)) { why = "tile_j"; return false; }
  if (o.warps_per_group && o.warps_per_group != 1 && o.warps_per_group != 2 && o.warps_per_group != 4 &&
      o.warps_per_group != 8) {
    why = "warps_per_group";
    return false;
  }
  if (o.sinks_per_thread && o.sinks_per_thread != 2 && o.sinks_per_thread != 4 && o.sinks_per_thread != 8) {
    why = "sinks_per_thread";
    return false;
  }
  if (o.flush_j < 0) { why = "flush_j"; return false; }
  if (o.arith < QG_ARITH_DEFAULT || o.arith > QG_ARITH_ENTRY_PAIRED) { why = "arith"; return false; }
  if (o.split_j < -1) { why = "split_j"; return false; }
  if (o.sinks_adaptive != 0 && o.sinks_adaptive != 1) { why = "sinks_adaptive"; return false; }
  if (o.sinks_adaptive &&
      (o.precision != QG_FP32_CENTRED || o.arith == QG_ARITH_PAIRED || (o.sinks_per_thread && o.sinks_per_thread != 4))) {
    why = "sinks_adaptive (FP32 centred, scalar or entry-paired, up to 4 sinks per thread)";
    return false;
  }
  return true;
}

// Offsets of length G+1: off[0] = 0, non-decreasing, off[G] = total.
bool valid_offsets(const int64_t *off, int64_t G, int64_t total) {
  if (off[0] != 0 || off[G] != total) return false;
  for (int64_t g = 0; g < G; g++)
    if (off[g + 1] < off[g]) return false;
  return true;
}

bool valid_offsets_any_total(const int64_t *off, int64_t G) {
  if (off[0] != 0) return false;
  for (int64_t g = 0; g < G; g++)
    if (off[g + 1] < off[g]) return false;
  return true;
}

int grid_for(int64_t n, int block) {
  int64_t b = (n + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4096));
}

// Host-side list lengths and device-side list ends of group g (CSR offsets
// or begin / end ranges).
int64_t plen(const qg_ctx *c, int64_t g) {
  return c->p_ranges ? c->h_pend[g] - c->h_poff[g] : c->h_poff[g + 1] - c->h_poff[g];
}
int64_t clen(const qg_ctx *c, int64_t g) {
  return c->c_ranges ? c->h_cend[g] - c->h_coff[g] : c->h_coff[g + 1] - c->h_coff[g];
}
const int64_t *pend_dev(const qg_ctx *c) { return c->p_ranges ? c->pend.p : c->poff.p + 1; }
const int64_t *cend_dev(const qg_ctx *c) { return c->c_ranges ? c->cend.p : c->coff.p + 1; }

// Stats that depend on every input.
void update_counts(qg_ctx *c) {
  c->stats.n_sinks = c->n;
  c->stats.n_groups = c->G < 0 ? 0 : c->G;
  c->stats.n_sources = c->ns;
  c->stats.n_cells = c->nc;
  c->stats.n_plist = c->np_list;
  c->stats.n_clist = c->nc_list;
  int64_t ipp = 0, ipc = 0;
  if (c->sinks_ok && (int64_t)c->h_goff.size() == c->G + 1) {
    for (int64_t g = 0; g < c->G; g++) {
      const int64_t ni = c->h_goff[g + 1] - c->h_goff[g];
      if (c->src_ok && c->G_src == c->G) ipp += ni * plen(c, g);
      if (c->cells_ok && c->G_cell == c->G) ipc += ni * clen(c, g);
    }
  }
  c->stats.i_pp = ipp;
  c->stats.i_pc = ipc;
}

qg_status choose_kernel(qg_ctx *c) {
  const qg_options &o = c->opt;
  const bool fp64 = o.precision == QG_FP64;
  const bool quad = o.expansion == QG_QUAD;
  const bool guard = !c->eps_positive;
  int R = o.sinks_per_thread ? o.sinks_per_thread : 4;
  if (fp64) R = 2;
  const bool paired = o.precision == QG_FP32_CENTRED && o.arith == QG_ARITH_PAIRED;
  // the entry-paired form is the default of the centred FP32 precision (up to
  // 4 sinks per thread), the scalar form otherwise
  const bool epaired = o.precision == QG_FP32_CENTRED &&
                       (o.arith == QG_ARITH_ENTRY_PAIRED || (o.arith == QG_ARITH_DEFAULT && R <= 4));
  int warps = o.warps_per_group ? o.warps_per_group : (epaired ? 2 : 4);
  if (R >= 8 && warps > 4) warps = 4;
  const int nt = 32 * warps;
  const bool adapt = o.sinks_adaptive != 0;
  const void *k = fp64 ? qg::force_kernel_f64(R, quad, guard)
                  : adapt ? qg::force_kernel_adapt(epaired, quad, guard)
                  : paired ? qg::force_kernel_f32x2(R, quad, guard)
                  : epaired ? qg::force_kernel_f32ep(R, quad, guard)
                            : qg::force_kernel_f32(R, quad, guard, o.precision == QG_FP32_CENTRED);
  if (!k) return fail(c, QG_ERR_ARG, "no kernel for precision %d, R %d", o.precision, R);
  const int tile = o.tile_j ? o.tile_j : 256;
  const size_t smem = qg::force_smem_bytes(fp64, paired, R, nt, tile);
  QG_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  QG_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, smem));
  if (per_sm < 1) return fail(c, QG_ERR_ARG, "force kernel does not fit on an SM (smem %zu)", smem);
  c->kernel = k;
  c->kernel_inplace = nullptr;
  if (o.precision == QG_FP32_CENTRED && !paired) {
    const void *ki = adapt ? qg::force_kernel_inplace_adapt(epaired, quad, guard)
                           : qg::force_kernel_inplace(R, quad, guard, epaired);
    int per_sm_i = 0;
    if (ki) {
      QG_CUDA(c, cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      QG_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_i, ki, nt, smem));
    }
    if (per_sm_i >= 1) {
      c->kernel_inplace = ki;
      c->grid_inplace = per_sm_i * c->num_sms;
    }
  }
  c->R = R;
  c->nthreads = nt;
  c->tile = tile;
  c->flush = o.flush_j ? o.flush_j : 256;
  c->smem = smem;
  c->grid = per_sm * c->num_sms;
  c->stats.block = nt;
  c->stats.sinks_per_thread = R;
  c->stats.tile_j = tile;
  c->stats.warps_per_group = warps;
  c->stats.flush_j = c->flush;
  c->stats.paired = paired ? 1 : epaired ? 2 : 0;
  c->stats.sinks_adaptive = adapt ? 1 : 0;
  return QG_OK;
}

// Kernel parameters for groups [g0, g0 + G): the offset arrays and the queue
// are passed from g0 on, so the queue's (relative) group numbers index them
// directly; sink, list and output positions stay absolute.
qg::ForceParams force_params(qg_ctx *c, int64_t g0, int64_t G, int *head) {
  qg::ForceParams p{};
  p.sink_x = c->sink_x.p;
  p.sink_eps2 = c->has_eps2 ? c->sink_eps2.p : nullptr;
  p.eps2_all = c->eps2_all;
  p.eps2_all_f = (float)c->eps2_all;
  p.group_off = c->goff.p + g0;
  p.gcentre = c->gcentre.p + 3 * g0;
  p.gcentre_f = c->gcentre_f.p + g0;
  p.sink_f = c->sink_f.p;
  p.src_f = c->src_f.p;
  p.cell_f = c->cell_f.p;
  p.src = c->src.p;
  p.src_m64 = c->src_m64.p;
  p.plist_off = c->poff.p + g0;
  p.plist_end = pend_dev(c) + g0;
  p.plist_idx = c->pidx.p;
  p.cell_pm = c->cell_pm.p;
  p.cell_m64 = c->cell_m64.p;
  p.cell_q = c->cell_q.p;
  p.cell_q64 = c->cell_q64.p;
  p.clist_off = c->coff.p + g0;
  p.clist_end = cend_dev(c) + g0;
  p.clist_idx = c->cidx.p;
  p.queue = c->queue.p + g0;
  p.nitems = (int32_t)G;
  p.head = head;
  p.a = c->a.p;
  p.phi = c->phi.p;
  p.tile = c->tile;
  p.flush_j = c->flush;
  p.zero = 0.0f;
  p.one = 1.0f;
  return p;
}

// Work items of a step with split lists (qg_options.split_j != 0): every
// group whose list is long (split_j > 0: more than split_j entries) or
// expensive (split_j = -1: more than a quarter of one CTA's average share of
// the step) is cut into parts of about equal FP32 work (particle entries
// weigh 13, cells 33 or 13), at most 64; the other groups stay one item.
// Host work O(groups), done when the step's graph is (re)built.
qg_status build_items(qg_ctx *c) {
  c->n_items = 0;
  c->n_split = 0;
  c->n_slots = 0;
  const int split = c->opt.split_j;
  const int64_t G = c->G;
  if (split == 0 || G <= 0) return QG_OK;
  const double cell_ops = c->opt.expansion == QG_QUAD ? 33.0 : 13.0;
  const std::vector<int64_t> &go = c->h_goff;
  double share = 0.0;
  if (split < 0) {
    for (int64_t g = 0; g < G; g++) {
      const double ni = (double)(go[g + 1] - go[g]), np = (double)plen(c, g), nc = (double)clen(c, g);
      share += ni * (13.0 * np + cell_ops * nc) + 64.0 * (np + nc) + 256.0;
    }
    share /= std::max(c->grid, 1);
  }
  std::vector<qg::Item> it;
  it.reserve((size_t)G);
  int64_t slot = 0;
  int ctr = 0;
  for (int64_t g = 0; g < G; g++) {
    const int64_t ni = go[g + 1] - go[g], np = plen(c, g), nc = clen(c, g), ne = np + nc;
    int64_t P = 1;
    if (ni > 0 && ne > 1) {
      if (split > 0) {
        P = (ne + split - 1) / split;
      } else {
        const double cost = (double)ni * (13.0 * np + cell_ops * nc) + 64.0 * ne + 256.0;
        if (cost > 0.25 * share) P = (int64_t)std::ceil(cost / (0.125 * share));
      }
      P = std::min<int64_t>(std::min<int64_t>(P, 64), ne);
    }
    if (P <= 1) {
      it.push_back(qg::Item{(int32_t)g, -1, 1, 0, 0, ne, 0});
      continue;
    }
    // cut points at equal FP32 work
    const double W = 13.0 * np + cell_ops * nc;
    int64_t prev = 0;
    for (int64_t k = 0; k < P; k++) {
      int64_t e = ne;
      if (k < P - 1) {
        const double target = W * (double)(k + 1) / (double)P;
        e = target <= 13.0 * np ? (int64_t)std::ceil(target / 13.0)
                                : np + (int64_t)std::ceil((target - 13.0 * np) / cell_ops);
        e = std::max(e, prev + 1);
        e = std::min(e, ne - (P - 1 - k));
      }
      it.push_back(qg::Item{(int32_t)g, (int32_t)k, (int32_t)P, ctr, prev, e, slot + k * ni});
      prev = e;
    }
    slot += P * ni;
    ctr++;
  }
  if (ctr == 0) return QG_OK;  // nothing long enough to split: one item per group
  if (it.size() >= (size_t)INT32_MAX) return fail(c, QG_ERR_SIZE, "too many work items (%zu)", it.size());
  cudaError_t e;
  if ((e = c->items.reserve(it.size())) != cudaSuccess || (e = c->partial.reserve(4 * slot)) != cudaSuccess ||
      (e = c->done.reserve(ctr)) != cudaSuccess)
    return fail(c, QG_ERR_NOMEM, "work item allocation: %s", cudaGetErrorString(e));
  QG_CUDA(c, cudaMemcpy(c->items.p, it.data(), it.size() * sizeof(qg::Item), cudaMemcpyHostToDevice));
  c->n_items = (int64_t)it.size();
  c->n_split = ctr;
  c->n_slots = slot;
  return QG_OK;
}

// Record the queue build and the persistent force launch on stream s.
qg_status record_step(qg_ctx *c, cudaStream_t s) {
  const int64_t G = c->G;
  int *hist = c->scratch.p, *cursor = hist + kBuckets, *head = cursor + kBuckets;
  QG_CUDA(c, cudaEventRecordWithFlags(c->ev[0], s, cudaEventRecordExternal));
  QG_CUDA(c, cudaMemsetAsync(hist, 0, (2 * kBuckets + 2) * sizeof(int), s));
  const double cell_ops = c->opt.expansion == QG_QUAD ? 33.0 : 13.0;
  const int64_t NI = c->n_items ? c->n_items : G;  // work items: groups, or groups and parts of split lists
  if (c->n_items) {
    QG_CUDA(c, cudaMemsetAsync(c->done.p, 0, std::max(c->n_split, 1) * sizeof(int), s));
    queue_hist_items_kernel<<<grid_for(NI, 256), 256, 0, s>>>(NI, c->items.p, c->goff.p, c->poff.p, pend_dev(c),
                                                               cell_ops, c->bucket.p, hist);
  } else {
    queue_hist_kernel<<<grid_for(G, 256), 256, 0, s>>>(G, c->goff.p, c->poff.p, pend_dev(c), c->coff.p,
                                                        cend_dev(c), cell_ops, c->bucket.p, hist);
  }
  QG_CUDA(c, cudaGetLastError());
  queue_scatter_kernel<<<grid_for(NI, 256), 256, 0, s>>>(NI, c->bucket.p, hist, cursor, c->queue.p);
  QG_CUDA(c, cudaGetLastError());
  qg::ForceParams p = force_params(c, 0, G, head);
  if (c->n_items) {
    p.items = c->items.p;
    p.partial = c->partial.p;
    p.done = c->done.p;
    p.nitems = (int32_t)NI;
  }
  const int grid = (int)std::min<int64_t>(c->grid, std::max<int64_t>(NI, 1));
  c->stats.n_items = NI;
  c->stats.n_split = c->n_split;
  c->stats.grid = grid;
  void *args[] = {&p};
  QG_CUDA(c, cudaEventRecordWithFlags(c->ev[1], s, cudaEventRecordExternal));
  QG_CUDA(c, cudaLaunchKernel(c->kernel, dim3(grid), dim3(c->nthreads), args, c->smem, s));
  QG_CUDA(c, cudaEventRecordWithFlags(c->ev[2], s, cudaEventRecordExternal));
  return QG_OK;
}

qg_status ensure_graph(qg_ctx *c) {
  if (c->graph_valid) return QG_OK;
  invalidate(c);
  qg_status st = choose_kernel(c);
  if (st != QG_OK) return st;
  if ((st = build_items(c)) != QG_OK) return st;
  const int64_t G = c->G;
  const int64_t NI = std::max(G, c->n_items);
  {
    cudaError_t e;
    if ((e = c->scratch.reserve(kScratchInts)) != cudaSuccess ||
        (e = c->bucket.reserve(NI)) != cudaSuccess || (e = c->queue.reserve(NI)) != cudaSuccess ||
        (e = c->a.reserve(3 * std::max<int64_t>(c->n, 1))) != cudaSuccess ||
        (e = c->phi.reserve(std::max<int64_t>(c->n, 1))) != cudaSuccess)
      return fail(c, QG_ERR_NOMEM, "device allocation: %s", cudaGetErrorString(e));
  }
  cudaStream_t cap;
  QG_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cap);
    return fail(c, QG_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
  }
  st = record_step(c, cap);
  e = cudaStreamEndCapture(cap, &graph);
  cudaStreamDestroy(cap);
  if (st != QG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(c, QG_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->exec = nullptr;
    return fail(c, QG_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  c->graph_valid = true;
  return QG_OK;
}

template <typename T>
qg_status upload(qg_ctx *c, DevBuf<T> &buf, const T *h, size_t count, cudaStream_t s) {
  cudaError_t e = buf.reserve(count);
  if (e != cudaSuccess) return fail(c, QG_ERR_NOMEM, "device allocation of %zu bytes", count * sizeof(T));
  if (count) QG_CUDA(c, cudaMemcpyAsync(buf.p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
  return QG_OK;
}

template <typename T>
qg_status copy_d2d(qg_ctx *c, DevBuf<T> &buf, const T *d, size_t count, cudaStream_t s) {
  cudaError_t e = buf.reserve(count);
  if (e != cudaSuccess) return fail(c, QG_ERR_NOMEM, "device allocation of %zu bytes", count * sizeof(T));
  if (count) QG_CUDA(c, cudaMemcpyAsync(buf.p, d, count * sizeof(T), cudaMemcpyDeviceToDevice, s));
  return QG_OK;
}

qg_status check_indices_dev(qg_ctx *c, const int32_t *idx, int64_t cnt, int64_t n, cudaStream_t s,
                            const char *what) {
  if (cnt == 0) return QG_OK;
  cudaError_t e = c->scratch.reserve(kScratchInts);
  if (e != cudaSuccess) return fail(c, QG_ERR_NOMEM, "scratch allocation");
  int *bad = c->scratch.p + 2 * kBuckets + 1;
  QG_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), s));
  check_index_kernel<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, idx, n, bad);
  QG_CUDA(c, cudaGetLastError());
  int h = 0;
  QG_CUDA(c, cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  QG_CUDA(c, cudaStreamSynchronize(s));
  if (h) return fail(c, QG_ERR_ARG, "%s: list entry outside [0, %lld)", what, (long long)n);
  return QG_OK;
}

// The input-value check flags of a qg_set_* call: zeroed on s before the
// kernels that check (and pack) the inputs ...
qg_status value_flags_begin(qg_ctx *c, cudaStream_t s, int **flags) {
  if (c->scratch.reserve(kScratchInts) != cudaSuccess) return fail(c, QG_ERR_NOMEM, "scratch allocation");
  *flags = c->scratch.p + kValueFlagSlot;
  QG_CUDA(c, cudaMemsetAsync(*flags, 0, sizeof(int), s));
  return QG_OK;
}

// ... and read back after them (synchronises s).
qg_status value_flags_end(qg_ctx *c, cudaStream_t s, const int *flags, int *value) {
  QG_CUDA(c, cudaGetLastError());
  QG_CUDA(c, cudaMemcpyAsync(value, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  QG_CUDA(c, cudaStreamSynchronize(s));
  return QG_OK;
}

}  // namespace

// ======================================================================= ABI

extern "C" {

qg_status qg_create(qg_ctx **out, int device, const qg_options *opt) {
  if (!out) return QG_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return QG_ERR_ARG;
  qg_ctx *c = new (std::nothrow) qg_ctx;
  if (!c) return QG_ERR_NOMEM;
  c->device = device;
  if (opt) {
    std::string why;
    if (!valid_options(*opt, why)) {
      delete c;
      return QG_ERR_ARG;
    }
    c->opt = *opt;
  }
  DeviceGuard dg(device);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return QG_ERR_CUDA;
  }
  c->last_stream = c->stream;
  for (auto &e : c->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      qg_destroy(c);
      return QG_ERR_CUDA;
    }
  }
  *out = c;
  return QG_OK;
}

void qg_destroy(qg_ctx *c) {
  if (!c) return;
  DeviceGuard dg(c->device);
  if (c->last_stream) cudaStreamSynchronize(c->last_stream);
  if (c->stream) cudaStreamSynchronize(c->stream);
  invalidate(c);
  c->sink_x.release(); c->sink_eps2.release(); c->goff.release();
  c->gcentre.release(); c->gcentre_f.release(); c->sink_f.release();
  c->items.release(); c->partial.release(); c->done.release();
  c->src.release(); c->src_f.release(); c->src_m64.release(); c->stage_x.release();
  c->poff.release(); c->pend.release(); c->pidx.release(); c->cend.release();
  c->cell_pm.release(); c->cell_f.release(); c->cell_m64.release(); c->cell_q.release(); c->cell_q64.release(); c->coff.release(); c->cidx.release();
  c->a.release(); c->phi.release(); c->scratch.release(); c->bucket.release(); c->queue.release();
  for (auto &e : c->ev)
    if (e) cudaEventDestroy(e);
  for (int k = 0; k < 8; k++) {
    if (c->chunk_in[k]) cudaEventDestroy(c->chunk_in[k]);
    if (c->chunk_done[k]) cudaEventDestroy(c->chunk_done[k]);
  }
  if (c->inputs_ready) cudaEventDestroy(c->inputs_ready);
  if (c->offsets_ready) cudaEventDestroy(c->offsets_ready);
  if (c->sinks_ready) cudaEventDestroy(c->sinks_ready);
  if (c->packed) cudaEventDestroy(c->packed);
  c->stage_src.release();
  for (cudaStream_t t : {c->copy_in, c->copy_out, c->chunk_stream[0], c->chunk_stream[1], c->chunk_stream[2],
                         c->chunk_stream[3]})
    if (t) {
      cudaStreamSynchronize(t);
      cudaStreamDestroy(t);
    }
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->hbad) cudaFreeHost(c->hbad);
  delete c;
}

qg_status qg_set_options(qg_ctx *c, const qg_options *opt) {
  if (!c || !opt) return QG_ERR_ARG;
  std::string why;
  if (!valid_options(*opt, why)) return fail(c, QG_ERR_ARG, "bad option: %s", why.c_str());
  c->opt = *opt;
  invalidate(c);
  return QG_OK;
}

// Group centres of the sinks now on the device (sink_x, goff), on stream s;
// the sinks' positions (and eps2, a device array or null) are checked into
// *flags on the way.
static qg_status group_centres(qg_ctx *c, int64_t n, int64_t G, const float *eps2, int *flags, cudaStream_t s) {
  cudaError_t e = c->gcentre.reserve(3 * std::max<int64_t>(G, 1));
  if (e == cudaSuccess) e = c->gcentre_f.reserve(std::max<int64_t>(G, 1));
  if (e == cudaSuccess) e = c->sink_f.reserve(std::max<int64_t>(n, 1));
  if (e != cudaSuccess) return fail(c, QG_ERR_NOMEM, "group centre allocation");
  if (G > 0) {
    group_centre_kernel<<<grid_for(32 * G, 256), 256, 0, s>>>(G, c->goff.p, c->sink_x.p, eps2, c->gcentre.p,
                                                               c->gcentre_f.p, c->sink_f.p, flags);
    QG_CUDA(c, cudaGetLastError());
  }
  return QG_OK;
}

static qg_status set_sinks_common(qg_ctx *c, int64_t n, const double *x, const float *eps2, double eps2_all,
                                  int64_t ngroups, const int64_t *group_off, bool dev, cudaStream_t s) {
  // inputs must not change under a step that is still running
  if (c->last_stream) cudaStreamSynchronize(c->last_stream);
  c->sinks_ok = false;
  invalidate(c);
  if (n < 0 || ngroups < 0 || ngroups >= INT32_MAX || !group_off || (n > 0 && !x))
    return fail(c, QG_ERR_ARG, "qg_set_sinks: bad sizes or NULL pointer");
  if (!(eps2_all >= 0 && eps2_all <= qg::kMaxInput))
    return fail(c, QG_ERR_ARG, "qg_set_sinks: eps2_all must be finite, >= 0 and at most 2^100");
  DeviceGuard dg(c->device);
  std::vector<int64_t> h(ngroups + 1);
  if (dev) {
    QG_CUDA(c, cudaMemcpyAsync(h.data(), group_off, (ngroups + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QG_CUDA(c, cudaStreamSynchronize(s));
  } else {
    std::memcpy(h.data(), group_off, (ngroups + 1) * sizeof(int64_t));
  }
  if (!valid_offsets(h.data(), ngroups, n)) return fail(c, QG_ERR_ARG, "qg_set_sinks: bad group offsets");
  // the unguarded kernels need every eps^2 to be a normal float (the FP32
  // kernels flush smaller values to zero); a device eps^2 array is checked
  // by group_centre_kernel below
  bool pos = eps2_all >= 0x1p-126;
  if (eps2) {
    pos = true;
    if (!dev) {
      for (int64_t i = 0; i < n; i++) {
        if (!(eps2[i] >= 0.f && (double)eps2[i] <= qg::kMaxInput))
          return fail(c, QG_ERR_ARG, "qg_set_sinks: eps2[%lld] invalid", (long long)i);
        if (!(eps2[i] >= 0x1p-126f)) pos = false;
      }
    }
  }
  qg_status st;
  if (dev) {
    if ((st = copy_d2d(c, c->sink_x, x, 3 * n, s)) != QG_OK) return st;
    if (eps2 && (st = copy_d2d(c, c->sink_eps2, eps2, n, s)) != QG_OK) return st;
    if ((st = copy_d2d(c, c->goff, group_off, ngroups + 1, s)) != QG_OK) return st;
  } else {
    if ((st = upload(c, c->sink_x, x, 3 * n, s)) != QG_OK) return st;
    if (eps2 && (st = upload(c, c->sink_eps2, eps2, n, s)) != QG_OK) return st;
    if ((st = upload(c, c->goff, group_off, ngroups + 1, s)) != QG_OK) return st;
  }
  int *flags = nullptr, fl = 0;
  if ((st = value_flags_begin(c, s, &flags)) != QG_OK) return st;
  if ((st = group_centres(c, n, ngroups, dev && eps2 ? c->sink_eps2.p : nullptr, flags, s)) != QG_OK) return st;
  if ((st = value_flags_end(c, s, flags, &fl)) != QG_OK) return st;
  if (fl & kBadPosition) return fail(c, QG_ERR_ARG, "qg_set_sinks: a position is not finite or exceeds 2^100");
  if (fl & kBadEps2) return fail(c, QG_ERR_ARG, "qg_set_sinks: an eps2 is negative, not finite or exceeds 2^100");
  if (fl & kZeroEps2) pos = false;
  c->n = n;
  c->G = ngroups;
  c->has_eps2 = eps2 != nullptr;
  c->eps2_all = eps2_all;
  c->eps_positive = pos;
  c->h_goff.swap(h);
  c->sinks_ok = true;
  c->ran = false;
  update_counts(c);
  return QG_OK;
}

qg_status qg_set_sinks(qg_ctx *c, int64_t n, const double *x, const float *eps2, double eps2_all,
                       int64_t ngroups, const int64_t *group_off) {
  if (!c) return QG_ERR_ARG;
  return set_sinks_common(c, n, x, eps2, eps2_all, ngroups, group_off, false, c->stream);
}

qg_status qg_set_sinks_dev(qg_ctx *c, int64_t n, const double *x, const float *eps2, double eps2_all,
                           int64_t ngroups, const int64_t *group_off, void *stream) {
  if (!c) return QG_ERR_ARG;
  return set_sinks_common(c, n, x, eps2, eps2_all, ngroups, group_off, true, pick_stream(c, stream));
}

static qg_status set_sources_common(qg_ctx *c, int64_t ns, const double *x, const double *m,
                                    const int64_t *list_off, const int32_t *list_idx, int64_t n_list_dev,
                                    bool dev, cudaStream_t s) {
  // inputs must not change under a step that is still running
  if (c->last_stream) cudaStreamSynchronize(c->last_stream);
  c->src_ok = false;
  invalidate(c);
  if (c->G < 0 || !c->sinks_ok) return fail(c, QG_ERR_STATE, "qg_set_sources: set the sinks first");
  if (ns < 0 || ns >= INT32_MAX || !list_off || (ns > 0 && (!x || !m)))
    return fail(c, QG_ERR_ARG, "qg_set_sources: bad sizes or NULL pointer");
  const int64_t G = c->G;
  DeviceGuard dg(c->device);
  std::vector<int64_t> h(G + 1);
  qg_status st;
  int *flags = nullptr;
  if (dev) {
    QG_CUDA(c, cudaMemcpyAsync(h.data(), list_off, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QG_CUDA(c, cudaStreamSynchronize(s));
    if (!valid_offsets(h.data(), G, n_list_dev)) return fail(c, QG_ERR_ARG, "qg_set_sources: bad list offsets");
    if (n_list_dev > 0 && !list_idx) return fail(c, QG_ERR_ARG, "qg_set_sources: list_idx is NULL");
    if ((st = check_indices_dev(c, list_idx, n_list_dev, ns, s, "qg_set_sources")) != QG_OK) return st;
  } else {
    std::memcpy(h.data(), list_off, (G + 1) * sizeof(int64_t));
    if (!valid_offsets_any_total(h.data(), G)) return fail(c, QG_ERR_ARG, "qg_set_sources: bad list offsets");
    if (h[G] > 0 && !list_idx) return fail(c, QG_ERR_ARG, "qg_set_sources: list_idx is NULL");
  }
  const int64_t cnt = h[G];
  if (dev) {
    if ((st = copy_d2d(c, c->poff, list_off, G + 1, s)) != QG_OK) return st;
    if ((st = copy_d2d(c, c->pidx, list_idx, cnt, s)) != QG_OK) return st;
    if ((st = copy_d2d(c, c->src_m64, m, ns, s)) != QG_OK) return st;
    cudaError_t e = c->src.reserve(ns);
    if (e == cudaSuccess) e = c->src_f.reserve(ns);
    if (e != cudaSuccess) return fail(c, QG_ERR_NOMEM, "source allocation");
    if ((st = value_flags_begin(c, s, &flags)) != QG_OK) return st;
    if (ns) pack_src_kernel<<<grid_for(ns, 256), 256, 0, s>>>(ns, x, c->src_m64.p, c->src.p, c->src_f.p, flags);
  } else {
    if ((st = upload(c, c->poff, list_off, G + 1, s)) != QG_OK) return st;
    if ((st = upload(c, c->pidx, list_idx, cnt, s)) != QG_OK) return st;
    // indices are checked on the device, after the copy, before any kernel uses them
    if ((st = check_indices_dev(c, c->pidx.p, cnt, ns, s, "qg_set_sources")) != QG_OK) return st;
    if ((st = upload(c, c->stage_x, x, 3 * ns, s)) != QG_OK) return st;
    if ((st = upload(c, c->src_m64, m, ns, s)) != QG_OK) return st;
    cudaError_t e = c->src.reserve(ns);
    if (e == cudaSuccess) e = c->src_f.reserve(ns);
    if (e != cudaSuccess) return fail(c, QG_ERR_NOMEM, "source allocation");
    if ((st = value_flags_begin(c, s, &flags)) != QG_OK) return st;
    if (ns)
      pack_src_kernel<<<grid_for(ns, 256), 256, 0, s>>>(ns, c->stage_x.p, c->src_m64.p, c->src.p, c->src_f.p, flags);
  }
  int fl = 0;
  if ((st = value_flags_end(c, s, flags, &fl)) != QG_OK) return st;
  if (fl) return fail(c, QG_ERR_ARG, "qg_set_sources: a position or mass is not finite or exceeds 2^100");
  c->ns = ns;
  c->G_src = G;
  c->np_list = cnt;
  c->h_poff.swap(h);
  c->p_ranges = false;
  c->src_ok = true;
  update_counts(c);
  return QG_OK;
}

qg_status qg_set_sources(qg_ctx *c, int64_t ns, const double *x, const double *m, const int64_t *list_off,
                         const int32_t *list_idx) {
  if (!c) return QG_ERR_ARG;
  return set_sources_common(c, ns, x, m, list_off, list_idx, 0, false, c->stream);
}

qg_status qg_set_sources_dev(qg_ctx *c, int64_t ns, const double *x, const double *m, const int64_t *list_off,
                             const int32_t *list_idx, int64_t n_list, void *stream) {
  if (!c) return QG_ERR_ARG;
  return set_sources_common(c, ns, x, m, list_off, list_idx, n_list, true, pick_stream(c, stream));
}

static qg_status set_cells_common(qg_ctx *c, int64_t nc, const double *com, const double *m, const double *q,
                                  const int64_t *list_off, const int32_t *list_idx, int64_t n_list_dev, bool dev,
                                  cudaStream_t s) {
  // inputs must not change under a step that is still running
  if (c->last_stream) cudaStreamSynchronize(c->last_stream);
  c->cells_ok = false;
  invalidate(c);
  if (c->G < 0 || !c->sinks_ok) return fail(c, QG_ERR_STATE, "qg_set_cells: set the sinks first");
  if (nc < 0 || nc >= INT32_MAX || !list_off || (nc > 0 && (!com || !m || !q)))
    return fail(c, QG_ERR_ARG, "qg_set_cells: bad sizes or NULL pointer");
  const int64_t G = c->G;
  DeviceGuard dg(c->device);
  std::vector<int64_t> h(G + 1);
  qg_status st;
  int *flags = nullptr;
  if (dev) {
    QG_CUDA(c, cudaMemcpyAsync(h.data(), list_off, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QG_CUDA(c, cudaStreamSynchronize(s));
    if (!valid_offsets(h.data(), G, n_list_dev)) return fail(c, QG_ERR_ARG, "qg_set_cells: bad list offsets");
    if (n_list_dev > 0 && !list_idx) return fail(c, QG_ERR_ARG, "qg_set_cells: list_idx is NULL");
    if ((st = check_indices_dev(c, list_idx, n_list_dev, nc, s, "qg_set_cells")) != QG_OK) return st;
  } else {
    std::memcpy(h.data(), list_off, (G + 1) * sizeof(int64_t));
    if (!valid_offsets_any_total(h.data(), G)) return fail(c, QG_ERR_ARG, "qg_set_cells: bad list offsets");
    if (h[G] > 0 && !list_idx) return fail(c, QG_ERR_ARG, "qg_set_cells: list_idx is NULL");
  }
  const int64_t cnt = h[G];
  if (c->cell_pm.reserve(nc) != cudaSuccess || c->cell_f.reserve(nc) != cudaSuccess ||
      c->cell_q.reserve(2 * nc) != cudaSuccess || c->cell_q64.reserve(6 * nc) != cudaSuccess)
    return fail(c, QG_ERR_NOMEM, "cell allocation");
  if (dev) {
    if ((st = copy_d2d(c, c->coff, list_off, G + 1, s)) != QG_OK) return st;
    if ((st = copy_d2d(c, c->cidx, list_idx, cnt, s)) != QG_OK) return st;
    if ((st = copy_d2d(c, c->cell_m64, m, nc, s)) != QG_OK) return st;
    if ((st = value_flags_begin(c, s, &flags)) != QG_OK) return st;
    if (nc)
      pack_cells_kernel<<<grid_for(nc, 256), 256, 0, s>>>(nc, com, c->cell_m64.p, q, c->cell_pm.p, c->cell_f.p,
                                                           c->cell_q.p, c->cell_q64.p, flags);
  } else {
    if ((st = upload(c, c->coff, list_off, G + 1, s)) != QG_OK) return st;
    if ((st = upload(c, c->cidx, list_idx, cnt, s)) != QG_OK) return st;
    if ((st = check_indices_dev(c, c->cidx.p, cnt, nc, s, "qg_set_cells")) != QG_OK) return st;
    if ((st = upload(c, c->stage_x, com, 3 * nc, s)) != QG_OK) return st;
    if ((st = upload(c, c->cell_m64, m, nc, s)) != QG_OK) return st;
    // Q goes straight into the FP64 copy, which the packer then reads
    if ((st = upload(c, c->cell_q64, q, 6 * nc, s)) != QG_OK) return st;
    if ((st = value_flags_begin(c, s, &flags)) != QG_OK) return st;
    if (nc)
      pack_cells_kernel<<<grid_for(nc, 256), 256, 0, s>>>(nc, c->stage_x.p, c->cell_m64.p, c->cell_q64.p,
                                                           c->cell_pm.p, c->cell_f.p, c->cell_q.p, c->cell_q64.p,
                                                           flags);
  }
  int fl = 0;
  if ((st = value_flags_end(c, s, flags, &fl)) != QG_OK) return st;
  if (fl) return fail(c, QG_ERR_ARG, "qg_set_cells: a position, mass or quadrupole component is not finite or exceeds 2^100");
  c->nc = nc;
  c->G_cell = G;
  c->nc_list = cnt;
  c->h_coff.swap(h);
  c->c_ranges = false;
  c->cells_ok = true;
  update_counts(c);
  return QG_OK;
}

qg_status qg_set_cells(qg_ctx *c, int64_t nc, const double *com, const double *m, const double *q,
                       const int64_t *list_off, const int32_t *list_idx) {
  if (!c) return QG_ERR_ARG;
  return set_cells_common(c, nc, com, m, q, list_off, list_idx, 0, false, c->stream);
}

qg_status qg_set_cells_dev(qg_ctx *c, int64_t nc, const double *com, const double *m, const double *q,
                           const int64_t *list_off, const int32_t *list_idx, int64_t n_list, void *stream) {
  if (!c) return QG_ERR_ARG;
  return set_cells_common(c, nc, com, m, q, list_off, list_idx, n_list, true, pick_stream(c, stream));
}

qg_status qg_run(qg_ctx *c, void *stream) {
  if (!c) return QG_ERR_ARG;
  if (!c->sinks_ok || !c->src_ok || !c->cells_ok)
    return fail(c, QG_ERR_STATE, "qg_run: sinks, sources and cells must all be set");
  if (c->G_src != c->G || c->G_cell != c->G)
    return fail(c, QG_ERR_STATE, "qg_run: lists were set for %lld / %lld groups, sinks have %lld",
                (long long)c->G_src, (long long)c->G_cell, (long long)c->G);
  DeviceGuard dg(c->device);
  cudaStream_t s = pick_stream(c, stream);
  c->last_stream = s;
  if (c->G == 0) {
    c->ran = true;
    return QG_OK;
  }
  qg_status st = ensure_graph(c);
  if (st != QG_OK) return st;
  QG_CUDA(c, cudaGraphLaunch(c->exec, s));
  c->ran = true;
  c->timed = true;
  return QG_OK;
}

qg_status qg_get_forces(qg_ctx *c, double *a, double *phi) {
  if (!c) return QG_ERR_ARG;
  if (!c->ran) return fail(c, QG_ERR_STATE, "qg_get_forces: nothing has been run for these sinks");
  DeviceGuard dg(c->device);
  cudaStream_t s = c->last_stream;
  if (c->n == 0) {
    QG_CUDA(c, cudaStreamSynchronize(s));
    return QG_OK;
  }
  if (a) QG_CUDA(c, cudaMemcpyAsync(a, c->a.p, 3 * c->n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (phi) QG_CUDA(c, cudaMemcpyAsync(phi, c->phi.p, c->n * sizeof(double), cudaMemcpyDeviceToHost, s));
  QG_CUDA(c, cudaStreamSynchronize(s));
  return QG_OK;
}

qg_status qg_get_forces_dev(qg_ctx *c, double *a, double *phi, void *stream) {
  if (!c) return QG_ERR_ARG;
  if (!c->ran) return fail(c, QG_ERR_STATE, "qg_get_forces_dev: nothing has been run for these sinks");
  if (c->n == 0) return QG_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = pick_stream(c, stream);
  if (a) QG_CUDA(c, cudaMemcpyAsync(a, c->a.p, 3 * c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (phi) QG_CUDA(c, cudaMemcpyAsync(phi, c->phi.p, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return QG_OK;
}

qg_status qg_get_stats(const qg_ctx *c, qg_stats *out) {
  if (!c || !out) return QG_ERR_ARG;
  *out = c->stats;
  return QG_OK;
}

qg_status qg_autotune(qg_ctx *c, void *stream, int reps, qg_options *best, float *best_ms) {
  if (!c || reps < 1) return c ? fail(c, QG_ERR_ARG, "qg_autotune: reps must be >= 1") : QG_ERR_ARG;
  if (!c->sinks_ok || !c->src_ok || !c->cells_ok || c->G_src != c->G || c->G_cell != c->G)
    return fail(c, QG_ERR_STATE, "qg_autotune: sinks, sources and cells must all be set");
  DeviceGuard dg(c->device);
  cudaStream_t s = pick_stream(c, stream);
  const qg_options base = c->opt;
  qg_options chosen = base;
  float chosen_ms = 0.f;
  if (c->G > 0) {
    // candidates: sinks per thread x warps x tile, in the scalar and the
    // entry-paired FP32 forms (the sink-paired form was slower at every
    // shape on every workload measured, so it is not tried)
    std::vector<qg_options> cand;
    const int Rs[3] = {2, 4, 8}, Ws[3] = {2, 4, 8}, Ts[4] = {128, 256, 512, 1024};
    const bool fp32c = base.precision == QG_FP32_CENTRED;
    for (int ai = 0; ai < (fp32c ? 2 : 1); ai++)
      for (int R : Rs)
        for (int W : Ws)
          for (int T : Ts) {
            qg_options o = base;
            o.sinks_per_thread = R;
            o.warps_per_group = W;
            o.tile_j = T;
            o.sinks_adaptive = 0;
            if (fp32c) o.arith = ai == 0 ? QG_ARITH_ENTRY_PAIRED : QG_ARITH_SCALAR;
            if (base.precision == QG_FP64 && R != 2) continue;
            if (R >= 8 && W > 4) continue;
            if (o.arith == QG_ARITH_ENTRY_PAIRED && R > 4) continue;
            cand.push_back(o);
            if (fp32c && R == 4) {  // the same shape with sinks per thread chosen per item
              o.sinks_adaptive = 1;
              cand.push_back(o);
            }
          }
    // mean force-kernel time of `runs` graph replays at options o (after
    // `warm` untimed ones); < 0 if the shape does not fit this device
    auto time_shape = [&](const qg_options &o, int warm, int runs, float *ms_out) -> qg_status {
      c->opt = o;
      invalidate(c);
      qg_status st = ensure_graph(c);
      if (st == QG_ERR_ARG) {
        *ms_out = -1.f;
        return QG_OK;
      }
      if (st != QG_OK) return st;
      float tot = 0.f;
      for (int k = 0; k < warm + runs; k++) {
        QG_CUDA(c, cudaGraphLaunch(c->exec, s));
        QG_CUDA(c, cudaStreamSynchronize(s));
        float ms = 0.f;
        QG_CUDA(c, cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]));
        if (k >= warm) tot += ms;
      }
      *ms_out = tot / runs;
      return QG_OK;
    };
    // stage 1: every shape once (one untimed run first where a run is short);
    // stage 2: the four fastest again, one untimed and `reps` timed runs each
    std::vector<std::pair<float, int>> first;
    for (int i = 0; i < (int)cand.size(); i++) {
      float ms = 0.f;
      qg_status st = time_shape(cand[i], 0, 1, &ms);
      if (st == QG_OK && ms >= 0.f && ms < 1.f) st = time_shape(cand[i], 0, 1, &ms);  // short: time it warm
      if (st != QG_OK) {
        c->opt = base;
        invalidate(c);
        return st;
      }
      if (ms >= 0.f) first.emplace_back(ms, i);
    }
    if (first.empty()) {
      c->opt = base;
      invalidate(c);
      return fail(c, QG_ERR_ARG, "qg_autotune: no launch shape fits this device");
    }
    std::sort(first.begin(), first.end());
    bool have = false;
    for (int k = 0; k < (int)first.size() && k < 4; k++) {
      float ms = 0.f;
      qg_status st = time_shape(cand[first[k].second], 1, reps, &ms);
      if (st != QG_OK) {
        c->opt = base;
        invalidate(c);
        return st;
      }
      if (!have || ms < chosen_ms) {
        have = true;
        chosen = cand[first[k].second];
        chosen_ms = ms;
      }
    }
  }
  c->opt = chosen;
  invalidate(c);
  if (c->G > 0) {
    qg_status st = ensure_graph(c);
    if (st != QG_OK) return st;
    QG_CUDA(c, cudaGraphLaunch(c->exec, s));
    QG_CUDA(c, cudaStreamSynchronize(s));
  }
  c->last_stream = s;
  c->ran = true;
  if (best) *best = chosen;
  if (best_ms) *best_ms = chosen_ms;
  return QG_OK;
}

qg_status qg_last_timing(qg_ctx *c, float *step_ms, float *force_ms) {
  if (!c) return QG_ERR_ARG;
  if (!c->ran || !c->timed) return fail(c, QG_ERR_STATE, "qg_last_timing: no timed run");
  DeviceGuard dg(c->device);
  QG_CUDA(c, cudaStreamSynchronize(c->last_stream));
  if (step_ms) QG_CUDA(c, cudaEventElapsedTime(step_ms, c->ev[0], c->ev[2]));
  if (force_ms) QG_CUDA(c, cudaEventElapsedTime(force_ms, c->ev[1], c->ev[2]));
  return QG_OK;
}

// Device address of page-locked host memory at h, or nullptr when the
// device cannot address it in place.  In-place access is only used on a GPU
// that reads host memory through the host's own page tables (a coherent
// CPU-GPU link): there every valid host address is reachable, so an array
// that starts in a page-locked allocation and runs past its end still reads
// correctly.
const void *in_place(qg_ctx *c, const void *h) {
  if (c->coherent_host < 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccessUsesHostPageTables, c->device) != cudaSuccess)
      v = 0;
    c->coherent_host = v ? 1 : 0;
  }
  if (!c->coherent_host || !h) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// One evaluation from host arrays.  The offsets, sinks, sources and cells
// are copied first, and each is packed as soon as it is there.  The lists
// are then either read in place by one
// persistent launch (page-locked host memory on a coherent link) or copied
// in chunks of groups on a second stream while the force kernel runs on the
// chunks already there, each chunk's results copied back on a third stream
// as soon as its kernel ends.
qg_status qg_evaluate_host(qg_ctx *c, int64_t n, const double *sink_x, const float *sink_eps2, double eps2_all,
                           int64_t ngroups, const int64_t *group_off, int64_t ns, const double *src_x,
                           const double *src_m, const int64_t *plist_off, const int32_t *plist_idx, int64_t nc,
                           const double *cell_com, const double *cell_m, const double *cell_q,
                           const int64_t *clist_off, const int32_t *clist_idx, double *a, double *phi) {
  if (!c) return QG_ERR_ARG;
  constexpr int kChunks = 4;
  // inputs must not change under a step that is still running
  if (c->last_stream) cudaStreamSynchronize(c->last_stream);
  c->sinks_ok = c->src_ok = c->cells_ok = false;
  c->ran = false;
  invalidate(c);
  // ---- host-side checks (the same as the qg_set_* calls)
  if (n < 0 || ngroups < 0 || ngroups >= INT32_MAX || !group_off || (n > 0 && (!sink_x || !a || !phi)))
    return fail(c, QG_ERR_ARG, "qg_evaluate_host: bad sink sizes or NULL pointer");
  if (!(eps2_all >= 0 && eps2_all <= qg::kMaxInput))
    return fail(c, QG_ERR_ARG, "qg_evaluate_host: eps2_all must be finite, >= 0 and at most 2^100");
  if (ns < 0 || ns >= INT32_MAX || !plist_off || (ns > 0 && (!src_x || !src_m)))
    return fail(c, QG_ERR_ARG, "qg_evaluate_host: bad source sizes or NULL pointer");
  if (nc < 0 || nc >= INT32_MAX || !clist_off || (nc > 0 && (!cell_com || !cell_m || !cell_q)))
    return fail(c, QG_ERR_ARG, "qg_evaluate_host: bad cell sizes or NULL pointer");
  const int64_t G = ngroups;
  // the offsets' end points here; that they never decrease is checked while
  // the first copies run (no kernel is queued before that)
  if (group_off[0] != 0 || group_off[G] != n) return fail(c, QG_ERR_ARG, "qg_evaluate_host: bad group offsets");
  const int64_t np_tot = plist_off[G], nc_tot = clist_off[G];
  if (plist_off[0] != 0 || clist_off[0] != 0 || np_tot < 0 || nc_tot < 0)
    return fail(c, QG_ERR_ARG, "qg_evaluate_host: bad list offsets");
  if ((np_tot > 0 && !plist_idx) || (nc_tot > 0 && !clist_idx))
    return fail(c, QG_ERR_ARG, "qg_evaluate_host: list_idx is NULL");
  // with no sources (cells) every entry of a non-empty list is out of range
  if ((np_tot > 0 && ns == 0) || (nc_tot > 0 && nc == 0))
    return fail(c, QG_ERR_ARG, "qg_evaluate_host: list entries but no sources or cells");
  DeviceGuard dg(c->device);
  cudaStream_t s = c->stream;
  if (!c->copy_in) QG_CUDA(c, cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking));
  if (!c->copy_out) QG_CUDA(c, cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking));
  if (!c->inputs_ready) QG_CUDA(c, cudaEventCreateWithFlags(&c->inputs_ready, cudaEventDisableTiming));
  if (!c->offsets_ready) QG_CUDA(c, cudaEventCreateWithFlags(&c->offsets_ready, cudaEventDisableTiming));
  if (!c->sinks_ready) QG_CUDA(c, cudaEventCreateWithFlags(&c->sinks_ready, cudaEventDisableTiming));
  if (!c->packed) QG_CUDA(c, cudaEventCreateWithFlags(&c->packed, cudaEventDisableTiming));
  if (!c->hbad) QG_CUDA(c, cudaMallocHost(&c->hbad, kChunks * sizeof(int)));
  for (int k = 0; k < kChunks; k++) {
    if (!c->chunk_stream[k]) QG_CUDA(c, cudaStreamCreateWithFlags(&c->chunk_stream[k], cudaStreamNonBlocking));
    if (!c->chunk_in[k]) QG_CUDA(c, cudaEventCreateWithFlags(&c->chunk_in[k], cudaEventDisableTiming));
    if (!c->chunk_done[k]) QG_CUDA(c, cudaEventCreateWithFlags(&c->chunk_done[k], cudaEventDisableTiming));
  }
  c->n = n;
  c->G = G;
  c->has_eps2 = sink_eps2 != nullptr;
  c->eps2_all = eps2_all;
  qg_status st;
  // ---- outputs, queue and per-chunk scratch (hist, cursor, head, bad);
  // allocations first, before any copy is queued
  constexpr int kScr = 2 * kBuckets + 2;
  cudaError_t e;
  if ((e = c->scratch.reserve(kChunks * kScr)) != cudaSuccess || (e = c->bucket.reserve(G)) != cudaSuccess ||
      (e = c->queue.reserve(G)) != cudaSuccess || (e = c->a.reserve(3 * std::max<int64_t>(n, 1))) != cudaSuccess ||
      (e = c->phi.reserve(std::max<int64_t>(n, 1))) != cudaSuccess || (e = c->pidx.reserve(np_tot)) != cudaSuccess ||
      (e = c->cidx.reserve(nc_tot)) != cudaSuccess)
    return fail(c, QG_ERR_NOMEM, "device allocation: %s", cudaGetErrorString(e));
  // ---- offsets, sinks and sources, cells: every host-to-device copy goes
  // on one stream (copy_in), in that order and the list chunks after them, so
  // the copy engine takes them in that order.  On s, the queue waits for the
  // offsets, the group centres and the source packing for the sinks and
  // sources (while the cells are still being copied), the cell packing for
  // the cells.  One copy of x when the sinks are the sources.
  cudaStream_t ci_s = c->copy_in;
  if ((st = upload(c, c->goff, group_off, G + 1, ci_s)) != QG_OK) return st;
  if ((st = upload(c, c->poff, plist_off, G + 1, ci_s)) != QG_OK) return st;
  if ((st = upload(c, c->coff, clist_off, G + 1, ci_s)) != QG_OK) return st;
  c->p_ranges = c->c_ranges = false;  // CSR lists
  QG_CUDA(c, cudaEventRecord(c->offsets_ready, ci_s));
  if ((st = upload(c, c->sink_x, sink_x, 3 * n, ci_s)) != QG_OK) return st;
  if (sink_eps2 && (st = upload(c, c->sink_eps2, sink_eps2, n, ci_s)) != QG_OK) return st;
  if ((st = upload(c, c->src_m64, src_m, ns, ci_s)) != QG_OK) return st;
  const bool same_x = src_x == sink_x && ns == n;
  if (!same_x && (st = upload(c, c->stage_src, src_x, 3 * ns, ci_s)) != QG_OK) return st;
  QG_CUDA(c, cudaEventRecord(c->sinks_ready, ci_s));
  if ((st = upload(c, c->stage_x, cell_com, 3 * nc, ci_s)) != QG_OK) return st;
  if ((st = upload(c, c->cell_m64, cell_m, nc, ci_s)) != QG_OK) return st;
  if (c->cell_pm.reserve(nc) != cudaSuccess || c->cell_q.reserve(2 * nc) != cudaSuccess ||
      c->cell_q64.reserve(6 * nc) != cudaSuccess || c->src.reserve(ns) != cudaSuccess ||
      c->src_f.reserve(ns) != cudaSuccess || c->cell_f.reserve(nc) != cudaSuccess)
    return fail(c, QG_ERR_NOMEM, "source or cell allocation");
  if ((st = upload(c, c->cell_q64, cell_q, 6 * nc, ci_s)) != QG_OK) return st;
  QG_CUDA(c, cudaEventRecord(c->inputs_ready, ci_s));
  // ---- the host-side checks that take a pass over the offsets or the
  // softenings, while those copies run; the kernel choice depends on them
  bool ok = valid_offsets(group_off, G, n) && valid_offsets_any_total(plist_off, G) &&
            valid_offsets_any_total(clist_off, G);
  bool pos = eps2_all >= 0x1p-126;
  int64_t bad_eps = -1;
  if (ok && sink_eps2) {
    pos = true;
    for (int64_t i = 0; i < n && bad_eps < 0; i++) {
      if (!(sink_eps2[i] >= 0.f && (double)sink_eps2[i] <= qg::kMaxInput)) bad_eps = i;
      if (!(sink_eps2[i] >= 0x1p-126f)) pos = false;
    }
  }
  if (!ok || bad_eps >= 0) {
    cudaStreamSynchronize(ci_s);  // the copies still read the caller's arrays
    if (!ok) return fail(c, QG_ERR_ARG, "qg_evaluate_host: offsets decrease");
    return fail(c, QG_ERR_ARG, "qg_evaluate_host: eps2[%lld] invalid", (long long)bad_eps);
  }
  c->eps_positive = pos;
  if ((st = choose_kernel(c)) != QG_OK) {
    cudaStreamSynchronize(ci_s);
    return st;
  }
  // ---- in place: lists and results in page-locked memory the device reads
  // and writes over a coherent link (FP32 centred, scalar or entry-paired
  // form).  One queue and one persistent launch over all groups; the kernel
  // reads each list index from the host, checks it and keeps it in the
  // device lists, and writes the results both to the device buffers and to
  // a / phi.  No list copy, no copy back.
  const void *pi_h = np_tot > 0 ? in_place(c, plist_idx) : nullptr, *ci_h = nc_tot > 0 ? in_place(c, clist_idx) : nullptr;
  const void *a_h = n > 0 ? in_place(c, a) : nullptr, *phi_h = n > 0 ? in_place(c, phi) : nullptr;
  const bool direct = c->kernel_inplace && n > 0 && G > 0 && (np_tot == 0 || pi_h) && (nc_tot == 0 || ci_h) && a_h &&
                      phi_h;
  c->stats.eval_in_place = direct ? 1 : 0;
  QG_CUDA(c, cudaStreamWaitEvent(s, c->offsets_ready, 0));
  QG_CUDA(c, cudaMemsetAsync(c->scratch.p, 0, kChunks * kScr * sizeof(int), s));
  if (direct) {  // the queue needs the offsets only
    int *hist = c->scratch.p, *cursor = hist + kBuckets;
    const double cell_ops = c->opt.expansion == QG_QUAD ? 33.0 : 13.0;
    queue_hist_kernel<<<grid_for(G, 256), 256, 0, s>>>(G, c->goff.p, c->poff.p, pend_dev(c), c->coff.p,
                                                        cend_dev(c), cell_ops, c->bucket.p, hist);
    queue_scatter_kernel<<<grid_for(G, 256), 256, 0, s>>>(G, c->bucket.p, hist, cursor, c->queue.p);
    QG_CUDA(c, cudaGetLastError());
  }
  // input values are checked into the first chunk's flag (the kernels below
  // still run on them, reading nothing out of bounds; the call then fails)
  int *vflags = c->scratch.p + 2 * kBuckets + 1;
  QG_CUDA(c, cudaStreamWaitEvent(s, c->sinks_ready, 0));
  if ((st = group_centres(c, n, G, nullptr, vflags, s)) != QG_OK) {
    cudaStreamSynchronize(ci_s);
    return st;
  }
  if (ns)
    pack_src_kernel<<<grid_for(ns, 256), 256, 0, s>>>(ns, same_x ? c->sink_x.p : c->stage_src.p, c->src_m64.p,
                                                      c->src.p, c->src_f.p, vflags);
  QG_CUDA(c, cudaStreamWaitEvent(s, c->inputs_ready, 0));
  if (nc)
    pack_cells_kernel<<<grid_for(nc, 256), 256, 0, s>>>(nc, c->stage_x.p, c->cell_m64.p, c->cell_q64.p,
                                                         c->cell_pm.p, c->cell_f.p, c->cell_q.p, c->cell_q64.p,
                                                         vflags);
  QG_CUDA(c, cudaGetLastError());
  QG_CUDA(c, cudaEventRecord(c->ev[0], s));
  if (direct) {
    int *head = c->scratch.p + 2 * kBuckets, *bad = head + 1;
    qg::ForceParams fp = force_params(c, 0, G, head);
    fp.plist_idx = static_cast<const int32_t *>(pi_h);
    fp.clist_idx = static_cast<const int32_t *>(ci_h);
    fp.plist_keep = c->pidx.p;
    fp.clist_keep = c->cidx.p;
    fp.n_src = (int32_t)ns;
    fp.n_cell = (int32_t)nc;
    fp.bad = bad;
    fp.a_host = static_cast<double *>(const_cast<void *>(a_h));
    fp.phi_host = static_cast<double *>(const_cast<void *>(phi_h));
    const int grid = (int)std::min<int64_t>(c->grid_inplace, G);
    void *args[] = {&fp};
    QG_CUDA(c, cudaEventRecord(c->ev[1], s));
    QG_CUDA(c, cudaLaunchKernel(c->kernel_inplace, dim3(grid), dim3(c->nthreads), args, c->smem, s));
    QG_CUDA(c, cudaEventRecord(c->ev[2], s));
    c->stats.grid = grid;
    QG_CUDA(c, cudaMemcpyAsync(c->hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  } else {
    QG_CUDA(c, cudaEventRecord(c->packed, s));
    // ---- chunks of groups by list entries: 1/8, 1/4, 1/4, 3/8 of them, so
    // that the first kernel waits for a small first copy
    int64_t gb[kChunks + 1];
    gb[0] = 0;
    {
      const int64_t total = np_tot + nc_tot;
      const int eighths[kChunks] = {1, 3, 5, 8};  // cumulative, in eighths
      int64_t g = 0;
      for (int k = 1; k < kChunks; k++) {
        const int64_t want = total / 8 * eighths[k - 1];
        while (g < G && plist_off[g] + clist_off[g] < want) g++;
        gb[k] = g;
      }
      gb[kChunks] = G;
    }
    for (int k = 0; k < kChunks; k++) {
      const int64_t g0 = gb[k], g1 = gb[k + 1];
      const int64_t p0 = plist_off[g0], p1 = plist_off[g1], c0 = clist_off[g0], c1 = clist_off[g1];
      if (p1 > p0)
        QG_CUDA(c, cudaMemcpyAsync(c->pidx.p + p0, plist_idx + p0, (p1 - p0) * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, c->copy_in));
      if (c1 > c0)
        QG_CUDA(c, cudaMemcpyAsync(c->cidx.p + c0, clist_idx + c0, (c1 - c0) * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, c->copy_in));
      QG_CUDA(c, cudaEventRecord(c->chunk_in[k], c->copy_in));
    }
    // each chunk on its own stream, so that a chunk's kernel fills the SMs its
    // predecessor's last groups leave idle
    const double cell_ops = c->opt.expansion == QG_QUAD ? 33.0 : 13.0;
    for (int k = 0; k < kChunks; k++) {
      const int64_t g0 = gb[k], g1 = gb[k + 1], Gk = g1 - g0;
      int *hist = c->scratch.p + k * kScr, *cursor = hist + kBuckets, *head = cursor + kBuckets, *bad = head + 1;
      cudaStream_t sk = c->chunk_stream[k];
      QG_CUDA(c, cudaStreamWaitEvent(sk, c->packed, 0));
      QG_CUDA(c, cudaStreamWaitEvent(sk, c->chunk_in[k], 0));
      if (Gk > 0) {
        const int64_t p0 = plist_off[g0], p1 = plist_off[g1], c0 = clist_off[g0], c1 = clist_off[g1];
        if (p1 > p0) sanitize_index_kernel<<<grid_for(p1 - p0, 256), 256, 0, sk>>>(p1 - p0, c->pidx.p + p0, ns, bad);
        if (c1 > c0) sanitize_index_kernel<<<grid_for(c1 - c0, 256), 256, 0, sk>>>(c1 - c0, c->cidx.p + c0, nc, bad);
        queue_hist_kernel<<<grid_for(Gk, 256), 256, 0, sk>>>(Gk, c->goff.p + g0, c->poff.p + g0, pend_dev(c) + g0,
                                                             c->coff.p + g0, cend_dev(c) + g0, cell_ops,
                                                             c->bucket.p + g0, hist);
        queue_scatter_kernel<<<grid_for(Gk, 256), 256, 0, sk>>>(Gk, c->bucket.p + g0, hist, cursor, c->queue.p + g0);
        QG_CUDA(c, cudaGetLastError());
        qg::ForceParams fp = force_params(c, g0, Gk, head);
        const int grid = (int)std::min<int64_t>(c->grid, Gk);
        void *args[] = {&fp};
        if (k == 0) QG_CUDA(c, cudaEventRecord(c->ev[1], sk));
        QG_CUDA(c, cudaLaunchKernel(c->kernel, dim3(grid), dim3(c->nthreads), args, c->smem, sk));
      } else if (k == 0) {
        QG_CUDA(c, cudaEventRecord(c->ev[1], sk));
      }
      QG_CUDA(c, cudaEventRecord(c->chunk_done[k], sk));
      QG_CUDA(c, cudaStreamWaitEvent(s, c->chunk_done[k], 0));
      // results of this chunk's sinks back to the host
      const int64_t s0 = group_off[g0], s1 = group_off[g1];
      QG_CUDA(c, cudaStreamWaitEvent(c->copy_out, c->chunk_done[k], 0));
      if (s1 > s0) {
        QG_CUDA(c, cudaMemcpyAsync(a + 3 * s0, c->a.p + 3 * s0, 3 * (s1 - s0) * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->copy_out));
        QG_CUDA(c, cudaMemcpyAsync(phi + s0, c->phi.p + s0, (s1 - s0) * sizeof(double), cudaMemcpyDeviceToHost,
                                   c->copy_out));
      }
    }
    QG_CUDA(c, cudaEventRecord(c->ev[2], s));
    c->stats.grid = (int)std::min<int64_t>(c->grid, std::max<int64_t>(G, 1));
    for (int k = 0; k < kChunks; k++)
      QG_CUDA(c, cudaMemcpyAsync(&c->hbad[k], c->scratch.p + k * kScr + 2 * kBuckets + 1, sizeof(int),
                                 cudaMemcpyDeviceToHost, c->copy_out));
  }
  // the context now holds these inputs, as after the qg_set_* calls and
  // qg_run (recorded while the kernel runs; undone below if an entry was bad)
  c->h_goff.assign(group_off, group_off + G + 1);
  c->h_poff.assign(plist_off, plist_off + G + 1);
  c->h_coff.assign(clist_off, clist_off + G + 1);
  c->ns = ns;
  c->nc = nc;
  c->G_src = c->G_cell = G;
  c->np_list = np_tot;
  c->nc_list = nc_tot;
  c->sinks_ok = c->src_ok = c->cells_ok = true;
  update_counts(c);
  c->last_stream = s;
  if (!direct) QG_CUDA(c, cudaStreamSynchronize(c->copy_out));
  QG_CUDA(c, cudaStreamSynchronize(s));
  for (int k = 0; k < (direct ? 1 : kChunks); k++)
    if (c->hbad[k]) {
      c->sinks_ok = c->src_ok = c->cells_ok = false;
      return fail(c, QG_ERR_ARG,
                  "qg_evaluate_host: a list entry outside its source or cell range, or an input value that is "
                  "not finite or exceeds 2^100");
    }
  c->ran = true;
  c->timed = true;
  return QG_OK;
}

const char *qg_last_error(const qg_ctx *c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"

// qg_gtree_attach_move: the three qg_set_*_dev calls in one, for a tree the
// library built and walked itself.  The list buffers are exchanged rather
// than copied and their indices are not checked (the walk produced them);
// positions, masses and moments are checked by the same kernels, and one
// synchronisation reads the checks and the host copies of the offsets.
qg_status qg::attach_tree_lists(qg_ctx *c, qg::TreeLists &t, double eps2_all, cudaStream_t s) {
  if (!c) return QG_ERR_ARG;
  // inputs must not change under a step that is still running
  if (c->last_stream) cudaStreamSynchronize(c->last_stream);
  c->sinks_ok = c->src_ok = c->cells_ok = false;
  invalidate(c);
  if (t.n < 0 || t.n >= INT32_MAX || t.G < 0 || t.G >= INT32_MAX || t.nn < 0 || t.nn >= INT32_MAX ||
      !t.poff || !t.coff || !t.pidx || !t.cidx || (t.ranges && (!t.pend || !t.cend)) || !t.goff ||
      (t.n > 0 && (!t.xs || !t.ms)) ||
      (t.nn > 0 && (!t.com || !t.mass || !t.q)))
    return fail(c, QG_ERR_ARG, "attach: bad sizes or NULL pointer");
  if (t.device != c->device) return fail(c, QG_ERR_ARG, "attach: the tree and the context are on different devices");
  if (!(eps2_all >= 0 && eps2_all <= qg::kMaxInput))
    return fail(c, QG_ERR_ARG, "attach: eps2_all must be finite, >= 0 and at most 2^100");
  DeviceGuard dg(c->device);
  const int64_t n = t.n, G = t.G, nc = t.nn;
  qg_status st;
  if ((st = copy_d2d(c, c->sink_x, t.xs, 3 * n, s)) != QG_OK) return st;
  if ((st = copy_d2d(c, c->goff, t.goff, G + 1, s)) != QG_OK) return st;
  std::swap(c->poff, *t.poff);
  std::swap(c->pidx, *t.pidx);
  std::swap(c->coff, *t.coff);
  std::swap(c->cidx, *t.cidx);
  if (t.ranges) {
    std::swap(c->pend, *t.pend);
    std::swap(c->cend, *t.cend);
  }
  c->p_ranges = c->c_ranges = t.ranges;
  if ((st = copy_d2d(c, c->src_m64, t.ms, n, s)) != QG_OK) return st;
  if ((st = copy_d2d(c, c->cell_m64, t.mass, nc, s)) != QG_OK) return st;
  if (c->src.reserve(n) != cudaSuccess || c->src_f.reserve(n) != cudaSuccess || c->cell_pm.reserve(nc) != cudaSuccess ||
      c->cell_f.reserve(nc) != cudaSuccess || c->cell_q.reserve(2 * nc) != cudaSuccess ||
      c->cell_q64.reserve(6 * nc) != cudaSuccess)
    return fail(c, QG_ERR_NOMEM, "attach: source and cell allocation");
  int *flags = nullptr;
  if ((st = value_flags_begin(c, s, &flags)) != QG_OK) return st;
  if ((st = group_centres(c, n, G, nullptr, flags, s)) != QG_OK) return st;
  if (n) pack_src_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, t.xs, c->src_m64.p, c->src.p, c->src_f.p, flags);
  if (nc)
    pack_cells_kernel<<<grid_for(nc, 256), 256, 0, s>>>(nc, t.com, c->cell_m64.p, t.q, c->cell_pm.p, c->cell_f.p,
                                                         c->cell_q.p, c->cell_q64.p, flags);
  QG_CUDA(c, cudaGetLastError());
  // host copies of the offsets (CSR: G + 1 of them; ranges: G begins and
  // G ends per list) and the value checks, with one synchronisation
  const int64_t nb = t.ranges ? G : G + 1;
  std::vector<int64_t> hg(G + 1), hp(nb), hc(nb), hpe(t.ranges ? G : 0), hce(t.ranges ? G : 0);
  QG_CUDA(c, cudaMemcpyAsync(hg.data(), c->goff.p, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (nb > 0) {
    QG_CUDA(c, cudaMemcpyAsync(hp.data(), c->poff.p, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QG_CUDA(c, cudaMemcpyAsync(hc.data(), c->coff.p, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  }
  if (t.ranges && G > 0) {
    QG_CUDA(c, cudaMemcpyAsync(hpe.data(), c->pend.p, G * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QG_CUDA(c, cudaMemcpyAsync(hce.data(), c->cend.p, G * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  }
  int fl = 0;
  if ((st = value_flags_end(c, s, flags, &fl)) != QG_OK) return st;
  if (fl & kBadPosition)
    return fail(c, QG_ERR_ARG, "attach: a position, mass or quadrupole component is not finite or exceeds 2^100");
  int64_t tp = 0, tc = 0;
  if (t.ranges) {
    for (int64_t g = 0; g < G; g++) {
      tp += hpe[g] - hp[g];
      tc += hce[g] - hc[g];
    }
  } else {
    tp = hp[G];
    tc = hc[G];
  }
  if (tp != t.np_list || tc != t.nc_list || hg[G] != n)
    return fail(c, QG_ERR_STATE, "attach: the tree's list sizes do not match its offsets");
  c->n = n;
  c->G = G;
  c->has_eps2 = false;
  c->eps2_all = eps2_all;
  c->eps_positive = eps2_all >= 0x1p-126;
  c->h_goff.swap(hg);
  c->sinks_ok = true;
  c->ran = false;
  c->ns = n;
  c->G_src = G;
  c->np_list = t.np_list;
  c->h_poff.swap(hp);
  c->h_pend.swap(hpe);
  c->src_ok = true;
  c->nc = nc;
  c->G_cell = G;
  c->nc_list = t.nc_list;
  c->h_coff.swap(hc);
  c->h_cend.swap(hce);
  c->cells_ok = true;
  update_counts(c);
  return QG_OK;
}
