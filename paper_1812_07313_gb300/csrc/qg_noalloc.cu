// qg_noalloc.cu -- qg_forces_noalloc: one force evaluation that allocates no
// memory, host or device.
//
// Some callers cannot allocate: a host code whose device memory is owned by
// its own pool or arena (it hands out slices of one up-front allocation and
// forbids cudaMalloc behind its back), or a time-stepping loop that must not
// allocate after start-up because cudaMalloc / cudaFree can block or
// synchronise the device in the middle of a step.  This entry point takes
// every input and output as caller-owned device arrays in the qg_set_*_dev
// layouts, and keeps the only scratch it needs -- the work queue of the step
// (group order, cost classes, counters) -- in one fixed file-scope device
// array, g_scratch, sized for at most QG_NOALLOC_MAX_GROUPS groups.
//
// The array lives in every GPU that loads this library until the process
// exits.  All calls on a device share it and it keeps the last call's
// contents: each call clears the counters it relies on, and two calls whose
// work overlaps on the GPU (different streams, or host threads racing)
// corrupt each other's queue.  The first call on a device looks the array's
// device address up (cudaGetSymbolAddress, with that device current) and
// caches it together with the kernels' occupancy.  Every call also waits on
// the host for its argument check: it copies the check's flags back and
// synchronises the caller's stream before it launches the step.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "qg_force.cuh"
#include "qg_internal.h"
#include "qg_queue.cuh"
#include "qgrav.h"

namespace {

constexpr int64_t kMaxGroups = QG_NOALLOC_MAX_GROUPS;
constexpr int kR = 4;           // sinks per thread
constexpr int kThreads = 128;   // threads per CTA
constexpr int kTile = 256;      // list entries per shared-memory tile
constexpr int kFlush = 256;     // list entries per thread between FP64 folds
constexpr int kMaxDevices = 64;

// scratch layout: queue int32 [kMaxGroups] | cost class uint8 [kMaxGroups] |
// counters int [hist kBuckets | cursor kBuckets | head | check flags | 2 spare]
constexpr size_t kQueueBytes = (size_t)kMaxGroups * sizeof(int32_t);
constexpr size_t kClassBytes = (size_t)kMaxGroups;
constexpr int kCounterInts = 2 * qg::kBuckets + 4;
constexpr size_t kScratchBytes = kQueueBytes + kClassBytes + kCounterInts * sizeof(int);

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSetup {
  bool ready = false;
  unsigned char *scratch = nullptr;  // device address of g_scratch on this device
  int sms = 0;
  int per_sm[2][2] = {{0, 0}, {0, 0}};  // [quad][guard] CTAs per SM
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

struct Args {
  const double *sink_x;
  const float *sink_eps2;
  float eps2_all;  // rounded to float on the host
  const int64_t *group_off;
  const double *src_x, *src_m;
  const int64_t *plist_off;
  const int32_t *plist_idx;
  const double *cell_com, *cell_m, *cell_q;
  const int64_t *clist_off;
  const int32_t *clist_idx;
  const int32_t *queue;
  int32_t nitems;
  int32_t *head;
  double *a, *phi;
};

// |v| <= kMaxInput and finite (false for NaN)
__device__ __forceinline__ bool in_range(double v) { return fabs(v) <= qg::kMaxInput; }

// The inputs checked before any force kernel reads them.  Bits of *flags:
// 1 group offsets (not starting at 0, decreasing, not ending at n, or a group
// of more than INT32_MAX sinks), 2 particle-list offsets, 4 cell-list
// offsets, 8 a particle index outside [0, ns), 16 a cell index outside
// [0, nc), 32 an input value that is not finite or exceeds kMaxInput in
// magnitude (positions, masses, quadrupole components, per-sink eps^2) or a
// negative eps^2; kGuardBit: a per-sink eps^2 below the smallest normal
// float (the kernel that skips rhat^2 == 0 pairs is needed).
constexpr int kGuardBit = 64;
__global__ void check_kernel(int64_t G, int64_t n, const int64_t *goff, const int64_t *poff, int64_t np_list,
                             const int64_t *coff, int64_t nc_list, int64_t ns, const int32_t *pidx, int64_t nc,
                             const int32_t *cidx, const double *sink_x, const float *sink_eps2,
                             const double *src_x, const double *src_m, const double *cell_com,
                             const double *cell_m, const double *cell_q, int *flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int f = 0;
  for (int64_t g = t0; g <= G; g += stride) {
    if (g == 0) {
      if (goff[0] != 0) f |= 1;
      if (poff[0] != 0) f |= 2;
      if (coff[0] != 0) f |= 4;
    }
    if (g == G) {
      if (goff[G] != n) f |= 1;
      if (poff[G] != np_list) f |= 2;
      if (coff[G] != nc_list) f |= 4;
    } else {
      if (goff[g + 1] < goff[g] || goff[g + 1] - goff[g] > (int64_t)INT32_MAX) f |= 1;
      if (poff[g + 1] < poff[g]) f |= 2;
      if (coff[g + 1] < coff[g]) f |= 4;
    }
  }
  for (int64_t i = t0; i < np_list; i += stride)
    if (pidx[i] < 0 || (int64_t)pidx[i] >= ns) f |= 8;
  for (int64_t i = t0; i < nc_list; i += stride)
    if (cidx[i] < 0 || (int64_t)cidx[i] >= nc) f |= 16;
  for (int64_t i = t0; i < 3 * n; i += stride)
    if (!in_range(sink_x[i])) f |= 32;
  if (sink_eps2)
    for (int64_t i = t0; i < n; i += stride) {
      const float e = sink_eps2[i];
      if (!(e >= 0.f && (double)e <= qg::kMaxInput)) f |= 32;
      else if (e < 0x1p-126f) f |= kGuardBit;
    }
  for (int64_t i = t0; i < 3 * ns; i += stride)
    if (!in_range(src_x[i])) f |= 32;
  for (int64_t i = t0; i < ns; i += stride)
    if (!in_range(src_m[i])) f |= 32;
  for (int64_t i = t0; i < 3 * nc; i += stride)
    if (!in_range(cell_com[i])) f |= 32;
  for (int64_t i = t0; i < nc; i += stride)
    if (!in_range(cell_m[i])) f |= 32;
  for (int64_t i = t0; i < 6 * nc; i += stride)
    if (!in_range(cell_q[i])) f |= 32;
  if (f) atomicOr(flags, f);
}

// The group-force kernel of qg_force.cuh (FP32 pairwise arithmetic, FP64
// centring and merges, the same pair functions), in a fixed launch shape and
// reading the caller's arrays in their qg_set_*_dev layouts directly instead
// of the packed records a context builds (which would need memory).
template <bool QUAD, bool GUARD>
__global__ void __launch_bounds__(kThreads) noalloc_force_kernel(const Args p) {
  __shared__ double acc64[4 * kR * kThreads];  // [4R][NT]; sink offsets alias it
  __shared__ float4 tA[kTile];
  __shared__ float4 tB[kTile];
  __shared__ float2 tC[kTile];
  __shared__ int s_item;
  __shared__ float s_box[kThreads / 32][6];
  __shared__ double s_c[3];
  float4 *sink_s = reinterpret_cast<float4 *>(acc64);
  const int NT = kThreads, tid = threadIdx.x;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(p.head, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= p.nitems) break;
    const int g = p.queue[item];
    const int64_t s0 = p.group_off[g];
    const int ni = (int)(p.group_off[g + 1] - s0);
    if (ni <= 0) continue;

    // group centre: centre of the sinks' bounding box, in FP64
    const double x0 = p.sink_x[3 * s0], y0 = p.sink_x[3 * s0 + 1], z0 = p.sink_x[3 * s0 + 2];
    float mn0 = 0.f, mn1 = 0.f, mn2 = 0.f, mx0 = 0.f, mx1 = 0.f, mx2 = 0.f;
    for (int i = tid; i < ni; i += NT) {
      const double *xi = p.sink_x + 3 * (s0 + i);
      const float o0 = qg::f64_to_f32_rn(xi[0] - x0);
      const float o1 = qg::f64_to_f32_rn(xi[1] - y0);
      const float o2 = qg::f64_to_f32_rn(xi[2] - z0);
      mn0 = fminf(mn0, o0); mn1 = fminf(mn1, o1); mn2 = fminf(mn2, o2);
      mx0 = fmaxf(mx0, o0); mx1 = fmaxf(mx1, o1); mx2 = fmaxf(mx2, o2);
    }
    mn0 = qg::warp_min(mn0); mn1 = qg::warp_min(mn1); mn2 = qg::warp_min(mn2);
    mx0 = qg::warp_max(mx0); mx1 = qg::warp_max(mx1); mx2 = qg::warp_max(mx2);
    if ((tid & 31) == 0) {
      const int w = tid >> 5;
      s_box[w][0] = mn0; s_box[w][1] = mn1; s_box[w][2] = mn2;
      s_box[w][3] = mx0; s_box[w][4] = mx1; s_box[w][5] = mx2;
    }
    __syncthreads();
    if (tid < 3) {
      float lo = s_box[0][tid], hi = s_box[0][tid + 3];
      for (int v = 1; v < NT / 32; v++) {
        lo = fminf(lo, s_box[v][tid]);
        hi = fmaxf(hi, s_box[v][tid + 3]);
      }
      s_c[tid] = (tid == 0 ? x0 : (tid == 1 ? y0 : z0)) + 0.5 * ((double)lo + (double)hi);
    }
    __syncthreads();
    const double cx = s_c[0], cy = s_c[1], cz = s_c[2];
    const int64_t p0 = p.plist_off[g], p1 = p.plist_off[g + 1];
    const int64_t c0 = p.clist_off[g], c1 = p.clist_off[g + 1];

    for (int sb = 0; sb < ni; sb += kR * NT) {
      const int nch = min(ni - sb, kR * NT);
      __syncthreads();
      for (int i = tid; i < nch; i += NT) {
        const int64_t si = s0 + sb + i;
        const double *xi = p.sink_x + 3 * si;
        const float e2 = p.sink_eps2 ? p.sink_eps2[si] : p.eps2_all;
        sink_s[i] = make_float4(qg::f64_to_f32_rn(xi[0] - cx), qg::f64_to_f32_rn(xi[1] - cy),
                                qg::f64_to_f32_rn(xi[2] - cz), e2);
      }
      __syncthreads();
      const int S = (nch + kR - 1) / kR;
      const int K = NT / S;
      const int s = tid % S, k = tid / S;
      const bool active = k < K;
      float sx[kR], sy[kR], sz[kR], se[kR], ax[kR], ay[kR], az[kR], pt[kR];
#pragma unroll
      for (int r = 0; r < kR; r++) {
        const int i = s + S * r;
        const float4 v = sink_s[i < nch ? i : 0];
        sx[r] = v.x; sy[r] = v.y; sz[r] = v.z; se[r] = v.w;
        ax[r] = ay[r] = az[r] = pt[r] = 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int v = 0; v < 4 * kR; v++) acc64[v * NT + tid] = 0.0;
      int nproc = 0;
      auto fold = [&]() {
#pragma unroll
        for (int r = 0; r < kR; r++) {
          double *q = acc64 + 4 * r * NT + tid;
          q[0] += (double)ax[r];
          q[NT] += (double)ay[r];
          q[2 * NT] += (double)az[r];
          q[3 * NT] += (double)pt[r];
          ax[r] = ay[r] = az[r] = pt[r] = 0.f;
        }
        nproc = 0;
      };

      for (int64_t base = p0; base < p1; base += kTile) {
        const int cnt = (int)min((int64_t)kTile, p1 - base);
        __syncthreads();
        for (int t = tid; t < cnt; t += NT) {
          const int64_t j = p.plist_idx[base + t];
          const double *xj = p.src_x + 3 * j;
          tA[t] = make_float4(qg::f64_to_f32_rn(xj[0] - cx), qg::f64_to_f32_rn(xj[1] - cy),
                              qg::f64_to_f32_rn(xj[2] - cz), qg::f64_to_f32_rn(p.src_m[j]));
        }
        __syncthreads();
        if (active) {
          for (int jj = k; jj < cnt; jj += K) {
            const float4 A = tA[jj];
#pragma unroll
            for (int r = 0; r < kR; r++)
              qg::mono_pair<float, GUARD>(A.x - sx[r], A.y - sy[r], A.z - sz[r], A.w, se[r], ax[r], ay[r], az[r],
                                          pt[r]);
          }
          nproc += (cnt - k + K - 1) / K;
          if (nproc >= kFlush) fold();
        }
      }
      for (int64_t base = c0; base < c1; base += kTile) {
        const int cnt = (int)min((int64_t)kTile, c1 - base);
        __syncthreads();
        for (int t = tid; t < cnt; t += NT) {
          const int64_t j = p.clist_idx[base + t];
          const double *xj = p.cell_com + 3 * j;
          tA[t] = make_float4(qg::f64_to_f32_rn(xj[0] - cx), qg::f64_to_f32_rn(xj[1] - cy),
                              qg::f64_to_f32_rn(xj[2] - cz), qg::f64_to_f32_rn(p.cell_m[j]));
          if (QUAD) {
            const double *q = p.cell_q + 6 * j;
            tB[t] = make_float4(qg::f64_to_f32_rn(q[0]), qg::f64_to_f32_rn(q[1]), qg::f64_to_f32_rn(q[2]),
                                qg::f64_to_f32_rn(q[3]));
            tC[t] = make_float2(qg::f64_to_f32_rn(q[4]), qg::f64_to_f32_rn(q[5]));
          }
        }
        __syncthreads();
        if (active) {
          for (int jj = k; jj < cnt; jj += K) {
            const float4 A = tA[jj];
            if (QUAD) {
              const float4 B = tB[jj];
              const float2 C = tC[jj];
#pragma unroll
              for (int r = 0; r < kR; r++)
                qg::quad_pair<float, GUARD>(A.x - sx[r], A.y - sy[r], A.z - sz[r], A.w, B.x, B.y, B.z, B.w, C.x,
                                            C.y, se[r], ax[r], ay[r], az[r], pt[r]);
            } else {
#pragma unroll
              for (int r = 0; r < kR; r++)
                qg::mono_pair<float, GUARD>(A.x - sx[r], A.y - sy[r], A.z - sz[r], A.w, se[r], ax[r], ay[r],
                                            az[r], pt[r]);
            }
          }
          nproc += (cnt - k + K - 1) / K;
          if (nproc >= kFlush) fold();
        }
      }

      if (active) fold();
      __syncthreads();
      for (int i = tid; i < nch; i += NT) {
        const int si = i % S, ri = i / S;
        double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
        for (int kk = 0; kk < K; kk++) {
          const double *q = acc64 + 4 * ri * NT + kk * S + si;
          m0 += q[0]; m1 += q[NT]; m2 += q[2 * NT]; m3 += q[3 * NT];
        }
        const int64_t o = s0 + sb + i;
        p.a[3 * o] = m0;
        p.a[3 * o + 1] = m1;
        p.a[3 * o + 2] = m2;
        p.phi[o] = -m3;
      }
    }
  }
}

const void *variant(bool quad, bool guard) {
  if (quad) return guard ? (const void *)noalloc_force_kernel<true, true> : (const void *)noalloc_force_kernel<true, false>;
  return guard ? (const void *)noalloc_force_kernel<false, true> : (const void *)noalloc_force_kernel<false, false>;
}

// Once per device, with that device current: the device address of the
// scratch array and the CTAs per SM of every variant.  No allocation.
qg_status setup_device(int device, DeviceSetup **out) {
  if (device < 0 || device >= kMaxDevices) return QG_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup &d = g_setup[device];
  if (!d.ready) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return QG_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return QG_ERR_CUDA;
    for (int q = 0; q < 2; q++)
      for (int gd = 0; gd < 2; gd++) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, variant(q, gd), kThreads, 0) != cudaSuccess ||
            per < 1)
          return QG_ERR_CUDA;
        d.per_sm[q][gd] = per;
      }
    d.scratch = static_cast<unsigned char *>(ptr);
    d.sms = sms;
    d.ready = true;
  }
  *out = &d;
  return QG_OK;
}

int grid_for(int64_t n, int block) {
  const int64_t b = (n + block - 1) / block;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

qg_status run(int device, int64_t n, const double *sink_x, const float *sink_eps2, double eps2_all, int64_t G,
              const int64_t *group_off, int64_t ns, const double *src_x, const double *src_m,
              const int64_t *plist_off, const int32_t *plist_idx, int64_t n_plist, int64_t nc,
              const double *cell_com, const double *cell_m, const double *cell_q, const int64_t *clist_off,
              const int32_t *clist_idx, int64_t n_clist, int expansion, double *a, double *phi,
              cudaStream_t s) {
  DeviceSetup *d = nullptr;
  qg_status st = setup_device(device, &d);
  if (st != QG_OK) return st;
  int32_t *queue = reinterpret_cast<int32_t *>(d->scratch);
  unsigned char *cls = d->scratch + kQueueBytes;
  int *counters = reinterpret_cast<int *>(d->scratch + kQueueBytes + kClassBytes);
  int *hist = counters, *cursor = counters + qg::kBuckets, *head = cursor + qg::kBuckets, *flags = head + 1;
  if (cudaMemsetAsync(counters, 0, kCounterInts * sizeof(int), s) != cudaSuccess) return QG_ERR_CUDA;
  const int64_t work = G + 1 + n_plist + n_clist + 4 * n + 4 * ns + 10 * nc;
  check_kernel<<<grid_for(work, 256), 256, 0, s>>>(G, n, group_off, plist_off, n_plist, clist_off, n_clist, ns,
                                                   plist_idx, nc, clist_idx, sink_x, sink_eps2, src_x, src_m,
                                                   cell_com, cell_m, cell_q, flags);
  int h_flags = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&h_flags, flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return QG_ERR_CUDA;
  if (h_flags & ~kGuardBit) return QG_ERR_ARG;
  if (G == 0) return QG_OK;
  const bool quad = expansion == QG_QUAD;
  const double cell_ops = quad ? 33.0 : 13.0;
  qg::queue_hist_kernel<<<grid_for(G, 256), 256, 0, s>>>(G, group_off, plist_off, plist_off + 1, clist_off,
                                                          clist_off + 1, cell_ops, cls, hist);
  if (cudaGetLastError() != cudaSuccess) return QG_ERR_CUDA;
  qg::queue_scatter_kernel<<<grid_for(G, 256), 256, 0, s>>>(G, cls, hist, cursor, queue);
  if (cudaGetLastError() != cudaSuccess) return QG_ERR_CUDA;
  Args p{sink_x, sink_eps2, (float)eps2_all, group_off, src_x, src_m, plist_off, plist_idx,
         cell_com, cell_m, cell_q, clist_off, clist_idx, queue, (int32_t)G, head, a, phi};
  // a softening that the FP32 arithmetic flushes to zero (below the smallest
  // normal float) needs the kernel that skips coincident pairs
  const bool guard = (h_flags & kGuardBit) != 0 || (sink_eps2 == nullptr && !(eps2_all >= 0x1p-126));
  const int64_t full = (int64_t)d->per_sm[quad][guard] * d->sms;
  const int grid = (int)(full < G ? full : G);
  void *args[] = {&p};
  if (cudaLaunchKernel(variant(quad, guard), dim3(grid), dim3(kThreads), args, 0, s) != cudaSuccess)
    return QG_ERR_CUDA;
  return QG_OK;
}

}  // namespace

extern "C" qg_status qg_forces_noalloc(int device, int64_t n, const double *sink_x, const float *sink_eps2,
                                       double eps2_all, int64_t ngroups, const int64_t *group_off, int64_t ns,
                                       const double *src_x, const double *src_m, const int64_t *plist_off,
                                       const int32_t *plist_idx, int64_t n_plist, int64_t nc,
                                       const double *cell_com, const double *cell_m, const double *cell_q,
                                       const int64_t *clist_off, const int32_t *clist_idx, int64_t n_clist,
                                       int expansion, double *a, double *phi, void *cuda_stream) {
  if (ngroups > kMaxGroups) return QG_ERR_SIZE;
  if (n < 0 || ngroups < 0 || ns < 0 || nc < 0 || n_plist < 0 || n_clist < 0 || ns >= INT32_MAX ||
      nc >= INT32_MAX || !(eps2_all >= 0.0 && eps2_all <= qg::kMaxInput))
    return QG_ERR_ARG;
  if (expansion != QG_QUAD && expansion != QG_MONO) return QG_ERR_ARG;
  if (!group_off || !plist_off || !clist_off) return QG_ERR_ARG;
  if (n > 0 && (!sink_x || !a || !phi)) return QG_ERR_ARG;
  if (ns > 0 && (!src_x || !src_m)) return QG_ERR_ARG;
  if (nc > 0 && (!cell_com || !cell_m || !cell_q)) return QG_ERR_ARG;
  if ((n_plist > 0 && !plist_idx) || (n_clist > 0 && !clist_idx)) return QG_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return QG_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return QG_ERR_ARG;
  const qg_status st = run(device, n, sink_x, sink_eps2, eps2_all, ngroups, group_off, ns, src_x, src_m, plist_off,
                           plist_idx, n_plist, nc, cell_com, cell_m, cell_q, clist_off, clist_idx, n_clist,
                           expansion, a, phi, (cudaStream_t)cuda_stream);
  if (prev != device) cudaSetDevice(prev);
  return st;
}
