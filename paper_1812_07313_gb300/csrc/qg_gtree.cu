// qg_gtree.cu -- oct-tree build, cell moments (Eq. 2), sink groups (Sec. 3.4)
// and the group walk on the GPU (include/qg_gtree.h).
//
// Built with -fmad=false (and the host side with -ffp-contract=off, like the
// host builder): every FP64 expression here is evaluated in the host
// builder's order without fused multiply-adds, so keys, moments and opening
// decisions are bit-for-bit the host's.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "qg_attach.h"
#include "qg_devbuf.h"
#include "qg_gtree.h"
#include "qgrav.h"

namespace {

constexpr int kMaxLevel = 21;   // 21 bits per axis -> 63-bit Morton keys
constexpr int kScanThreads = 256, kScanItems = 4, kScanTile = kScanThreads * kScanItems;
constexpr int kSortThreads = 256, kSortItems = 8, kSortTile = kSortThreads * kSortItems;
// the digit histograms give each thread of a block one of the 256 digits
static_assert(kSortThreads == 256, "radix sort blocks have one thread per digit");

template <typename T>
using DBuf = qg::DevBuf<T>;

int blocks_for(int64_t n, int per_block) {
  const int64_t b = (n + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of int32 counts into int64 offsets; out may be
// [n+1] long: out[n] receives the total when with_total.

__global__ void scan_block_kernel(int64_t n, const int32_t *__restrict__ in, int64_t *__restrict__ out,
                                  int64_t *__restrict__ sums, int64_t *__restrict__ total) {
  __shared__ int64_t s[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t tot = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = base + k < n ? (int64_t)in[base + k] : 0;
    tot += v[k];
  }
  s[threadIdx.x] = tot;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {  // Hillis-Steele over the thread totals
    const int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = s[threadIdx.x] - tot;  // exclusive prefix of this thread
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) {
    sums[blockIdx.x] = s[threadIdx.x];
    if (total && gridDim.x == 1) *total = s[threadIdx.x];  // one block: its sum is the total
  }
}

// out[j] += offs[block of j]; with in and total (the last level of a scan of
// int32 counts over several blocks), also *total = out[n - 1] + in[n - 1].
__global__ void scan_add_kernel(int64_t n, int64_t *__restrict__ out, const int64_t *__restrict__ offs,
                                const int32_t *__restrict__ in, int64_t *__restrict__ total) {
  const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  const int64_t off = offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    const int64_t j = i + (int64_t)k * kScanThreads;
    if (j < n) {
      const int64_t o = out[j] + off;
      out[j] = o;
      if (total && j == n - 1) *total = o + (int64_t)in[j];
    }
  }
}

// int64 -> int64 variant for the recursive level
__global__ void scan_block64_kernel(int64_t n, const int64_t *__restrict__ in, int64_t *__restrict__ out,
                                    int64_t *__restrict__ sums) {
  __shared__ int64_t s[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t tot = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = base + k < n ? in[base + k] : 0;
    tot += v[k];
  }
  s[threadIdx.x] = tot;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = s[threadIdx.x] - tot;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = s[threadIdx.x];
}


}  // namespace

struct qg_gtree {
  int device = 0;
  int64_t n = 0, nsys = 0, nnodes = 0, G = 0, np_list = 0, nc_list = 0;
  int leaf_max = 8, n_crit = 64;
  bool built = false, walked = false;
  bool lists_moved = false;  // the last walk's lists went to a force context (qg_gtree_attach_move)
  // the single-pass walk leaves each group's lists in the scratch arrays, in
  // the order the groups finished; the CSR lists (plist_off / plist_idx ...)
  // are made from them on the first request (csr_ready)
  bool lists_scratch = false, csr_ready = false;
  cudaStream_t walk_stream = nullptr;
  std::vector<int64_t> h_sys_off;
  // particles
  DBuf<int64_t> perm;
  DBuf<double> xs, ms;
  DBuf<int32_t> psys;
  DBuf<int64_t> sys_off;
  DBuf<unsigned long long> bmin, bmax;
  DBuf<double> lo, scale;
  // sort scratch
  DBuf<unsigned long long> keys, keys2;
  DBuf<int32_t> vals, vals2, hist;
  DBuf<int64_t> hoff;
  // tree
  DBuf<int64_t> nbeg, nend, range;
  DBuf<int32_t> nlevel, nparent, nfirst, nnchild, nsysid, flag;
  DBuf<int64_t> cstart;  // per level: the eight octant starts of each node
  DBuf<int64_t> excl;
  DBuf<double> centre, half, side, com, mass, q;
  DBuf<int32_t> morder;  // node indices grouped for the moments passes (node_bucket)
  DBuf<int> mbuckets;    // bucket sizes, cursors and starts
  std::vector<int64_t> level_begin;
  DBuf<int32_t> sys_root;
  // groups and lists
  DBuf<int32_t> gflag, gnode_at, group_node, cnt_p, cnt_c;
  DBuf<int64_t> gidx, group_off, plist_off, clist_off;
  DBuf<int32_t> plist_idx, clist_idx;
  DBuf<int64_t> scan_tmp[5];
  DBuf<int32_t> stacks;  // per-warp walk stacks
  // single-pass walk: per-warp staging areas, scratch lists in completion order
  DBuf<int32_t> stage_p, stage_c, scratch_p, scratch_c;
  DBuf<int64_t> gstart_p, gstart_c, gend_p, gend_c;  // each group's scratch list range
  DBuf<unsigned long long> cursor;
  int64_t stage_cap_p = int64_t(1) << 15, stage_cap_c = int64_t(1) << 14;
  DBuf<float4> geom;     // per node: (com - o, side) / S, ((centre - o) / S, 0) in FP32; o, S: system root cube
  DBuf<int4> topo;       // per node: (first particle, end, first child, children)
  DBuf<int> err;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

#define GT_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess)                                              \
      return e_ == cudaErrorMemoryAllocation ? QG_ERR_NOMEM : QG_ERR_CUDA; \
  } while (0)

// Exclusive scan of an int64 array in place: block scans, the block sums
// scanned recursively (one scratch level per recursion), then added back.
qg_status scan_inplace64(qg_gtree *t, int64_t m, int64_t *arr, int lvl, cudaStream_t s) {
  if (m <= 1) {
    if (m == 1) GT_CUDA(cudaMemsetAsync(arr, 0, sizeof(int64_t), s));
    return QG_OK;
  }
  if (lvl >= 4) return QG_ERR_ARG;  // beyond 2^40 elements
  const int64_t mb = (m + kScanTile - 1) / kScanTile;
  GT_CUDA(t->scan_tmp[lvl].reserve(mb));
  scan_block64_kernel<<<(unsigned)mb, kScanThreads, 0, s>>>(m, arr, arr, t->scan_tmp[lvl].p);
  GT_CUDA(cudaGetLastError());
  if (mb > 1) {
    const qg_status st = scan_inplace64(t, mb, t->scan_tmp[lvl].p, lvl + 1, s);
    if (st != QG_OK) return st;
    scan_add_kernel<<<(unsigned)mb, kScanThreads, 0, s>>>(m, arr, t->scan_tmp[lvl].p, nullptr, nullptr);
    GT_CUDA(cudaGetLastError());
  }
  return QG_OK;
}

// out[0..n) = exclusive scan of the int32 counts in; out[n] = their total
// (written by the scan's last kernel).  out must hold n + 1 elements.
qg_status scan_excl(qg_gtree *t, int64_t n, const int32_t *in, int64_t *out, cudaStream_t s) {
  if (n == 0) {
    GT_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return QG_OK;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  GT_CUDA(t->scan_tmp[0].reserve(nb));
  scan_block_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(n, in, out, t->scan_tmp[0].p, out + n);
  GT_CUDA(cudaGetLastError());
  if (nb > 1) {
    const qg_status st = scan_inplace64(t, nb, t->scan_tmp[0].p, 1, s);
    if (st != QG_OK) return st;
    scan_add_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(n, out, t->scan_tmp[0].p, in, out + n);
    GT_CUDA(cudaGetLastError());
  }
  return QG_OK;
}

// ------------------------------------------------------------------ radix sort
// Stable LSD radix sort of (uint64 key, int32 value) pairs by the low `bits`
// bits, 8 bits per pass.  Per pass: per-tile digit histograms, an exclusive
// scan over (digit, tile), and a scatter that ranks equal digits in tile order
// (warp by warp, 32 keys at a time with __match_any_sync).

__global__ void sort_hist_kernel(int64_t n, const unsigned long long *__restrict__ keys, int shift,
                                 int32_t *__restrict__ hist, int64_t nblocks) {
  __shared__ int32_t c[256];
  c[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
    const int64_t i = base + k;
    if (i < n) atomicAdd(&c[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = c[threadIdx.x];
}

__global__ void sort_scatter_kernel(int64_t n, const unsigned long long *__restrict__ kin,
                                    const int32_t *__restrict__ vin, unsigned long long *__restrict__ kout,
                                    int32_t *__restrict__ vout, int shift, const int64_t *__restrict__ offs,
                                    int64_t nblocks) {
  __shared__ int32_t wc[kSortThreads / 32][256];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = lane; d < 256; d += 32) wc[w][d] = 0;
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  // warp w owns keys [base + w * 32 * kSortItems, ...) in order
  const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)w * 32 * kSortItems;
  unsigned long long key[kSortItems];
  int32_t val[kSortItems], rank[kSortItems];
  int dig[kSortItems];
#pragma unroll
  for (int c = 0; c < kSortItems; c++) {
    const int64_t i = base + (int64_t)c * 32 + lane;
    const bool valid = i < n;
    key[c] = valid ? kin[i] : 0ull;
    val[c] = valid ? vin[i] : 0;
    const int d = valid ? (int)((key[c] >> shift) & 255) : 256;
    dig[c] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = valid ? wc[w][d] : 0;
    rank[c] = before + __popc(peers & lt);
    __syncwarp();
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wc[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over the warps
  if (threadIdx.x < 256) {
    int run = 0;
    for (int v = 0; v < kSortThreads / 32; v++) {
      const int t = wc[v][threadIdx.x];
      wc[v][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kSortItems; c++) {
    const int d = dig[c];
    if (d < 256) {
      const int64_t pos = offs[(int64_t)d * nblocks + blockIdx.x] + wc[w][d] + rank[c];
      kout[pos] = key[c];
      vout[pos] = val[c];
    }
  }
}

qg_status radix_sort(qg_gtree *t, int64_t n, int bits, cudaStream_t s) {
  // sorts t->keys / t->vals in place (ping-pong with keys2 / vals2)
  if (n <= 1) return QG_OK;
  const int64_t nb = (n + kSortTile - 1) / kSortTile;
  GT_CUDA(t->keys2.reserve(n));
  GT_CUDA(t->vals2.reserve(n));
  GT_CUDA(t->hist.reserve(256 * nb));
  GT_CUDA(t->hoff.reserve(256 * nb + 1));
  unsigned long long *ka = t->keys.p, *kb = t->keys2.p;
  int32_t *va = t->vals.p, *vb = t->vals2.p;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8, passes++) {
    sort_hist_kernel<<<(unsigned)nb, kSortThreads, 0, s>>>(n, ka, shift, t->hist.p, nb);
    GT_CUDA(cudaGetLastError());
    qg_status st = scan_excl(t, 256 * nb, t->hist.p, t->hoff.p, s);
    if (st != QG_OK) return st;
    sort_scatter_kernel<<<(unsigned)nb, kSortThreads, 0, s>>>(n, ka, va, kb, vb, shift, t->hoff.p, nb);
    GT_CUDA(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (passes & 1) {
    GT_CUDA(cudaMemcpyAsync(t->keys.p, ka, n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
    GT_CUDA(cudaMemcpyAsync(t->vals.p, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  return QG_OK;
}

// ------------------------------------------------------------------ keys

__device__ __forceinline__ unsigned long long ordered(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double unordered(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double v;
  memcpy(&v, &b, sizeof v);
  return v;
}

__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__global__ void psys_kernel(int64_t n, int64_t nsys, const int64_t *__restrict__ sys_off, int32_t *psys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = nsys;  // largest s with sys_off[s] <= i
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (sys_off[mid] <= i) lo = mid; else hi = mid;
    }
    psys[i] = (int32_t)lo;
  }
}

// per-system min / max of every coordinate (ordered integer encodings)
// Per-system bounding box (ordered-integer min / max).  Each warp scans one
// contiguous chunk and keeps a running box while the system does not change
// (systems are contiguous ranges), so the atomics are one set per warp and
// system met instead of one per 32 particles.
__global__ void bbox_kernel(int64_t n, int64_t chunk, const double *__restrict__ x, const int32_t *__restrict__ psys,
                            unsigned long long *bmin, unsigned long long *bmax) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t b0 = warp * chunk, b1 = min(n, b0 + chunk);
  int cur = -1;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  auto flush = [&]() {
    if (cur < 0) return;
#pragma unroll
    for (int d = 0; d < 3; d++) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn[d], o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx[d], o);
        mn[d] = a < mn[d] ? a : mn[d];
        mx[d] = b > mx[d] ? b : mx[d];
      }
      if (lane == 0) {
        atomicMin(&bmin[3 * cur + d], mn[d]);
        atomicMax(&bmax[3 * cur + d], mx[d]);
      }
      mn[d] = ~0ull;
      mx[d] = 0ull;
    }
  };
  for (int64_t base = b0; base < b1; base += 32) {
    const int64_t i = base + lane;
    const bool valid = i < b1;
    const int sy = valid ? psys[i] : -1;
    const int s0 = __shfl_sync(0xffffffffu, sy, 0);
    if (__all_sync(0xffffffffu, !valid || sy == s0)) {
      if (s0 != cur) {
        flush();
        cur = s0;
      }
      if (valid)
#pragma unroll
        for (int d = 0; d < 3; d++) {
          const unsigned long long k = ordered(x[3 * i + d]);
          mn[d] = k < mn[d] ? k : mn[d];
          mx[d] = k > mx[d] ? k : mx[d];
        }
    } else {  // a system boundary inside these 32 particles
      flush();
      cur = -1;
      if (valid)
        for (int d = 0; d < 3; d++) {
          const unsigned long long k = ordered(x[3 * i + d]);
          atomicMin(&bmin[3 * sy + d], k);
          atomicMax(&bmax[3 * sy + d], k);
        }
    }
  }
  flush();
}

__global__ void fill_ull_kernel(int64_t n, unsigned long long *p, unsigned long long v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void keys_kernel(int64_t n, const double *__restrict__ x, const int32_t *__restrict__ psys,
                            const double *__restrict__ lo, const double *__restrict__ scale,
                            unsigned long long *__restrict__ keys, int32_t *__restrict__ vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int s = psys[i];
    unsigned long long k = 0;
    for (int d = 0; d < 3; d++) {
      const double f = __dmul_rn(__dsub_rn(x[3 * i + d], lo[3 * s + d]), scale[s]);
      long long c = (long long)floor(f);
      c = c < 0 ? 0 : (c > (1ll << kMaxLevel) - 1 ? (1ll << kMaxLevel) - 1 : c);
      k |= spread3((unsigned long long)c) << (2 - d);
    }
    keys[i] = k;
    vals[i] = (int32_t)i;
  }
}

// after the Morton sort: the system of each sorted element as the next key
__global__ void syskey_kernel(int64_t n, const int32_t *__restrict__ vals, const int32_t *__restrict__ psys,
                              const unsigned long long *__restrict__ keys, unsigned long long *__restrict__ key2,
                              int32_t *__restrict__ pos, unsigned long long *__restrict__ morton_copy) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    key2[i] = (unsigned long long)psys[vals[i]];
    pos[i] = (int32_t)i;
    morton_copy[i] = keys[i];
  }
}

__global__ void gather_sorted_kernel(int64_t n, const int32_t *__restrict__ vals, const int32_t *__restrict__ pos,
                                     const unsigned long long *__restrict__ morton_in,
                                     unsigned long long *__restrict__ morton_out, const double *__restrict__ x,
                                     const double *__restrict__ m, int64_t *__restrict__ perm,
                                     double *__restrict__ xs, double *__restrict__ ms, int use_pos) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = use_pos ? pos[i] : i;           // position in the Morton-sorted order
    const int64_t src = use_pos ? vals[j] : vals[i];  // input index
    perm[i] = src;
    if (use_pos) morton_out[i] = morton_in[j];
    xs[3 * i] = x[3 * src];
    xs[3 * i + 1] = x[3 * src + 1];
    xs[3 * i + 2] = x[3 * src + 2];
    ms[i] = m[src];
  }
}

// ------------------------------------------------------------------ nodes

__device__ __forceinline__ int digit_at(unsigned long long key, int level) {
  return (int)((key >> (3 * (kMaxLevel - 1 - level))) & 7);
}

// Children of the open nodes of one level (more than leaf_max particles,
// level below kMaxLevel): eight lanes per node, lane o finds where octant o
// starts in the node's key range -- the digit at this level never decreases
// inside a node's range -- so octant o holds [start_o, start_o+1), the last
// one ending at the node's end.  cnt[p - lb] = the non-empty octants;
// cstart keeps the eight starts for the emit pass.  Launched with exactly
// 8 (le - lb) threads rounded up to whole blocks (every lane of a warp
// reaches the shuffles).
__global__ void count_children_kernel(int32_t lb, int32_t le, int level, int leaf_max,
                                      const unsigned long long *__restrict__ keys, const int64_t *__restrict__ nbeg,
                                      const int64_t *__restrict__ nend, int64_t *__restrict__ cstart,
                                      int32_t *__restrict__ cnt) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p = lb + (t >> 3);
  const int o = (int)(t & 7);
  const bool valid = p < le;
  int64_t b = 0, e = 0;
  if (valid) {
    b = nbeg[p];
    e = nend[p];
  }
  const bool open = valid && e - b > leaf_max && level < kMaxLevel;
  int64_t start = e;
  if (open) {  // first index of [b, e) whose digit is >= o
    int64_t lo = b, hi = e;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (digit_at(keys[mid], level) < o) lo = mid + 1;
      else hi = mid;
    }
    start = lo;
  }
  const int64_t next = __shfl_down_sync(0xffffffffu, start, 1);  // octant o + 1's start (same node for o < 7)
  const bool nonempty = open && (o == 7 ? e : next) > start;
  const unsigned g = threadIdx.x & 24u;  // this node's first lane in the warp
  const unsigned mask = (__ballot_sync(0xffffffffu, nonempty) >> g) & 0xffu;
  if (open) cstart[8 * (p - lb) + o] = start;
  if (valid && o == 0) cnt[p - lb] = __popc(mask);
}

// The children themselves: child k of node p (octants in order, empty ones
// skipped) is node base + excl[p - lb] + k; its range, level, parent,
// system and cube; the parent's first child and child count.  Same launch
// shape as count_children_kernel.
__global__ void emit_children_kernel(int32_t lb, int32_t le, int32_t base, int level,
                                     const int64_t *__restrict__ cstart, const int64_t *__restrict__ excl,
                                     int64_t *__restrict__ nbeg, int64_t *__restrict__ nend,
                                     int32_t *__restrict__ nlevel, int32_t *__restrict__ nparent,
                                     int32_t *__restrict__ nfirst, int32_t *__restrict__ nnchild,
                                     int32_t *__restrict__ nsysid, double *__restrict__ centre,
                                     double *__restrict__ half) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p = lb + (t >> 3);
  const int o = (int)(t & 7);
  const bool valid = p < le;
  int64_t c0 = 0, cn = 0;
  if (valid) {
    c0 = excl[p - lb];
    cn = excl[p - lb + 1] - c0;
  }
  int64_t so = 0, eo = 0;
  if (cn > 0) {
    so = cstart[8 * (p - lb) + o];
    eo = o == 7 ? nend[p] : cstart[8 * (p - lb) + o + 1];
  }
  const bool nonempty = cn > 0 && eo > so;
  const unsigned g = threadIdx.x & 24u;
  const unsigned mask = (__ballot_sync(0xffffffffu, nonempty) >> g) & 0xffu;
  if (nonempty) {
    const int32_t c = base + (int32_t)c0 + __popc(mask & ((1u << o) - 1u));
    nbeg[c] = so;
    nend[c] = eo;
    nlevel[c] = level + 1;
    nparent[c] = (int32_t)p;
    nfirst[c] = -1;
    nnchild[c] = 0;
    nsysid[c] = nsysid[p];
    const double h = half[p] * 0.5;
    centre[3 * c] = centre[3 * p] + (((o >> 2) & 1) ? h : -h);
    centre[3 * c + 1] = centre[3 * p + 1] + (((o >> 1) & 1) ? h : -h);
    centre[3 * c + 2] = centre[3 * p + 2] + ((o & 1) ? h : -h);
    half[c] = h;
  }
  if (o == 0 && cn > 0) {
    nfirst[p] = base + (int32_t)c0;
    nnchild[p] = (int32_t)cn;
  }
}

// ------------------------------------------------------------------ moments (Eq. 2)

constexpr int kMomentBatch = 8;  // leaves of up to this many particles load them all first

// Nodes grouped for the moments passes: a leaf of c <= kMomentBatch particles
// goes to bucket c - 1, a larger one (coincident particles at the deepest
// level) to bucket kMomentBatch; an internal node of level l with k children
// to bucket kLeafBuckets + 8 l + k - 1.  The leaf pass runs the leaf buckets,
// each internal level its eight buckets, so that the lanes of a warp sum the
// same number of particles or children: these passes are bound by the FP64
// pipe, and a warp of mixed nodes would issue every slot of its largest node
// (and idle the lanes of the other kind).
constexpr int kLeafBuckets = kMomentBatch + 1;
constexpr int kNodeBuckets = kLeafBuckets + 8 * kMaxLevel;
static_assert(kMomentBatch == 8, "the moments passes dispatch nodes of 1 to 8 particles or children");

__device__ __forceinline__ int node_bucket(int64_t cnt, int nc, int level) {
  if (nc == 0) return cnt >= 1 && cnt <= kMomentBatch ? (int)cnt - 1 : kMomentBatch;
  // an open node has a level below kMaxLevel and 1 to 8 children; the clamps
  // only keep the index inside the table
  level = level < 0 ? 0 : (level >= kMaxLevel ? kMaxLevel - 1 : level);
  nc = nc > 8 ? 8 : nc;
  return kLeafBuckets + 8 * level + nc - 1;
}

// hist[b] += nodes in bucket b (hist zeroed before)
__global__ void node_hist_kernel(int32_t nn, const int32_t *__restrict__ nnchild, const int64_t *__restrict__ nbeg,
                                 const int64_t *__restrict__ nend, const int32_t *__restrict__ nlevel,
                                 int *__restrict__ hist) {
  __shared__ int h[kNodeBuckets];
  for (int k = threadIdx.x; k < kNodeBuckets; k += blockDim.x) h[k] = 0;
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[node_bucket(nend[j] - nbeg[j], nnchild[j], nlevel[j])], 1);
  __syncthreads();
  for (int k = threadIdx.x; k < kNodeBuckets; k += blockDim.x)
    if (h[k] > 0) atomicAdd(&hist[k], h[k]);
}

// pre[b] = nodes in the buckets before b (pre[kNodeBuckets] = all); one thread
__global__ void bucket_scan_kernel(const int *__restrict__ hist, int *__restrict__ pre) {
  int acc = 0;
  for (int k = 0; k < kNodeBuckets; k++) {
    pre[k] = acc;
    acc += hist[k];
  }
  pre[kNodeBuckets] = acc;
}

// Every node's index into its bucket of order[] (cursor zeroed before).  A
// block places its share of each bucket with one atomic add per bucket; the
// order inside a bucket does not matter, since every node is summed on its own.
__global__ void node_fill_kernel(int32_t nn, const int32_t *__restrict__ nnchild, const int64_t *__restrict__ nbeg,
                                 const int64_t *__restrict__ nend, const int32_t *__restrict__ nlevel,
                                 const int *__restrict__ pre, int *__restrict__ cursor, int32_t *__restrict__ order) {
  __shared__ int h[kNodeBuckets], off[kNodeBuckets];
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nn; base += (int64_t)gridDim.x * blockDim.x) {
    for (int k = threadIdx.x; k < kNodeBuckets; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const int64_t j = base + threadIdx.x;
    int b = -1, r = 0;
    if (j < nn) {
      b = node_bucket(nend[j] - nbeg[j], nnchild[j], nlevel[j]);
      r = atomicAdd(&h[b], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kNodeBuckets; k += blockDim.x)
      off[k] = h[k] > 0 ? atomicAdd(&cursor[k], h[k]) : 0;
    __syncthreads();
    if (b >= 0) order[pre[b] + off[b] + r] = (int32_t)j;
  }
}

// Mass, centre of mass and Q of a leaf of CNT particles from [b, b + CNT):
// every position and mass requested before the sums start; the sums run in
// particle order, the host builder's expressions.
template <int CNT>
__device__ __forceinline__ void leaf_sums(int64_t b, const double *__restrict__ xs, const double *__restrict__ ms,
                                          double &M, double (&c)[3], double (&qq)[6]) {
  double px[CNT], py[CNT], pz[CNT], pm[CNT];
#pragma unroll
  for (int k = 0; k < CNT; k++) {
    px[k] = xs[3 * (b + k)];
    py[k] = xs[3 * (b + k) + 1];
    pz[k] = xs[3 * (b + k) + 2];
    pm[k] = ms[b + k];
  }
  double c0 = 0.0, c1 = 0.0, c2 = 0.0;
  M = 0.0;
#pragma unroll
  for (int k = 0; k < CNT; k++) {
    M += pm[k];
    c0 = fma(pm[k], px[k], c0);
    c1 = fma(pm[k], py[k], c1);
    c2 = fma(pm[k], pz[k], c2);
  }
  if (M > 0) {  // one FP64 division, the host builder's expressions
    const double inv = 1.0 / M;
    c0 *= inv;
    c1 *= inv;
    c2 *= inv;
  }
  // Q = 3 S - tr(S) I with S = sum m r r^T
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, s5 = 0.0;
#pragma unroll
  for (int k = 0; k < CNT; k++) {
    const double r0 = px[k] - c0, r1 = py[k] - c1, r2c = pz[k] - c2;
    const double m0 = pm[k] * r0, m1 = pm[k] * r1, m2 = pm[k] * r2c;
    s0 = fma(m0, r0, s0);
    s1 = fma(m0, r1, s1);
    s2 = fma(m0, r2c, s2);
    s3 = fma(m1, r1, s3);
    s4 = fma(m1, r2c, s4);
    s5 = fma(m2, r2c, s5);
  }
  const double tr = s0 + s3 + s5;
  c[0] = c0;
  c[1] = c1;
  c[2] = c2;
  qq[0] = 3 * s0 - tr;
  qq[1] = 3 * s1;
  qq[2] = 3 * s2;
  qq[3] = 3 * s3 - tr;
  qq[4] = 3 * s4;
  qq[5] = 3 * s5 - tr;
}

// The same for a leaf of any size (coincident particles at the deepest level
// can exceed kMomentBatch), reading its particles as it sums them.
__device__ __forceinline__ void leaf_sums_any(int64_t b, int64_t e, const double *__restrict__ xs,
                                              const double *__restrict__ ms, double &M, double (&c)[3],
                                              double (&qq)[6]) {
  double c0 = 0.0, c1 = 0.0, c2 = 0.0;
  M = 0.0;
  for (int64_t i = b; i < e; i++) {
    M += ms[i];
    c0 = fma(ms[i], xs[3 * i], c0);
    c1 = fma(ms[i], xs[3 * i + 1], c1);
    c2 = fma(ms[i], xs[3 * i + 2], c2);
  }
  if (M > 0) {
    const double inv = 1.0 / M;
    c0 *= inv;
    c1 *= inv;
    c2 *= inv;
  }
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, s5 = 0.0;
  for (int64_t i = b; i < e; i++) {
    const double r0 = xs[3 * i] - c0, r1 = xs[3 * i + 1] - c1, r2c = xs[3 * i + 2] - c2;
    const double mi = ms[i];
    const double m0 = mi * r0, m1 = mi * r1, m2 = mi * r2c;
    s0 = fma(m0, r0, s0);
    s1 = fma(m0, r1, s1);
    s2 = fma(m0, r2c, s2);
    s3 = fma(m1, r1, s3);
    s4 = fma(m1, r2c, s4);
    s5 = fma(m2, r2c, s5);
  }
  const double tr = s0 + s3 + s5;
  c[0] = c0;
  c[1] = c1;
  c[2] = c2;
  qq[0] = 3 * s0 - tr;
  qq[1] = 3 * s1;
  qq[2] = 3 * s2;
  qq[3] = 3 * s3 - tr;
  qq[4] = 3 * s4;
  qq[5] = 3 * s5 - tr;
}

// Moments (Eq. 2) of every leaf, bucket by bucket (order[] and pre[] from
// node_fill_kernel and bucket_scan_kernel).
__global__ void leaf_moments_kernel(const int *__restrict__ pre, const int32_t *__restrict__ order,
                                    const int64_t *__restrict__ nbeg, const int64_t *__restrict__ nend,
                                    const double *__restrict__ xs, const double *__restrict__ ms,
                                    double *__restrict__ com, double *__restrict__ mass, double *__restrict__ q,
                                    double *__restrict__ side, const double *__restrict__ half,
                                    int64_t *__restrict__ range) {
  const int64_t lo = pre[0], hi = pre[kLeafBuckets];
  for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = order[i];
    const int64_t b = nbeg[j], e = nend[j];
    double M, c[3], qq[6];
    switch (e - b) {
      case 1: leaf_sums<1>(b, xs, ms, M, c, qq); break;
      case 2: leaf_sums<2>(b, xs, ms, M, c, qq); break;
      case 3: leaf_sums<3>(b, xs, ms, M, c, qq); break;
      case 4: leaf_sums<4>(b, xs, ms, M, c, qq); break;
      case 5: leaf_sums<5>(b, xs, ms, M, c, qq); break;
      case 6: leaf_sums<6>(b, xs, ms, M, c, qq); break;
      case 7: leaf_sums<7>(b, xs, ms, M, c, qq); break;
      case 8: leaf_sums<8>(b, xs, ms, M, c, qq); break;
      default: leaf_sums_any(b, e, xs, ms, M, c, qq);
    }
    mass[j] = M;
    com[3 * j] = c[0];
    com[3 * j + 1] = c[1];
    com[3 * j + 2] = c[2];
#pragma unroll
    for (int k = 0; k < 6; k++) q[6 * j + k] = qq[k];
    side[j] = 2.0 * half[j];
    range[2 * j] = b;
    range[2 * j + 1] = e;
  }
}

// Mass, centre of mass and Q of an internal node from its NC children
// [f, f + NC): the children's masses and centres requested before the sums
// start, then their tensors; every sum runs in child order, the host
// builder's expressions (parallel-axis shift: Q = sum Q_c + 3 S - tr(S) I
// with S = sum m_c d d^T).
template <int NC>
__device__ __forceinline__ void internal_sums(int f, const double *__restrict__ mass, const double *__restrict__ com,
                                              const double *q, double &M, double (&c)[3], double (&qq)[6]) {
  double cm[NC], cx[NC], cy[NC], cz[NC];
#pragma unroll
  for (int k = 0; k < NC; k++) {
    cm[k] = mass[f + k];
    cx[k] = com[3 * (f + k)];
    cy[k] = com[3 * (f + k) + 1];
    cz[k] = com[3 * (f + k) + 2];
  }
  double c0 = 0.0, c1 = 0.0, c2 = 0.0;
  M = 0.0;
#pragma unroll
  for (int k = 0; k < NC; k++) {
    M += cm[k];
    c0 = fma(cm[k], cx[k], c0);
    c1 = fma(cm[k], cy[k], c1);
    c2 = fma(cm[k], cz[k], c2);
  }
  if (M > 0) {  // one FP64 division, the host builder's expressions
    const double inv = 1.0 / M;
    c0 *= inv;
    c1 *= inv;
    c2 *= inv;
  }
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, s5 = 0.0;
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const double r0 = cx[k] - c0, r1 = cy[k] - c1, r2c = cz[k] - c2;
    const double m0 = cm[k] * r0, m1 = cm[k] * r1, m2 = cm[k] * r2c;
    s0 = fma(m0, r0, s0);
    s1 = fma(m0, r1, s1);
    s2 = fma(m0, r2c, s2);
    s3 = fma(m1, r1, s3);
    s4 = fma(m1, r2c, s4);
    s5 = fma(m2, r2c, s5);
  }
  double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0, q4 = 0.0, q5 = 0.0;
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const double *qc = q + 6 * (f + k);
    q0 += qc[0];
    q1 += qc[1];
    q2 += qc[2];
    q3 += qc[3];
    q4 += qc[4];
    q5 += qc[5];
  }
  const double tr = s0 + s3 + s5;
  c[0] = c0;
  c[1] = c1;
  c[2] = c2;
  qq[0] = q0 + (3 * s0 - tr);
  qq[1] = q1 + 3 * s1;
  qq[2] = q2 + 3 * s2;
  qq[3] = q3 + (3 * s3 - tr);
  qq[4] = q4 + 3 * s4;
  qq[5] = q5 + (3 * s5 - tr);
}

// Moments (Eq. 2) of the internal nodes of one level from their children's
// (the level below, done before), bucket by bucket of child count.
__global__ void internal_moments_kernel(int level, const int *__restrict__ pre, const int32_t *__restrict__ order,
                                        const int64_t *__restrict__ nbeg, const int64_t *__restrict__ nend,
                                        const int32_t *__restrict__ nfirst, const int32_t *__restrict__ nnchild,
                                        double *__restrict__ com, double *__restrict__ mass, double *q,
                                        double *__restrict__ side, const double *__restrict__ half,
                                        int64_t *__restrict__ range) {
  const int64_t lo = pre[kLeafBuckets + 8 * level], hi = pre[kLeafBuckets + 8 * level + 8];
  for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = order[i];
    const int f = nfirst[j];
    double M, c[3], qq[6];
    switch (nnchild[j]) {
      case 1: internal_sums<1>(f, mass, com, q, M, c, qq); break;
      case 2: internal_sums<2>(f, mass, com, q, M, c, qq); break;
      case 3: internal_sums<3>(f, mass, com, q, M, c, qq); break;
      case 4: internal_sums<4>(f, mass, com, q, M, c, qq); break;
      case 5: internal_sums<5>(f, mass, com, q, M, c, qq); break;
      case 6: internal_sums<6>(f, mass, com, q, M, c, qq); break;
      case 7: internal_sums<7>(f, mass, com, q, M, c, qq); break;
      default: internal_sums<8>(f, mass, com, q, M, c, qq);
    }
    mass[j] = M;
    com[3 * j] = c[0];
    com[3 * j + 1] = c[1];
    com[3 * j + 2] = c[2];
#pragma unroll
    for (int k = 0; k < 6; k++) q[6 * j + k] = qq[k];
    side[j] = 2.0 * half[j];
    range[2 * j] = nbeg[j];
    range[2 * j + 1] = nend[j];
  }
}

// ------------------------------------------------------------------ groups

// group: (count <= n_crit or leaf) and (root or parent count > n_crit)
__global__ void group_mark_kernel(int32_t nn, int n_crit, const int64_t *__restrict__ nbeg,
                                  const int64_t *__restrict__ nend, const int32_t *__restrict__ nparent,
                                  const int32_t *__restrict__ nnchild, int32_t *__restrict__ gflag,
                                  int32_t *__restrict__ gnode_at) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cnt = nend[j] - nbeg[j];
    const int p = nparent[j];
    const bool mine = cnt <= n_crit || nnchild[j] == 0;
    const bool reached = p < 0 || nend[p] - nbeg[p] > n_crit;
    if (mine && reached) {
      gflag[nbeg[j]] = 1;
      gnode_at[nbeg[j]] = (int32_t)j;
    }
  }
}

__global__ void group_emit_kernel(int64_t n, const int32_t *__restrict__ gflag, const int64_t *__restrict__ gidx,
                                  const int32_t *__restrict__ gnode_at, int64_t *__restrict__ group_off,
                                  int32_t *__restrict__ group_node) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (gflag[i]) {
      group_off[gidx[i]] = i;
      group_node[gidx[i]] = gnode_at[i];
    }
  }
}

__global__ void group_last_kernel(int64_t G, int64_t n, int64_t *group_off) {
  if (threadIdx.x == 0 && blockIdx.x == 0) group_off[G] = n;
}

// ------------------------------------------------------------------ walk

// Compact per-node walk data: the FP32 geometry relative to the node's
// system root cube (centre o, side S: (x - o) / S, in [-1/2, 1/2]) for the
// walk's FP32 pre-test, and the topology in one int4, so that a visited node
// costs two aligned 32- and 16-byte loads.
__global__ void walk_data_kernel(int32_t nn, const int32_t *__restrict__ nsysid, const int32_t *__restrict__ sys_root,
                                 const double *__restrict__ centre, const double *__restrict__ side,
                                 const double *__restrict__ com, const int64_t *__restrict__ nbeg,
                                 const int64_t *__restrict__ nend, const int32_t *__restrict__ nfirst,
                                 const int32_t *__restrict__ nnchild, float4 *__restrict__ geom,
                                 int4 *__restrict__ topo) {
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x) {
    const int32_t r = sys_root[nsysid[k]];
    const double o0 = centre[3 * r], o1 = centre[3 * r + 1], o2 = centre[3 * r + 2], u = 1.0 / side[r];
    geom[2 * k] = make_float4(__double2float_rn((com[3 * k] - o0) * u), __double2float_rn((com[3 * k + 1] - o1) * u),
                              __double2float_rn((com[3 * k + 2] - o2) * u), __double2float_rn(side[k] * u));
    geom[2 * k + 1] = make_float4(__double2float_rn((centre[3 * k] - o0) * u),
                                  __double2float_rn((centre[3 * k + 1] - o1) * u),
                                  __double2float_rn((centre[3 * k + 2] - o2) * u), 0.0f);
    topo[k] = make_int4((int)nbeg[k], (int)nend[k], nfirst[k], nnchild[k]);
  }
}


// Group walk, one warp per group (a persistent grid; each warp owns a stack in
// global memory).  Per iteration the lanes take up to kWalkPop = 64 nodes off
// the top segment of the stack, two per lane (both nodes' records requested
// before either is tested: the walk waits on load latency, and two loads in
// flight per lane halve the waits of wide segments), and test them;
// accepted cells, opened leaves' particles and opened nodes' children are
// emitted / pushed through warp prefix sums, the lanes' first nodes before
// their second.  The children of one iteration form a new segment one level
// deeper, and pops never cross a segment boundary, so segment d holds nodes of
// level d only: at most 21 segments left behind with <= 448 entries each
// (512 children of 64 nodes, less the 64 popped) plus the top one (<= 512)
// ever sit on the stack.  The lists hold the same entries as a depth-first
// walk, in this walk's own fixed order.  walk_group walks one group;
// walk_single_kernel (one pass, groups taken from a counter, lists staged per
// warp and placed with one atomic add per list) and walk_warp_kernel (count,
// then fill at scanned offsets: the fallback) drive it.
//
// The opening test decides exactly as the FP64 test (node_opens64) does, but
// first tries it in FP32 on the root-cube coordinates (x - o) / S, all within
// [-1/2, 1/2]: there every FP32 quantity is within dl = 2^-20 + 2^-40 (|o| +
// S) / S of the exact (scaled) value -- a few FP32 roundings of 2^-24 each,
// plus the FP64 test's own rounding on absolute coordinates -- and a decision
// is taken in FP32 only when the compared quantities are apart by more than
// their error bounds.  Otherwise (ties and near-ties) the FP64 test decides.
// Scaling both sides of side^2 < theta^2 d^2 by 1/S^2 does not change it.
constexpr int kWalkPop = 64;  // nodes taken off the stack per walk iteration (two per lane)
constexpr int kWarpStack = kMaxLevel * (8 * kWalkPop - kWalkPop) + 8 * kWalkPop;
constexpr int kWalkBlock = 128;       // threads per block of the walk kernels
constexpr int kWalkBlocksPerSM = 9;   // the single-pass walk's register bound (56): 36 warps per SM

__device__ __forceinline__ int warp_excl(int v, int lane, int *total) {
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// The opening test in FP64 (Sec. 1 criterion against the group's box): true
// if node k must be opened.  The caller has already excluded nodes that hold
// particles of the group.
__device__ __forceinline__ bool node_opens64(int32_t k, double theta2, const double *__restrict__ centre,
                                             const double *__restrict__ side, const double *__restrict__ com,
                                             const double bmin[3], const double bmax[3]) {
  const double h = 0.5 * side[k];
  const double cc0 = centre[3 * k], cc1 = centre[3 * k + 1], cc2 = centre[3 * k + 2];
  bool meets = true;
  if (cc0 + h < bmin[0] || cc0 - h > bmax[0]) meets = false;
  if (cc1 + h < bmin[1] || cc1 - h > bmax[1]) meets = false;
  if (cc2 + h < bmin[2] || cc2 - h > bmax[2]) meets = false;
  if (meets) return true;
  double d2 = 0.0;
  const double x0 = com[3 * k], x1 = com[3 * k + 1], x2 = com[3 * k + 2];
  const double e0 = x0 < bmin[0] ? bmin[0] - x0 : (x0 > bmax[0] ? x0 - bmax[0] : 0.0);
  d2 += e0 * e0;
  const double e1 = x1 < bmin[1] ? bmin[1] - x1 : (x1 > bmax[1] ? x1 - bmax[1] : 0.0);
  d2 += e1 * e1;
  const double e2 = x2 < bmin[2] ? bmin[2] - x2 : (x2 > bmax[2] ? x2 - bmax[2] : 0.0);
  d2 += e2 * e2;
  return !(side[k] * side[k] < theta2 * d2);
}

// The same test in FP32 on root-relative data: 0 = accept as a cell,
// 1 = open, 2 = too close to call (the FP64 test decides).
__device__ __forceinline__ int node_opens32(float4 ga, float4 gb, float th2, float dl, float3 lo, float3 hi) {
  const float h = 0.5f * ga.w;
  float sep = fmaxf(lo.x - (gb.x + h), (gb.x - h) - hi.x);  // > 0: cube apart from the box on this axis
  sep = fmaxf(sep, fmaxf(lo.y - (gb.y + h), (gb.y - h) - hi.y));
  sep = fmaxf(sep, fmaxf(lo.z - (gb.z + h), (gb.z - h) - hi.z));
  if (sep < -dl) return 1;  // meets the box
  if (!(sep > dl)) return 2;
  const float e0 = fmaxf(fmaxf(lo.x - ga.x, ga.x - hi.x), 0.0f);
  const float e1 = fmaxf(fmaxf(lo.y - ga.y, ga.y - hi.y), 0.0f);
  const float e2 = fmaxf(fmaxf(lo.z - ga.z, ga.z - hi.z), 0.0f);
  const float A = ga.w * ga.w;
  const float B = th2 * (e0 * e0 + e1 * e1 + e2 * e2);
  const float tol = 0x1p-16f * (A + B) + th2 * dl * (2.0f * (e0 + e1 + e2) + 4.0f * dl);
  if (A < B - tol) return 0;
  if (A > B + tol) return 1;
  return 2;
}

// Finite doubles as signed 64-bit integers in the same order: a negative
// value's magnitude bits are flipped (-0 then sorts just below +0, which
// changes no comparison made with the result).  A group's box is reduced on
// these keys and turned back into the exact FP64 extremes.
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 ? b ^ 0x7fffffffffffffffLL : b;
}
__device__ __forceinline__ double key_value(long long k) {
  return __longlong_as_double(k < 0 ? k ^ 0x7fffffffffffffffLL : k);
}

// Where one group's list entries go: particle entries at p[0, cap_p), cell
// entries at c[0, cap_c); entries past a capacity (or with a null pointer)
// are counted but not written.
struct ListOut {
  int32_t *p, *c;
  int64_t cap_p, cap_c;
};

struct WalkTree {
  const int64_t *group_off;
  const int32_t *group_node, *nsysid, *sys_root;
  const double *xs;
  const float4 *geom;
  const int4 *topo;
  const double *centre, *side, *com;
};

// Walk group g with the calling warp; np, nc: its list sizes (warp-uniform).
// Returns false if the stack would overflow (not reachable, see above).
__device__ bool walk_group(const WalkTree &T, int64_t g, double theta2, float th2, int32_t *stack, ListOut out,
                           int64_t &np, int64_t &nc, double *box64) {
  const int lane = threadIdx.x & 31;
  const int32_t gb = (int32_t)T.group_off[g], ge = (int32_t)T.group_off[g + 1];
  // the group's box, reduced on ordered integer keys of the coordinates (the
  // integer pipes; the FP64 pipe is the scarcest one on this GPU)
  long long kmin[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, kmax[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  for (int64_t i = gb + lane; i < ge; i += 32)
    for (int d = 0; d < 3; d++) {
      const long long k = order_key(T.xs[3 * i + d]);
      kmin[d] = min(kmin[d], k);
      kmax[d] = max(kmax[d], k);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    for (int d = 0; d < 3; d++) {
      kmin[d] = min(kmin[d], __shfl_xor_sync(0xffffffffu, kmin[d], o));
      kmax[d] = max(kmax[d], __shfl_xor_sync(0xffffffffu, kmax[d], o));
    }
  const double bmin[3] = {key_value(kmin[0]), key_value(kmin[1]), key_value(kmin[2])};
  const double bmax[3] = {key_value(kmax[0]), key_value(kmax[1]), key_value(kmax[2])};
  const int32_t root = T.sys_root[T.nsysid[T.group_node[g]]];
  const double o0 = T.centre[3 * root], o1 = T.centre[3 * root + 1], o2 = T.centre[3 * root + 2], S = T.side[root];
  const double u = 1.0 / S, omax = fmax(fabs(o0), fmax(fabs(o1), fabs(o2)));
  const float dl = __double2float_ru(0x1p-20 + 0x1p-40 * (omax + S) * u);
  const float3 lo = make_float3(__double2float_rn((bmin[0] - o0) * u), __double2float_rn((bmin[1] - o1) * u),
                                __double2float_rn((bmin[2] - o2) * u));
  const float3 hi = make_float3(__double2float_rn((bmax[0] - o0) * u), __double2float_rn((bmax[1] - o1) * u),
                                __double2float_rn((bmax[2] - o2) * u));
  __syncwarp();  // the previous group's last stack and box reads are done
  if (lane == 0) {
    stack[0] = root;
    // the FP64 box, only needed by the (rare) FP64 decisions, waits in shared
    // memory instead of twelve registers
    for (int d = 0; d < 3; d++) {
      box64[d] = bmin[d];
      box64[3 + d] = bmax[d];
    }
  }
  __syncwarp();
  int sp = 1, depth = 0;
  int seg = 0;  // lane d: first stack slot of the segment at depth d
  np = 0;
  nc = 0;
  // kind of a popped node: 1 = accepted cell, 2 = opened leaf (its
  // particles), 3 = opened internal node (its children); 0 = no node
  const bool test = theta2 > 0.0;  // theta = 0 opens every node
  auto classify = [&](int32_t k, const int4 &tp, const float4 &ga, const float4 &gb2) -> int {
    bool open = true;
    if (test && !(tp.x < ge && tp.y > gb)) {
      const int dec = node_opens32(ga, gb2, th2, dl, lo, hi);
      open = dec == 2 ? node_opens64(k, theta2, T.centre, T.side, T.com, box64, box64 + 3) : dec == 1;
    }
    return !open ? 1 : (tp.w == 0 ? 2 : 3);
  };
  while (sp > 0) {
    const int base = __shfl_sync(0xffffffffu, seg, depth);
    if (sp == base) {  // this level's segment is used up: back to the one below
      depth--;
      continue;
    }
    const int take = sp - base < kWalkPop ? sp - base : kWalkPop;
    sp -= take;
    const bool haveA = lane < take, haveB = lane + 32 < take;
    const int32_t kA = haveA ? stack[sp + lane] : -1;
    const int32_t kB = haveB ? stack[sp + 32 + lane] : -1;
    __syncwarp();  // every lane has read its entries before the stack is written again
    int4 tpA = make_int4(0, 0, 0, 0), tpB = make_int4(0, 0, 0, 0);
    float4 gA0 = make_float4(0.f, 0.f, 0.f, 0.f), gA1 = gA0, gB0 = gA0, gB1 = gA0;
    if (haveA) {  // both nodes' records requested before either is tested
      tpA = T.topo[kA];
      gA0 = T.geom[2 * kA];
      gA1 = T.geom[2 * kA + 1];
    }
    if (haveB) {
      tpB = T.topo[kB];
      gB0 = T.geom[2 * kB];
      gB1 = T.geom[2 * kB + 1];
    }
    const int kindA = haveA ? classify(kA, tpA, gA0, gA1) : 0;
    const int kindB = haveB ? classify(kB, tpB, gB0, gB1) : 0;
    // accepted cells: the lanes' first nodes, then their second
    const unsigned lt = (1u << lane) - 1u;
    const unsigned cellsA = __ballot_sync(0xffffffffu, kindA == 1), cellsB = __ballot_sync(0xffffffffu, kindB == 1);
    if (out.c) {
      if (kindA == 1) {
        const int64_t at = nc + __popc(cellsA & lt);
        if (at < out.cap_c) out.c[at] = kA;
      }
      if (kindB == 1) {
        const int64_t at = nc + __popc(cellsA) + __popc(cellsB & lt);
        if (at < out.cap_c) out.c[at] = kB;
      }
    }
    nc += __popc(cellsA) + __popc(cellsB);
    // particles of opened leaves
    int ptA = 0, ptB = 0;
    const int pofsA = warp_excl(kindA == 2 ? tpA.y - tpA.x : 0, lane, &ptA);
    const int pofsB = warp_excl(kindB == 2 ? tpB.y - tpB.x : 0, lane, &ptB);
    if (out.p) {
      if (kindA == 2)
        for (int32_t i = tpA.x; i < tpA.y; i++) {
          const int64_t at = np + pofsA + (i - tpA.x);
          if (at < out.cap_p) out.p[at] = i;
        }
      if (kindB == 2)
        for (int32_t i = tpB.x; i < tpB.y; i++) {
          const int64_t at = np + ptA + pofsB + (i - tpB.x);
          if (at < out.cap_p) out.p[at] = i;
        }
    }
    np += ptA + ptB;
    // children of opened internal nodes: one new segment one level deeper
    int ctA = 0, ctB = 0;
    const int cofsA = warp_excl(kindA == 3 ? tpA.w : 0, lane, &ctA);
    const int cofsB = warp_excl(kindB == 3 ? tpB.w : 0, lane, &ctB);
    const int ctotal = ctA + ctB;
    if (ctotal > 0) {
      if (depth + 1 > kMaxLevel || sp + ctotal > kWarpStack) return false;  // not reachable for 21 levels
      if (kindA == 3)
        for (int c = 0; c < tpA.w; c++) stack[sp + cofsA + c] = tpA.z + c;
      if (kindB == 3)
        for (int c = 0; c < tpB.w; c++) stack[sp + ctA + cofsB + c] = tpB.z + c;
      depth++;
      if (lane == depth) seg = sp;
      sp += ctotal;
    }
    __syncwarp();
  }
  return true;
}

// Two-pass walk (the fallback): FILL == false counts each group's entries,
// FILL == true writes them at the scanned offsets.
template <bool FILL>
__global__ void walk_warp_kernel(int64_t G, double theta2, WalkTree T, int32_t *__restrict__ cnt_p,
                                 int32_t *__restrict__ cnt_c, const int64_t *__restrict__ plist_off,
                                 const int64_t *__restrict__ clist_off, int32_t *__restrict__ plist_idx,
                                 int32_t *__restrict__ clist_idx, int32_t *__restrict__ stacks, int *err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t *stack = stacks + warp * kWarpStack;
  __shared__ double s_box[kWalkBlock / 32][6];
  const float th2 = __double2float_rn(theta2);
  for (int64_t g = warp; g < G; g += nwarps) {
    ListOut out{nullptr, nullptr, 0, 0};
    if (FILL) out = ListOut{plist_idx + plist_off[g], clist_idx + clist_off[g], plist_off[g + 1] - plist_off[g],
                            clist_off[g + 1] - clist_off[g]};
    int64_t np = 0, nc = 0;
    if (!walk_group(T, g, theta2, th2, stack, out, np, nc, s_box[threadIdx.x >> 5])) {
      if (lane == 0) atomicOr(err, 1);
      return;
    }
    if (!FILL && lane == 0) {
      cnt_p[g] = (int32_t)(np < INT32_MAX ? np : INT32_MAX);
      cnt_c[g] = (int32_t)(nc < INT32_MAX ? nc : INT32_MAX);
    }
  }
}

// Single-pass walk: warps take groups from a shared counter, write each
// group's entries to their own staging area (capacities sp_cap, sc_cap),
// then reserve the group's place in the scratch lists with one atomic add per
// list and copy it there (groups land in completion order; gstart / cnt
// record where).  cursor[0]: next group, [1], [2]: particle / cell entries
// reserved so far (the exact totals, even when they exceed the scratch
// capacities).  err bit 0: stack, bit 1: a group longer than its staging
// area, bit 2: scratch too small.
__global__ void __launch_bounds__(kWalkBlock, kWalkBlocksPerSM) walk_single_kernel(int64_t G, double theta2, WalkTree T, int32_t *__restrict__ stage_p,
                                   int32_t *__restrict__ stage_c, int64_t sp_cap, int64_t sc_cap,
                                   int32_t *__restrict__ scratch_p, int32_t *__restrict__ scratch_c, int64_t cap_p,
                                   int64_t cap_c, unsigned long long *__restrict__ cursor,
                                   int64_t *__restrict__ gstart_p, int64_t *__restrict__ gstart_c,
                                   int64_t *__restrict__ gend_p, int64_t *__restrict__ gend_c,
                                   int32_t *__restrict__ cnt_p, int32_t *__restrict__ cnt_c,
                                   int32_t *__restrict__ stacks, int *err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int32_t *stack = stacks + warp * kWarpStack;
  __shared__ double s_box[kWalkBlock / 32][6];
  int32_t *mp = stage_p + warp * sp_cap, *mc = stage_c + warp * sc_cap;
  const float th2 = __double2float_rn(theta2);
  for (;;) {
    unsigned long long gg = 0;
    if (lane == 0) gg = atomicAdd(&cursor[0], 1ull);
    const int64_t g = (int64_t)__shfl_sync(0xffffffffu, gg, 0);
    if (g >= G) return;
    int64_t np = 0, nc = 0;
    if (!walk_group(T, g, theta2, th2, stack, ListOut{mp, mc, sp_cap, sc_cap}, np, nc, s_box[threadIdx.x >> 5])) {
      if (lane == 0) atomicOr(err, 1);
      return;
    }
    unsigned long long bp = 0, bc = 0;
    if (lane == 0) {
      bp = atomicAdd(&cursor[1], (unsigned long long)np);
      bc = atomicAdd(&cursor[2], (unsigned long long)nc);
    }
    bp = __shfl_sync(0xffffffffu, bp, 0);
    bc = __shfl_sync(0xffffffffu, bc, 0);
    __syncwarp();  // the staging writes of all lanes are visible to the copy
    if (np > sp_cap || nc > sc_cap) {
      if (lane == 0) atomicOr(err, 2);
    } else if ((int64_t)bp + np > cap_p || (int64_t)bc + nc > cap_c) {
      if (lane == 0) atomicOr(err, 4);
    } else {
      // streaming stores: the lists are read by the next kernel, not by this
      // one, so they should not push the tree's node records and the staging
      // areas out of L2
      for (int64_t i = lane; i < np; i += 32) __stcs(scratch_p + bp + i, mp[i]);
      for (int64_t i = lane; i < nc; i += 32) __stcs(scratch_c + bc + i, mc[i]);
    }
    if (lane == 0) {
      gstart_p[g] = (int64_t)bp;
      gstart_c[g] = (int64_t)bc;
      gend_p[g] = (int64_t)bp + np;
      gend_c[g] = (int64_t)bc + nc;
      cnt_p[g] = (int32_t)(np < INT32_MAX ? np : INT32_MAX);
      cnt_c[g] = (int32_t)(nc < INT32_MAX ? nc : INT32_MAX);
    }
    __syncwarp();  // the copy has read the staging area before the next group writes it
  }
}

// Scratch lists (groups in completion order) to CSR order: one warp per group.
__global__ void lists_to_csr_kernel(int64_t G, const int64_t *__restrict__ gstart, const int64_t *__restrict__ off,
                                    const int32_t *__restrict__ scratch, int32_t *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = warp; g < G; g += nwarps) {
    const int64_t s = gstart[g], o = off[g], n = off[g + 1] - off[g];
    for (int64_t i = lane; i < n; i += 32) out[o + i] = scratch[s + i];
  }
}

__global__ void unsort_kernel(int64_t n, int k, const int64_t *__restrict__ perm, const double *__restrict__ in,
                              double *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = perm[i];
    for (int c = 0; c < k; c++) out[o * k + c] = in[i * k + c];
  }
}

__global__ void roots_kernel(int64_t nsys, const int64_t *__restrict__ sys_off, const double *__restrict__ lo,
                             const double *__restrict__ width, const int32_t *__restrict__ root_of_sys,
                             int64_t *nbeg, int64_t *nend, int32_t *nlevel, int32_t *nparent, int32_t *nfirst,
                             int32_t *nnchild, int32_t *nsysid, double *centre, double *half) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nsys; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = root_of_sys[s];
    if (r < 0) continue;
    nbeg[r] = sys_off[s];
    nend[r] = sys_off[s + 1];
    nlevel[r] = 0;
    nparent[r] = -1;
    nfirst[r] = -1;
    nnchild[r] = 0;
    nsysid[r] = (int32_t)s;
    centre[3 * r] = lo[3 * s] + 0.5 * width[s];
    centre[3 * r + 1] = lo[3 * s + 1] + 0.5 * width[s];
    centre[3 * r + 2] = lo[3 * s + 2] + 0.5 * width[s];
    half[r] = 0.5 * width[s];
  }
}

int grid1(int64_t n) { return blocks_for(n, 256); }

}  // namespace

// ======================================================================= ABI

extern "C" {

qg_status qg_gtree_create(qg_gtree **out, int device) {
  if (!out) return QG_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return QG_ERR_ARG;
  qg_gtree *t = new (std::nothrow) qg_gtree;
  if (!t) return QG_ERR_NOMEM;
  t->device = device;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  bool ok = true;
  for (auto &e : t->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  if (ok) ok = t->err.reserve(1) == cudaSuccess;
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (!ok) {
    qg_gtree_destroy(t);
    return QG_ERR_CUDA;
  }
  *out = t;
  return QG_OK;
}

void qg_gtree_destroy(qg_gtree *t) {
  if (!t) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != t->device) cudaSetDevice(t->device);
  for (auto &e : t->ev)
    if (e) cudaEventDestroy(e);
  t->perm.release(); t->xs.release(); t->ms.release(); t->psys.release(); t->sys_off.release();
  t->bmin.release(); t->bmax.release(); t->lo.release(); t->scale.release();
  t->keys.release(); t->keys2.release(); t->vals.release(); t->vals2.release(); t->hist.release(); t->hoff.release();
  t->nbeg.release(); t->nend.release(); t->range.release(); t->nlevel.release(); t->nparent.release();
  t->nfirst.release(); t->nnchild.release(); t->nsysid.release(); t->cstart.release(); t->flag.release();
  t->excl.release(); t->centre.release(); t->half.release(); t->side.release(); t->com.release();
  t->mass.release(); t->q.release(); t->morder.release(); t->mbuckets.release(); t->sys_root.release(); t->gflag.release(); t->gnode_at.release();
  t->group_node.release(); t->cnt_p.release(); t->cnt_c.release(); t->gidx.release(); t->group_off.release();
  t->plist_off.release(); t->clist_off.release(); t->plist_idx.release(); t->clist_idx.release();
  for (auto &b : t->scan_tmp) b.release();
  t->stacks.release();
  for (DBuf<int32_t> *b : {&t->stage_p, &t->stage_c, &t->scratch_p, &t->scratch_c}) b->release();
  t->gstart_p.release();
  t->gstart_c.release();
  t->gend_p.release();
  t->gend_c.release();
  t->cursor.release();
  t->geom.release();
  t->topo.release();
  t->err.release();
  if (prev >= 0 && prev != t->device) cudaSetDevice(prev);
  delete t;
}

static qg_status build_impl(qg_gtree *t, int64_t n, const double *x, const double *m, int64_t nsys,
                            const int64_t *sys_off, int leaf_max, int n_crit, cudaStream_t s) {
  t->built = t->walked = false;
  t->n = n;
  t->nsys = nsys;
  t->leaf_max = leaf_max;
  t->n_crit = n_crit;
  t->h_sys_off.assign(sys_off, sys_off + nsys + 1);
  GT_CUDA(cudaEventRecord(t->ev[0], s));
  GT_CUDA(t->sys_off.reserve(nsys + 1));
  GT_CUDA(cudaMemcpyAsync(t->sys_off.p, sys_off, (nsys + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  GT_CUDA(t->psys.reserve(n));
  GT_CUDA(t->perm.reserve(n));
  GT_CUDA(t->xs.reserve(3 * n));
  GT_CUDA(t->ms.reserve(n));
  GT_CUDA(t->keys.reserve(n));
  GT_CUDA(t->vals.reserve(n));
  GT_CUDA(t->bmin.reserve(3 * nsys));
  GT_CUDA(t->bmax.reserve(3 * nsys));
  if (n > 0) {
    psys_kernel<<<grid1(n), 256, 0, s>>>(n, nsys, t->sys_off.p, t->psys.p);
    GT_CUDA(cudaGetLastError());
  }
  fill_ull_kernel<<<grid1(3 * nsys), 256, 0, s>>>(3 * nsys, t->bmin.p, ~0ull);
  fill_ull_kernel<<<grid1(3 * nsys), 256, 0, s>>>(3 * nsys, t->bmax.p, 0ull);
  GT_CUDA(cudaGetLastError());
  if (n > 0) {
    int sms = 0;
    GT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, t->device));
    const int64_t bw = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 32, (n + 1023) / 1024));
    const int64_t chunk = ((n + bw - 1) / bw + 31) / 32 * 32;
    bbox_kernel<<<(unsigned)((bw + 7) / 8), 256, 0, s>>>(n, chunk, x, t->psys.p, t->bmin.p, t->bmax.p);
    GT_CUDA(cudaGetLastError());
  }
  // per system cube on the host, the host builder's expressions exactly
  std::vector<unsigned long long> hmn(3 * nsys), hmx(3 * nsys);
  if (nsys > 0) {
    GT_CUDA(cudaMemcpyAsync(hmn.data(), t->bmin.p, 3 * nsys * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaMemcpyAsync(hmx.data(), t->bmax.p, 3 * nsys * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  }
  GT_CUDA(cudaStreamSynchronize(s));
  std::vector<double> hlo(3 * nsys), hwidth(nsys), hscale(nsys);
  std::vector<int32_t> hroot(nsys, -1);
  int32_t nroots = 0;
  for (int64_t q = 0; q < nsys; q++) {
    const int64_t b = sys_off[q], e = sys_off[q + 1];
    double mn[3], mx[3];
    for (int d = 0; d < 3; d++) {
      mn[d] = e > b ? unordered(hmn[3 * q + d]) : INFINITY;
      mx[d] = e > b ? unordered(hmx[3 * q + d]) : -INFINITY;
    }
    double w = 0.0;
    for (int d = 0; d < 3; d++) w = std::max(w, mx[d] - mn[d]);
    if (!(w > 0.0)) w = 1.0;
    w *= 1.0 + 1e-9;
    for (int d = 0; d < 3; d++) {
      const double c = 0.5 * (mn[d] + mx[d]);
      hlo[3 * q + d] = e > b ? c - 0.5 * w : 0.0;
    }
    hwidth[q] = w;
    hscale[q] = (double)(1u << kMaxLevel) / w;
    if (e > b) hroot[q] = nroots++;
  }
  GT_CUDA(t->lo.reserve(3 * nsys));
  GT_CUDA(t->scale.reserve(2 * nsys));
  GT_CUDA(t->sys_root.reserve(nsys));
  GT_CUDA(cudaMemcpyAsync(t->lo.p, hlo.data(), 3 * nsys * sizeof(double), cudaMemcpyHostToDevice, s));
  GT_CUDA(cudaMemcpyAsync(t->scale.p, hscale.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, s));
  GT_CUDA(cudaMemcpyAsync(t->scale.p + nsys, hwidth.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, s));
  GT_CUDA(cudaMemcpyAsync(t->sys_root.p, hroot.data(), nsys * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (n > 0) {
    keys_kernel<<<grid1(n), 256, 0, s>>>(n, x, t->psys.p, t->lo.p, t->scale.p, t->keys.p, t->vals.p);
    GT_CUDA(cudaGetLastError());
  }
  qg_status st = radix_sort(t, n, 64, s);  // Morton keys (bit 63 is always 0)
  if (st != QG_OK) return st;
  GT_CUDA(t->flag.reserve(n + 1));
  if (nsys > 1 && n > 0) {
    // stable second sort by system: (system, Morton) order, systems contiguous
    GT_CUDA(t->excl.reserve(n + 1));  // reused as scratch below
    DBuf<unsigned long long> morton;
    GT_CUDA(morton.reserve(n));
    DBuf<int32_t> morton_vals;
    GT_CUDA(morton_vals.reserve(n));
    GT_CUDA(cudaMemcpyAsync(morton_vals.p, t->vals.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    syskey_kernel<<<grid1(n), 256, 0, s>>>(n, t->vals.p, t->psys.p, t->keys.p, t->keys.p, t->vals.p, morton.p);
    GT_CUDA(cudaGetLastError());
    int bits = 8;
    while ((1ll << bits) < nsys) bits += 8;
    st = radix_sort(t, n, bits, s);
    if (st != QG_OK) {
      morton.release();
      morton_vals.release();
      return st;
    }
    gather_sorted_kernel<<<grid1(n), 256, 0, s>>>(n, morton_vals.p, t->vals.p, morton.p, t->keys.p, x, m,
                                                  t->perm.p, t->xs.p, t->ms.p, 1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    morton.release();
    morton_vals.release();
    if (e != cudaSuccess) return QG_ERR_CUDA;
  } else if (n > 0) {
    gather_sorted_kernel<<<grid1(n), 256, 0, s>>>(n, t->vals.p, nullptr, nullptr, nullptr, x, m, t->perm.p,
                                                  t->xs.p, t->ms.p, 0);
    GT_CUDA(cudaGetLastError());
  }
  // ---- nodes, level by level
  size_t cap = (size_t)std::max<int64_t>(1024, n / 2 + nroots + 16);
  auto reserve_nodes = [&](size_t need, size_t keep) -> qg_status {
    GT_CUDA(t->nbeg.grow(need, keep, s));
    GT_CUDA(t->nend.grow(need, keep, s));
    GT_CUDA(t->nlevel.grow(need, keep, s));
    GT_CUDA(t->nparent.grow(need, keep, s));
    GT_CUDA(t->nfirst.grow(need, keep, s));
    GT_CUDA(t->nnchild.grow(need, keep, s));
    GT_CUDA(t->nsysid.grow(need, keep, s));
    GT_CUDA(t->centre.grow(3 * need, 3 * keep, s));
    GT_CUDA(t->half.grow(need, keep, s));
    return QG_OK;
  };
  st = reserve_nodes(cap, 0);
  if (st != QG_OK) return st;
  roots_kernel<<<grid1(nsys), 256, 0, s>>>(nsys, t->sys_off.p, t->lo.p, t->scale.p + nsys, t->sys_root.p,
                                           t->nbeg.p, t->nend.p, t->nlevel.p, t->nparent.p, t->nfirst.p,
                                           t->nnchild.p, t->nsysid.p, t->centre.p, t->half.p);
  GT_CUDA(cudaGetLastError());
  // level by level: the open nodes of a level find their children by binary
  // search in their key ranges; children are numbered by parent, then octant
  t->level_begin.assign(1, 0);
  int64_t lb = 0, le = nroots;
  for (int level = 0; level < kMaxLevel && n > 0 && le > lb; level++) {
    t->level_begin.push_back(le);
    const int64_t L = le - lb;
    GT_CUDA(t->flag.reserve(L + 1));
    GT_CUDA(t->excl.reserve(L + 1));
    GT_CUDA(t->cstart.reserve(8 * L));
    const int64_t nb = (8 * L + 255) / 256;
    if (nb >= INT32_MAX) return QG_ERR_ARG;
    count_children_kernel<<<(unsigned)nb, 256, 0, s>>>((int32_t)lb, (int32_t)le, level, leaf_max, t->keys.p,
                                                       t->nbeg.p, t->nend.p, t->cstart.p, t->flag.p);
    GT_CUDA(cudaGetLastError());
    st = scan_excl(t, L, t->flag.p, t->excl.p, s);
    if (st != QG_OK) return st;
    int64_t C = 0;
    GT_CUDA(cudaMemcpyAsync(&C, t->excl.p + L, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    if (C == 0) break;
    if (le + C >= INT32_MAX) return QG_ERR_ARG;
    if ((size_t)(le + C) > t->nbeg.cap) {
      st = reserve_nodes((size_t)(le + C), (size_t)le);
      if (st != QG_OK) return st;
    }
    emit_children_kernel<<<(unsigned)nb, 256, 0, s>>>((int32_t)lb, (int32_t)le, (int32_t)le, level, t->cstart.p,
                                                      t->excl.p, t->nbeg.p, t->nend.p, t->nlevel.p, t->nparent.p,
                                                      t->nfirst.p, t->nnchild.p, t->nsysid.p, t->centre.p,
                                                      t->half.p);
    GT_CUDA(cudaGetLastError());
    lb = le;
    le += C;
  }
  const int64_t nn = le;
  t->nnodes = nn;
  if (t->level_begin.back() != nn) t->level_begin.push_back(nn);
  // ---- moments, deepest level first
  GT_CUDA(t->com.reserve(3 * nn));
  GT_CUDA(t->mass.reserve(nn));
  GT_CUDA(t->q.reserve(6 * nn));
  GT_CUDA(t->side.reserve(nn));
  GT_CUDA(t->range.reserve(2 * nn));
  // every leaf at once (their moments come from particles only), then the
  // internal nodes level by level, deepest first; the nodes grouped by
  // particle or child count first (node_bucket)
  GT_CUDA(t->morder.reserve(std::max<int64_t>(nn, 1)));
  GT_CUDA(t->mbuckets.reserve(3 * kNodeBuckets + 1));
  int *mhist = t->mbuckets.p, *mcursor = mhist + kNodeBuckets, *mpre = mcursor + kNodeBuckets;
  GT_CUDA(cudaMemsetAsync(mhist, 0, 2 * kNodeBuckets * sizeof(int), s));
  if (nn > 0) {
    node_hist_kernel<<<grid1(nn), 256, 0, s>>>((int32_t)nn, t->nnchild.p, t->nbeg.p, t->nend.p, t->nlevel.p, mhist);
    bucket_scan_kernel<<<1, 1, 0, s>>>(mhist, mpre);
    node_fill_kernel<<<grid1(nn), 256, 0, s>>>((int32_t)nn, t->nnchild.p, t->nbeg.p, t->nend.p, t->nlevel.p, mpre,
                                               mcursor, t->morder.p);
    leaf_moments_kernel<<<grid1(nn), 256, 0, s>>>(mpre, t->morder.p, t->nbeg.p, t->nend.p, t->xs.p, t->ms.p,
                                                  t->com.p, t->mass.p, t->q.p, t->side.p, t->half.p, t->range.p);
  }
  GT_CUDA(cudaGetLastError());
  for (int l = (int)t->level_begin.size() - 2; l >= 0; l--) {
    const int64_t a = t->level_begin[l], b = t->level_begin[l + 1];
    if (b > a && l + 2 < (int)t->level_begin.size() && l < kMaxLevel)  // the deepest level holds leaves only
      internal_moments_kernel<<<grid1(b - a), 256, 0, s>>>(l, mpre, t->morder.p, t->nbeg.p, t->nend.p, t->nfirst.p,
                                                           t->nnchild.p, t->com.p, t->mass.p, t->q.p, t->side.p,
                                                           t->half.p, t->range.p);
    GT_CUDA(cudaGetLastError());
  }
  // ---- compact walk data
  GT_CUDA(t->geom.reserve(2 * nn));
  GT_CUDA(t->topo.reserve(nn));
  if (nn > 0)
    walk_data_kernel<<<grid1(nn), 256, 0, s>>>((int32_t)nn, t->nsysid.p, t->sys_root.p, t->centre.p, t->side.p,
                                               t->com.p, t->nbeg.p, t->nend.p, t->nfirst.p, t->nnchild.p, t->geom.p,
                                               t->topo.p);
  GT_CUDA(cudaGetLastError());
  // ---- groups
  GT_CUDA(t->gflag.reserve(n + 1));
  GT_CUDA(t->gnode_at.reserve(n + 1));
  GT_CUDA(t->gidx.reserve(n + 1));
  if (n > 0) GT_CUDA(cudaMemsetAsync(t->gflag.p, 0, n * sizeof(int32_t), s));
  if (nn > 0)
    group_mark_kernel<<<grid1(nn), 256, 0, s>>>((int32_t)nn, n_crit, t->nbeg.p, t->nend.p, t->nparent.p,
                                                t->nnchild.p, t->gflag.p, t->gnode_at.p);
  GT_CUDA(cudaGetLastError());
  st = scan_excl(t, n, t->gflag.p, t->gidx.p, s);
  if (st != QG_OK) return st;
  int64_t G = 0;
  GT_CUDA(cudaMemcpyAsync(&G, t->gidx.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  t->G = G;
  GT_CUDA(t->group_off.reserve(G + 1));
  GT_CUDA(t->group_node.reserve(G + 1));
  if (n > 0)
    group_emit_kernel<<<grid1(n), 256, 0, s>>>(n, t->gflag.p, t->gidx.p, t->gnode_at.p, t->group_off.p,
                                               t->group_node.p);
  group_last_kernel<<<1, 1, 0, s>>>(G, n, t->group_off.p);
  GT_CUDA(cudaGetLastError());
  GT_CUDA(cudaEventRecord(t->ev[1], s));
  GT_CUDA(cudaStreamSynchronize(s));
  t->built = true;
  return QG_OK;
}

qg_status qg_gtree_build(qg_gtree *t, int64_t n, const double *x, const double *m, int64_t nsys,
                         const int64_t *sys_off, int leaf_max, int n_crit, void *stream) {
  if (!t || n < 0 || n >= INT32_MAX || nsys < 1 || !sys_off || leaf_max < 1 || n_crit < 1) return QG_ERR_ARG;
  if (n > 0 && (!x || !m)) return QG_ERR_ARG;
  if (sys_off[0] != 0 || sys_off[nsys] != n) return QG_ERR_ARG;
  for (int64_t q = 0; q < nsys; q++)
    if (sys_off[q + 1] < sys_off[q]) return QG_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != t->device) cudaSetDevice(t->device);
  const qg_status st = build_impl(t, n, x, m, nsys, sys_off, leaf_max, n_crit, (cudaStream_t)stream);
  if (prev >= 0 && prev != t->device) cudaSetDevice(prev);
  return st;
}

// Two-pass walk: count, scan, fill (the fallback of the single pass).
static qg_status walk_two_pass(qg_gtree *t, double theta2, const WalkTree &T, unsigned wg, int wb, cudaStream_t s,
                               int64_t tot[2]) {
  const int64_t G = t->G;
  if (G > 0) {
    walk_warp_kernel<false><<<wg, wb, 0, s>>>(G, theta2, T, t->cnt_p.p, t->cnt_c.p, nullptr, nullptr, nullptr,
                                              nullptr, t->stacks.p, t->err.p);
    GT_CUDA(cudaGetLastError());
  }
  qg_status st = scan_excl(t, G, t->cnt_p.p, t->plist_off.p, s);
  if (st != QG_OK) return st;
  st = scan_excl(t, G, t->cnt_c.p, t->clist_off.p, s);
  if (st != QG_OK) return st;
  int herr = 0;
  GT_CUDA(cudaMemcpyAsync(&tot[0], t->plist_off.p + G, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaMemcpyAsync(&tot[1], t->clist_off.p + G, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaMemcpyAsync(&herr, t->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  if (herr) return QG_ERR_STATE;
  GT_CUDA(t->plist_idx.reserve(tot[0]));
  GT_CUDA(t->clist_idx.reserve(tot[1]));
  if (G > 0) {
    walk_warp_kernel<true><<<wg, wb, 0, s>>>(G, theta2, T, t->cnt_p.p, t->cnt_c.p, t->plist_off.p, t->clist_off.p,
                                             t->plist_idx.p, t->clist_idx.p, t->stacks.p, t->err.p);
    GT_CUDA(cudaGetLastError());
  }
  t->lists_scratch = false;
  t->csr_ready = true;
  return QG_OK;
}

// The last walk's lists in group (CSR) order, made on the first request after
// a single-pass walk from its scratch lists (a scan of the list lengths and a
// copy), on stream s, which it synchronises so that the arrays are complete
// on return.
static qg_status ensure_csr(qg_gtree *t, cudaStream_t s) {
  if (!t->walked || t->lists_moved || t->csr_ready || !t->lists_scratch) return QG_OK;
  const int64_t G = t->G;
  qg_status st = scan_excl(t, G, t->cnt_p.p, t->plist_off.p, s);
  if (st != QG_OK) return st;
  st = scan_excl(t, G, t->cnt_c.p, t->clist_off.p, s);
  if (st != QG_OK) return st;
  GT_CUDA(t->plist_idx.reserve(t->np_list));
  GT_CUDA(t->clist_idx.reserve(t->nc_list));
  if (G > 0) {
    lists_to_csr_kernel<<<grid1(32 * G), 256, 0, s>>>(G, t->gstart_p.p, t->plist_off.p, t->scratch_p.p,
                                                       t->plist_idx.p);
    lists_to_csr_kernel<<<grid1(32 * G), 256, 0, s>>>(G, t->gstart_c.p, t->clist_off.p, t->scratch_c.p,
                                                       t->clist_idx.p);
    GT_CUDA(cudaGetLastError());
  }
  GT_CUDA(cudaStreamSynchronize(s));
  t->csr_ready = true;
  return QG_OK;
}

// Single-pass walk; *done = false when a group outgrew its staging area (the
// caller then walks in two passes; the staging areas are doubled for the
// next walk).
static qg_status walk_single_pass(qg_gtree *t, double theta2, const WalkTree &T, unsigned wg, int wb,
                                  cudaStream_t s, int64_t tot[2], bool *done) {
  const int64_t G = t->G, nw = (int64_t)wg * (wb / 32);
  *done = false;
  GT_CUDA(t->stage_p.reserve((size_t)(nw * t->stage_cap_p)));
  GT_CUDA(t->stage_c.reserve((size_t)(nw * t->stage_cap_c)));
  GT_CUDA(t->gstart_p.reserve(G));
  GT_CUDA(t->gstart_c.reserve(G));
  GT_CUDA(t->gend_p.reserve(G));
  GT_CUDA(t->gend_c.reserve(G));
  GT_CUDA(t->cursor.reserve(3));
  int64_t want_p = std::max<int64_t>(1024, 48 * t->n), want_c = std::max<int64_t>(1024, 24 * t->n);
  for (int attempt = 0; attempt < 2; attempt++) {
    GT_CUDA(t->scratch_p.reserve((size_t)std::max<int64_t>(want_p, (int64_t)t->scratch_p.cap)));
    GT_CUDA(t->scratch_c.reserve((size_t)std::max<int64_t>(want_c, (int64_t)t->scratch_c.cap)));
    GT_CUDA(cudaMemsetAsync(t->cursor.p, 0, 3 * sizeof(unsigned long long), s));
    GT_CUDA(cudaMemsetAsync(t->err.p, 0, sizeof(int), s));
    walk_single_kernel<<<wg, wb, 0, s>>>(G, theta2, T, t->stage_p.p, t->stage_c.p, t->stage_cap_p, t->stage_cap_c,
                                         t->scratch_p.p, t->scratch_c.p, (int64_t)t->scratch_p.cap,
                                         (int64_t)t->scratch_c.cap, t->cursor.p, t->gstart_p.p, t->gstart_c.p,
                                         t->gend_p.p, t->gend_c.p, t->cnt_p.p, t->cnt_c.p, t->stacks.p, t->err.p);
    GT_CUDA(cudaGetLastError());
    unsigned long long cur[3] = {0, 0, 0};
    int herr = 0;
    GT_CUDA(cudaMemcpyAsync(cur, t->cursor.p, sizeof(cur), cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaMemcpyAsync(&herr, t->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    if (herr & 1) return QG_ERR_STATE;
    if (herr & 2) {  // a list longer than a staging area
      t->stage_cap_p = std::min<int64_t>(t->stage_cap_p * 2, int64_t(1) << 24);
      t->stage_cap_c = std::min<int64_t>(t->stage_cap_c * 2, int64_t(1) << 24);
      return QG_OK;
    }
    tot[0] = (int64_t)cur[1];
    tot[1] = (int64_t)cur[2];
    if (herr & 4) {  // the scratch lists were too small: now the totals are known
      want_p = tot[0] + tot[0] / 8 + 1024;
      want_c = tot[1] + tot[1] / 8 + 1024;
      continue;
    }
    // the lists stay in the scratch arrays; CSR on request (ensure_csr)
    t->lists_scratch = true;
    t->csr_ready = false;
    *done = true;
    return QG_OK;
  }
  return QG_OK;  // not reached: the second attempt has room for the exact totals
}

static qg_status walk_impl(qg_gtree *t, double theta, cudaStream_t s) {
  t->walked = false;
  t->lists_scratch = t->csr_ready = false;
  t->walk_stream = s;
  const int64_t G = t->G;
  const double theta2 = theta > 0 ? theta * theta : 0.0;
  GT_CUDA(cudaEventRecord(t->ev[2], s));
  GT_CUDA(t->cnt_p.reserve(G + 1));
  GT_CUDA(t->cnt_c.reserve(G + 1));
  GT_CUDA(t->plist_off.reserve(G + 1));
  GT_CUDA(t->clist_off.reserve(G + 1));
  GT_CUDA(cudaMemsetAsync(t->err.p, 0, sizeof(int), s));
  // persistent warp grid: one stack (and staging area) per warp
  int sms = 0;
  GT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, t->device));
  const int wb = kWalkBlock;
  const int64_t warps = std::min<int64_t>(std::max<int64_t>(G, 1), (int64_t)sms * 4 * kWalkBlocksPerSM);
  const unsigned wg = (unsigned)((warps * 32 + wb - 1) / wb);
  GT_CUDA(t->stacks.reserve((size_t)wg * (wb / 32) * kWarpStack));
  const WalkTree T{t->group_off.p, t->group_node.p, t->nsysid.p, t->sys_root.p, t->xs.p, t->geom.p,
                   t->topo.p, t->centre.p, t->side.p, t->com.p};
  int64_t tot[2] = {0, 0};
  bool done = false;
  if (G > 0) {
    const qg_status st = walk_single_pass(t, theta2, T, wg, wb, s, tot, &done);
    if (st != QG_OK) return st;
  }
  if (!done) {
    GT_CUDA(cudaMemsetAsync(t->err.p, 0, sizeof(int), s));
    const qg_status st = walk_two_pass(t, theta2, T, wg, wb, s, tot);
    if (st != QG_OK) return st;
  }
  int herr = 0;
  GT_CUDA(cudaEventRecord(t->ev[3], s));
  GT_CUDA(cudaMemcpyAsync(&herr, t->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  if (herr) return QG_ERR_STATE;
  t->np_list = tot[0];
  t->nc_list = tot[1];
  t->walked = true;
  t->lists_moved = false;
  return QG_OK;
}

qg_status qg_gtree_walk(qg_gtree *t, double theta, void *stream) {
  if (!t || !std::isfinite(theta)) return QG_ERR_ARG;
  if (!t->built) return QG_ERR_STATE;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != t->device) cudaSetDevice(t->device);
  const qg_status st = walk_impl(t, theta, (cudaStream_t)stream);
  if (prev >= 0 && prev != t->device) cudaSetDevice(prev);
  return st;
}

qg_status qg_gtree_sizes(const qg_gtree *t, int64_t *n, int64_t *nnodes, int64_t *ngroups, int64_t *n_plist,
                         int64_t *n_clist) {
  if (!t) return QG_ERR_ARG;
  if (n) *n = t->n;
  if (nnodes) *nnodes = t->built ? t->nnodes : 0;
  if (ngroups) *ngroups = t->built ? t->G : 0;
  if (n_plist) *n_plist = t->walked ? t->np_list : 0;
  if (n_clist) *n_clist = t->walked ? t->nc_list : 0;
  return QG_OK;
}

qg_status qg_gtree_arrays(const qg_gtree *t, const int64_t **perm, const double **xs, const double **ms,
                          const int64_t **node_range, const int32_t **node_level, const double **cell_com,
                          const double **cell_m, const double **cell_q, const double **cell_side,
                          const int64_t **group_off, const int64_t **plist_off, const int32_t **plist_idx,
                          const int64_t **clist_off, const int32_t **clist_idx) {
  if (!t || !t->built) return QG_ERR_STATE;
  if (plist_off || plist_idx || clist_off || clist_idx) {
    // CSR lists on request (the tree's state, not its content, changes)
    qg_gtree *mt = const_cast<qg_gtree *>(t);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != t->device) cudaSetDevice(t->device);
    const qg_status st = ensure_csr(mt, t->walk_stream);
    if (prev >= 0 && prev != t->device) cudaSetDevice(prev);
    if (st != QG_OK) return st;
  }
  if (perm) *perm = t->perm.p;
  if (xs) *xs = t->xs.p;
  if (ms) *ms = t->ms.p;
  if (node_range) *node_range = t->range.p;
  if (node_level) *node_level = t->nlevel.p;
  if (cell_com) *cell_com = t->com.p;
  if (cell_m) *cell_m = t->mass.p;
  if (cell_q) *cell_q = t->q.p;
  if (cell_side) *cell_side = t->side.p;
  if (group_off) *group_off = t->group_off.p;
  const bool lists = t->walked && !t->lists_moved;
  if (plist_off) *plist_off = lists ? t->plist_off.p : nullptr;
  if (plist_idx) *plist_idx = lists ? t->plist_idx.p : nullptr;
  if (clist_off) *clist_off = lists ? t->clist_off.p : nullptr;
  if (clist_idx) *clist_idx = lists ? t->clist_idx.p : nullptr;
  return QG_OK;
}

qg_status qg_gtree_attach(qg_gtree *t, qg_ctx *ctx, double eps2_all, void *stream) {
  if (!t || !ctx) return QG_ERR_ARG;
  if (!t->built || !t->walked || t->lists_moved) return QG_ERR_STATE;
  {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != t->device) cudaSetDevice(t->device);
    const qg_status st = ensure_csr(t, (cudaStream_t)stream);
    if (prev >= 0 && prev != t->device) cudaSetDevice(prev);
    if (st != QG_OK) return st;
  }
  qg_status st = qg_set_sinks_dev(ctx, t->n, t->xs.p, nullptr, eps2_all, t->G, t->group_off.p, stream);
  if (st != QG_OK) return st;
  st = qg_set_sources_dev(ctx, t->n, t->xs.p, t->ms.p, t->plist_off.p, t->plist_idx.p, t->np_list, stream);
  if (st != QG_OK) return st;
  return qg_set_cells_dev(ctx, t->nnodes, t->com.p, t->mass.p, t->q.p, t->clist_off.p, t->clist_idx.p, t->nc_list,
                          stream);
}

qg_status qg_gtree_attach_move(qg_gtree *t, qg_ctx *ctx, double eps2_all, void *stream) {
  if (!t || !ctx) return QG_ERR_ARG;
  if (!t->built || !t->walked || t->lists_moved) return QG_ERR_STATE;
  qg::TreeLists L;
  L.device = t->device;
  L.n = t->n;
  L.G = t->G;
  L.nn = t->nnodes;
  L.np_list = t->np_list;
  L.nc_list = t->nc_list;
  L.xs = t->xs.p;
  L.ms = t->ms.p;
  L.com = t->com.p;
  L.mass = t->mass.p;
  L.q = t->q.p;
  L.goff = t->group_off.p;
  L.ranges = t->lists_scratch;  // the walk's own order: no CSR pass
  if (L.ranges) {
    L.poff = &t->gstart_p;
    L.pend = &t->gend_p;
    L.pidx = &t->scratch_p;
    L.coff = &t->gstart_c;
    L.cend = &t->gend_c;
    L.cidx = &t->scratch_c;
  } else {
    L.poff = &t->plist_off;
    L.coff = &t->clist_off;
    L.pidx = &t->plist_idx;
    L.cidx = &t->clist_idx;
  }
  t->lists_moved = true;  // from here on the list buffers may be the context's former ones
  return qg::attach_tree_lists(ctx, L, eps2_all, (cudaStream_t)stream);
}

qg_status qg_gtree_unsort(const qg_gtree *t, const double *in, double *out, int k, void *stream) {
  if (!t || !in || !out || k < 1) return QG_ERR_ARG;
  if (!t->built) return QG_ERR_STATE;
  if (t->n == 0) return QG_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != t->device) cudaSetDevice(t->device);
  unsort_kernel<<<grid1(t->n), 256, 0, (cudaStream_t)stream>>>(t->n, k, t->perm.p, in, out);
  const cudaError_t e = cudaGetLastError();
  if (prev >= 0 && prev != t->device) cudaSetDevice(prev);
  return e == cudaSuccess ? QG_OK : QG_ERR_CUDA;
}

qg_status qg_gtree_timing(const qg_gtree *t, float *build_ms, float *walk_ms) {
  if (!t) return QG_ERR_ARG;
  if (build_ms) {
    if (!t->built || cudaEventElapsedTime(build_ms, t->ev[0], t->ev[1]) != cudaSuccess) return QG_ERR_STATE;
  }
  if (walk_ms) {
    if (!t->walked || cudaEventElapsedTime(walk_ms, t->ev[2], t->ev[3]) != cudaSuccess) return QG_ERR_STATE;
  }
  return QG_OK;
}

}  // extern "C"
