// qg_queue.cuh -- device work queue of one force step: every group gets a
// cost class (4 per octave of its FP32 work plus its list staging), and the
// groups are scattered into a queue in descending class, so that the
// persistent force kernel takes the most expensive groups first.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qg_internal.h"

namespace qg {

constexpr int kBuckets = 128;  // cost classes of the work queue (4 per octave)

__device__ __forceinline__ int cost_bucket(double cost) {
  if (!(cost > 1.0)) return 0;
  const int b = (int)(4.0 * log2(cost));
  return b < kBuckets ? b : kBuckets - 1;
}

// Work queue, pass 1: cost class of every group and a histogram of classes.
// cost = n_i * (13 n_p + c_cell n_c) FP32 ops + staging of the list entries.
// Group g's lists are [pbeg[g], pend[g]) and [cbeg[g], cend[g]) (CSR lists:
// pend = pbeg + 1).
static __global__ void queue_hist_kernel(int64_t G, const int64_t *__restrict__ goff, const int64_t *__restrict__ pbeg,
                                  const int64_t *__restrict__ pend, const int64_t *__restrict__ cbeg,
                                  const int64_t *__restrict__ cend, double cell_ops, unsigned char *bucket,
                                  int *hist) {
  __shared__ int h[kBuckets];
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) h[b] = 0;
  __syncthreads();
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
    const double ni = (double)(goff[g + 1] - goff[g]);
    const double np = (double)(pend[g] - pbeg[g]);
    const double nc = (double)(cend[g] - cbeg[g]);
    const double cost = ni * (13.0 * np + cell_ops * nc) + 64.0 * (np + nc) + 256.0;
    const int b = cost_bucket(cost);
    bucket[g] = (unsigned char)b;
    atomicAdd(&h[b], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
}

// Work queue, pass 1 when lists are split: the same cost classes for work
// items (a group's list, or one part of it: its entries [e0, e1) of the
// particle entries followed by the cell entries).
static __global__ void queue_hist_items_kernel(int64_t n, const Item *__restrict__ items,
                                               const int64_t *__restrict__ goff, const int64_t *__restrict__ pbeg,
                                               const int64_t *__restrict__ pend, double cell_ops,
                                               unsigned char *bucket, int *hist) {
  __shared__ int h[kBuckets];
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) h[b] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Item it = items[i];
    const double ni = (double)(goff[it.g + 1] - goff[it.g]);
    const int64_t npg = pend[it.g] - pbeg[it.g];
    const double np = (double)(min(it.e1, npg) - min(it.e0, npg));
    const double nc = (double)(max(it.e1 - npg, (int64_t)0) - max(it.e0 - npg, (int64_t)0));
    const double cost = ni * (13.0 * np + cell_ops * nc) + 64.0 * (np + nc) + 256.0;
    const int b = cost_bucket(cost);
    bucket[i] = (unsigned char)b;
    atomicAdd(&h[b], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
}

// Work queue, pass 2: groups (or work items) scattered in descending cost class.
static __global__ void queue_scatter_kernel(int64_t G, const unsigned char *__restrict__ bucket,
                                     const int *__restrict__ hist, int *cursor, int32_t *queue) {
  __shared__ int start[kBuckets];
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) {
    int s = 0;
    for (int c = b + 1; c < kBuckets; c++) s += hist[c];
    start[b] = s;
  }
  __syncthreads();
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
    const int b = bucket[g];
    const int pos = start[b] + atomicAdd(&cursor[b], 1);
    queue[pos] = (int32_t)g;
  }
}

}  // namespace qg
