// qg_devbuf.h -- an owning device array for the library's contexts: it only
// grows (reserve keeps the allocation while it is large enough and does not
// keep the contents when it grows; grow does) and is freed by release().
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>

namespace qg {

template <typename T>
struct DevBuf {
  T *p = nullptr;
  size_t cap = 0;  // elements
  cudaError_t reserve(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e == cudaSuccess) cap = n;
    return e;
  }
  // grow to at least n elements keeping the first `keep` (synchronises s)
  cudaError_t grow(size_t n, size_t keep, cudaStream_t s) {
    if (n <= cap && p) return cudaSuccess;
    const size_t c = std::max(n, cap * 2);
    T *q = nullptr;
    cudaError_t e = cudaMalloc(&q, c * sizeof(T));
    if (e != cudaSuccess) return e;
    if (keep && p) e = cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (p) cudaFree(p);
    p = q;
    cap = c;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace qg
