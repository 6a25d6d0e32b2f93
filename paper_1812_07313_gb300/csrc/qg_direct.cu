// qg_direct.cu -- direct O(N^2) summation on the GPU in FP64: the reference
// of the paper's relative force error (Eq. 8), used to measure the tree
// method's own error.  Not part of the timed force step.
#include <cuda_runtime.h>

#include <cstdint>

#include "qg_internal.h"
#include "qgrav.h"

namespace {

__global__ void round_f32_kernel(int64_t n, const double *__restrict__ in, float *__restrict__ out,
                                 float *__restrict__ out_hw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = qg::f64_to_f32_rn(in[i]);
    out_hw[i] = __double2float_rn(in[i]);
  }
}

constexpr int kThreads = 128;

__global__ void __launch_bounds__(kThreads) direct_kernel(int64_t nsink, const double *__restrict__ sx, double eps2,
                                                          int64_t nsrc, const double *__restrict__ x,
                                                          const double *__restrict__ m, double *__restrict__ a,
                                                          double *__restrict__ phi) {
  __shared__ double4_32a tile[kThreads];
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const bool live = i < nsink;
  const double xi = live ? sx[3 * i] : 0.0, yi = live ? sx[3 * i + 1] : 0.0, zi = live ? sx[3 * i + 2] : 0.0;
  double ax = 0.0, ay = 0.0, az = 0.0, pot = 0.0;
  for (int64_t base = 0; base < nsrc; base += kThreads) {
    const int cnt = (int)((nsrc - base) < kThreads ? (nsrc - base) : kThreads);
    __syncthreads();
    if (threadIdx.x < cnt) {
      const int64_t j = base + threadIdx.x;
      tile[threadIdx.x] = make_double4_32a(x[3 * j], x[3 * j + 1], x[3 * j + 2], m[j]);
    }
    __syncthreads();
    for (int t = 0; t < cnt; t++) {
      const double4_32a s = tile[t];
      const double dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
      const double r2 = dx * dx + dy * dy + dz * dz + eps2;
      if (r2 == 0.0) continue;
      const double ri = 1.0 / sqrt(r2);
      const double pm = s.w * ri;
      const double c = pm * ri * ri;
      pot += pm;
      ax += c * dx;
      ay += c * dy;
      az += c * dz;
    }
  }
  if (live) {
    a[3 * i] = ax;
    a[3 * i + 1] = ay;
    a[3 * i + 2] = az;
    phi[i] = -pot;
  }
}

}  // namespace

extern "C" qg_status qg_direct_dev(int device, int64_t nsink, const double *sink_x, double eps2, int64_t nsrc,
                                   const double *src_x, const double *src_m, double *a, double *phi,
                                   void *cuda_stream) {
  if (nsink < 0 || nsrc < 0 || !(eps2 >= 0.0)) return QG_ERR_ARG;
  if (nsink == 0) return QG_OK;
  if (!sink_x || !a || !phi || (nsrc > 0 && (!src_x || !src_m))) return QG_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return QG_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return QG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int64_t blocks = (nsink + kThreads - 1) / kThreads;
  qg_status st = QG_OK;
  if (blocks > 0x7fffffff) st = QG_ERR_ARG;
  if (st == QG_OK) {
    direct_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(nsink, sink_x, eps2, nsrc, src_x, src_m, a, phi);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = QG_ERR_CUDA;
  }
  if (prev != device) cudaSetDevice(prev);
  return st;
}

extern "C" qg_status qg_round_f32_host(int64_t n, const double *in, float *out) {
  if (n < 0 || (n > 0 && (!in || !out))) return QG_ERR_ARG;
  for (int64_t i = 0; i < n; i++) out[i] = qg::f64_to_f32_rn(in[i]);
  return QG_OK;
}

extern "C" qg_status qg_round_f32_dev(int64_t n, const double *in, float *out, float *out_hw, void *cuda_stream) {
  if (n < 0 || (n > 0 && (!in || !out || !out_hw))) return QG_ERR_ARG;
  if (n == 0) return QG_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int64_t blocks = (n + 255) / 256;
  round_f32_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(n, in, out, out_hw);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return QG_ERR_CUDA;
  return QG_OK;
}
