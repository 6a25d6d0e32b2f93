// qg_sim.cu -- leapfrog time integration on the GPU (include/qg_sim.h): the
// kick-drift-kick step around the GPU tree build, group walk and force
// kernel, state resident in device memory in the caller's particle order.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "qg_devbuf.h"
#include "qg_gtree.h"
#include "qg_sim.h"
#include "qgrav.h"

namespace {

template <typename T>
using Buf = qg::DevBuf<T>;

constexpr int kThreads = 256;
constexpr int kRedBlocks = 592;  // fixed, so that the energy sums have a fixed order
constexpr int kRedVals = 5;      // K, W, p_x, p_y, p_z

unsigned blocks_for(int64_t work) {
  const int64_t b = (work + kThreads - 1) / kThreads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

// v += a h; x += v dt over the flat [3n] arrays (the first kick and the drift).
__global__ void kick_drift_kernel(int64_t n3, double *__restrict__ x, double *__restrict__ v,
                                  const double *__restrict__ a, double h, double dt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = v[i] + a[i] * h;
    v[i] = vi;
    x[i] += vi * dt;
  }
}

// Sorted position of every particle of the caller's order: rank[perm[i]] = i
// (perm is the tree's permutation of 0 .. n-1, n < 2^31).
__global__ void rank_kernel(int64_t n, const int64_t *__restrict__ perm, int32_t *__restrict__ rank) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rank[perm[i]] = (int32_t)i;
}

// Forces from the tree's sorted order back to the caller's order, and the
// second kick (h = 0: store only).  Threads run over the caller's order and
// gather through rank: the writes (and the read-modify-write of v) stay
// coalesced, and only the 4-byte ranks are scattered, by rank_kernel.
__global__ void unsort_kick_kernel(int64_t n, const int32_t *__restrict__ rank, const double *__restrict__ a_s,
                                   const double *__restrict__ phi_s, double *__restrict__ a,
                                   double *__restrict__ phi, double *__restrict__ v, double h, int kick) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rank[j];
    phi[j] = phi_s[i];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double ad = a_s[3 * i + d];
      a[3 * j + d] = ad;
      if (kick) v[3 * j + d] += ad * h;
    }
  }
}

__device__ __forceinline__ void block_sum(double (&val)[kRedVals], double *sh) {
  for (int k = 0; k < kRedVals; k++) sh[k * kThreads + threadIdx.x] = val[k];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < kRedVals; k++) sh[k * kThreads + threadIdx.x] += sh[k * kThreads + threadIdx.x + s];
    __syncthreads();
  }
  for (int k = 0; k < kRedVals; k++) val[k] = sh[k * kThreads];
}

// Per-particle softening in the tree's sorted order: eps2_s[i] = eps2[perm[i]].
__global__ void gather_eps2_kernel(int64_t n, const int64_t *__restrict__ perm, const float *__restrict__ eps2,
                                   float *__restrict__ eps2_s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    eps2_s[i] = eps2[perm[i]];
}

// Per block: K = 1/2 sum m v^2, W = 1/2 sum m (phi + m / eps), p = sum m v
// (eps per particle when eps2 is given, else 1/eps = inv_eps for all).
__global__ void energy_partial_kernel(int64_t n, const double *__restrict__ v, const double *__restrict__ m,
                                      const double *__restrict__ phi, double inv_eps, const float *__restrict__ eps2,
                                      double *__restrict__ part) {
  __shared__ double sh[kRedVals * kThreads];
  double val[kRedVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const double mi = m[i], v0 = v[3 * i], v1 = v[3 * i + 1], v2 = v[3 * i + 2];
    val[0] += 0.5 * mi * (v0 * v0 + v1 * v1 + v2 * v2);
    const double ie = eps2 ? (eps2[i] > 0.f ? 1.0 / sqrt((double)eps2[i]) : 0.0) : inv_eps;
    val[1] += 0.5 * mi * (phi[i] + mi * ie);
    val[2] += mi * v0;
    val[3] += mi * v1;
    val[4] += mi * v2;
  }
  block_sum(val, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < kRedVals; k++) part[k * kRedBlocks + blockIdx.x] = val[k];
}

__global__ void energy_final_kernel(const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double sh[kRedVals * kThreads];
  double val[kRedVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < kRedBlocks; b += kThreads)
    for (int k = 0; k < kRedVals; k++) val[k] += part[k * kRedBlocks + b];
  block_sum(val, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < kRedVals; k++) out[k] = val[k];
}

}  // namespace

struct qg_sim {
  int device = 0;
  qg_sim_params prm{};
  qg_options opt{};
  qg_gtree *tree = nullptr;
  qg_ctx *ctx = nullptr;
  int64_t n = 0;
  std::vector<int64_t> sys_off;
  Buf<double> x, v, m, a, phi, a_s, phi_s, red;
  Buf<int32_t> rank;        // sorted position of each particle of the caller's order
  Buf<float> eps2, eps2_s;  // per-particle softening (caller order, sorted order)
  bool per_particle_eps = false;
  bool has_state = false, tuned = false;
  int64_t tuned_entries = 0;  // list entries of the step the launch shape was last tuned on
  qg_options best{};          // the force launch in use outside trials
  // online re-tuning: launch shapes near `best`, one per force evaluation,
  // each timed by that evaluation's own force kernel
  std::vector<qg_options> trial;
  std::vector<float> trial_ms;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t stream = nullptr;  // used when the caller passes no stream
  qg_sim_times times{};
  // every call below runs on one stream, so the tree, force and integrator
  // steps are ordered without further synchronisation
  cudaStream_t use(void *caller) const { return caller ? (cudaStream_t)caller : stream; }
};

namespace {

#define SIM_CUDA(call)                                                      \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      return e_ == cudaErrorMemoryAllocation ? QG_ERR_NOMEM : QG_ERR_CUDA;  \
  } while (0)
#define SIM_OK(call)                        \
  do {                                      \
    const qg_status st_ = (call);           \
    if (st_ != QG_OK) return st_;           \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// The shapes an online trial runs: the current one and its neighbours --
// 2, 4 or 8 warps per CTA at the same list entries staged per warp and, at 4
// sinks per thread in an FP32 centred form, sinks per thread fixed or chosen
// per work item.  These are the dimensions along which the full tuner's
// choice moved as a collapsing sphere's lists grew.
std::vector<qg_options> neighbour_shapes(const qg_options &best) {
  std::vector<qg_options> out;
  const int W0 = best.warps_per_group > 0 ? best.warps_per_group : 4;
  const int T0 = best.tile_j > 0 ? best.tile_j : 256;
  const bool adapt = best.precision == QG_FP32_CENTRED && best.sinks_per_thread == 4 &&
                     best.arith != QG_ARITH_PAIRED;
  for (int W : {2, 4, 8}) {
    if (best.sinks_per_thread >= 8 && W > 4) continue;
    qg_options o = best;
    o.warps_per_group = W;
    o.tile_j = std::min(1024, std::max(128, T0 * W / W0 / 32 * 32));
    for (int a = 0; a < (adapt ? 2 : 1); a++) {
      o.sinks_adaptive = adapt ? a : best.sinks_adaptive;
      out.push_back(o);
    }
  }
  return out;
}

// forces(x) -> a, phi in the caller's order; with kick, also v += a h.
qg_status evaluate(qg_sim *s, cudaStream_t st, bool kick, double h) {
  SIM_OK(qg_gtree_build(s->tree, s->n, s->x.p, s->m.p, (int64_t)s->sys_off.size() - 1, s->sys_off.data(),
                        s->prm.leaf_max, s->prm.n_crit, st));
  SIM_OK(qg_gtree_walk(s->tree, s->prm.theta, st));
  if (s->per_particle_eps) {
    // the tree's arrays, with each sink's own softening in sorted order
    const int64_t *perm = nullptr, *goff = nullptr, *poff = nullptr, *coff = nullptr;
    const double *xs = nullptr, *ms = nullptr, *ccom = nullptr, *cm = nullptr, *cq = nullptr;
    const int32_t *pidx = nullptr, *cidx = nullptr;
    SIM_OK(qg_gtree_arrays(s->tree, &perm, &xs, &ms, nullptr, nullptr, &ccom, &cm, &cq, nullptr, &goff, &poff, &pidx,
                           &coff, &cidx));
    int64_t nn = 0, G = 0, np = 0, nc = 0;
    SIM_OK(qg_gtree_sizes(s->tree, nullptr, &nn, &G, &np, &nc));
    gather_eps2_kernel<<<blocks_for(s->n), kThreads, 0, st>>>(s->n, perm, s->eps2.p, s->eps2_s.p);
    SIM_CUDA(cudaGetLastError());
    SIM_OK(qg_set_sinks_dev(s->ctx, s->n, xs, s->eps2_s.p, 0.0, G, goff, st));
    SIM_OK(qg_set_sources_dev(s->ctx, s->n, xs, ms, poff, pidx, np, st));
    SIM_OK(qg_set_cells_dev(s->ctx, nn, ccom, cm, cq, coff, cidx, nc, st));
  } else {
    SIM_OK(qg_gtree_attach_move(s->tree, s->ctx, s->prm.eps2, st));
  }
  if (s->prm.autotune) {
    // a full qg_autotune at the first force evaluation; afterwards, whenever
    // the lists have grown or shrunk by more than a quarter since the last
    // tuning (a collapsing system changes its groups' lists several-fold),
    // an online trial: the next few evaluations each run one shape near the
    // current one, and the fastest of them is kept
    int64_t np = 0, nc = 0;
    SIM_OK(qg_gtree_sizes(s->tree, nullptr, nullptr, nullptr, &np, &nc));
    const int64_t entries = np + nc;
    if (!s->tuned) {
      SIM_OK(qg_autotune(s->ctx, st, 2, &s->best, nullptr));
      s->tuned = true;
      s->tuned_entries = entries;
      s->times.retunes++;
    } else if (s->trial.empty() && 4 * std::llabs(entries - s->tuned_entries) > s->tuned_entries) {
      s->trial = neighbour_shapes(s->best);
      s->trial_ms.clear();
      s->tuned_entries = entries;
      s->times.retunes++;
    }
    if (!s->trial.empty()) SIM_OK(qg_set_options(s->ctx, &s->trial[s->trial_ms.size()]));
  }
  qg_status run = qg_run(s->ctx, st);
  bool misfit = false;
  if (run == QG_ERR_ARG && !s->trial.empty()) {
    // the trial shape does not fit this device: run the current one instead
    misfit = true;
    SIM_OK(qg_set_options(s->ctx, &s->best));
    run = qg_run(s->ctx, st);
  }
  SIM_OK(run);
  SIM_OK(qg_get_forces_dev(s->ctx, s->a_s.p, s->phi_s.p, st));
  const int64_t *perm = nullptr;
  SIM_OK(qg_gtree_arrays(s->tree, &perm, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, nullptr, nullptr, nullptr, nullptr));
  SIM_CUDA(cudaEventRecord(s->ev[2], st));
  rank_kernel<<<blocks_for(s->n), kThreads, 0, st>>>(s->n, perm, s->rank.p);
  unsort_kick_kernel<<<blocks_for(s->n), kThreads, 0, st>>>(s->n, s->rank.p, s->a_s.p, s->phi_s.p, s->a.p, s->phi.p,
                                                            s->v.p, h, kick ? 1 : 0);
  SIM_CUDA(cudaGetLastError());
  SIM_CUDA(cudaEventRecord(s->ev[3], st));
  SIM_CUDA(cudaStreamSynchronize(st));
  float b = 0.f, w = 0.f, f = 0.f;
  SIM_OK(qg_gtree_timing(s->tree, &b, &w));
  SIM_OK(qg_last_timing(s->ctx, &f, nullptr));
  s->times.build_ms = b;
  s->times.walk_ms = w;
  s->times.force_ms = f;
  qg_stats stt{};
  SIM_OK(qg_get_stats(s->ctx, &stt));
  s->times.groups = stt.n_groups;
  s->times.n_plist = stt.n_plist;
  s->times.n_clist = stt.n_clist;
  s->times.i_pp = stt.i_pp;
  s->times.i_pc = stt.i_pc;
  s->times.sinks_per_thread = stt.sinks_per_thread;
  s->times.sinks_adaptive = stt.sinks_adaptive;
  s->times.warps_per_group = stt.warps_per_group;
  s->times.tile_j = stt.tile_j;
  s->times.form = stt.paired;
  // the times above are of the shape this evaluation ran; a trial that has
  // now run all its shapes keeps the fastest for the evaluations after it
  if (!s->trial.empty()) {
    s->trial_ms.push_back(misfit ? INFINITY : f);
    if (s->trial_ms.size() == s->trial.size()) {
      const size_t k = std::min_element(s->trial_ms.begin(), s->trial_ms.end()) - s->trial_ms.begin();
      if (std::isfinite(s->trial_ms[k])) s->best = s->trial[k];
      s->trial.clear();
      s->trial_ms.clear();
      SIM_OK(qg_set_options(s->ctx, &s->best));
    }
  }
  s->times.trial_left = (int32_t)(s->trial.size() - s->trial_ms.size());
  return QG_OK;
}

}  // namespace

extern "C" {

qg_status qg_sim_create(qg_sim **out, int device, const qg_sim_params *p, const qg_options *force_opt) {
  if (!out || !p) return QG_ERR_ARG;
  *out = nullptr;
  if (!(p->theta > 0.0) || !std::isfinite(p->theta) || !(p->eps2 >= 0.0) || !std::isfinite(p->eps2) ||
      p->n_crit < 1 || p->leaf_max < 1 || (p->expansion != QG_QUAD && p->expansion != QG_MONO))
    return QG_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return QG_ERR_ARG;
  DeviceGuard g(device);
  qg_sim *s = new (std::nothrow) qg_sim();
  if (!s) return QG_ERR_NOMEM;
  s->device = device;
  s->prm = *p;
  if (force_opt) s->opt = *force_opt;
  s->opt.expansion = p->expansion;
  qg_status st = qg_gtree_create(&s->tree, device);
  if (st == QG_OK) st = qg_create(&s->ctx, device, &s->opt);
  for (int k = 0; k < 4 && st == QG_OK; k++)
    if (cudaEventCreate(&s->ev[k]) != cudaSuccess) st = QG_ERR_CUDA;
  if (st == QG_OK && s->red.reserve(kRedVals * kRedBlocks + kRedVals) != cudaSuccess) st = QG_ERR_NOMEM;
  if (st == QG_OK && cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) st = QG_ERR_CUDA;
  if (st != QG_OK) {
    qg_sim_destroy(s);
    return st;
  }
  *out = s;
  return QG_OK;
}

void qg_sim_destroy(qg_sim *s) {
  if (!s) return;
  DeviceGuard g(s->device);
  if (s->ctx) qg_destroy(s->ctx);
  if (s->tree) qg_gtree_destroy(s->tree);
  for (auto &e : s->ev)
    if (e) cudaEventDestroy(e);
  if (s->stream) {
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  for (Buf<double> *b : {&s->x, &s->v, &s->m, &s->a, &s->phi, &s->a_s, &s->phi_s, &s->red}) b->release();
  s->eps2.release();
  s->eps2_s.release();
  s->rank.release();
  delete s;
}

qg_status qg_sim_set_state(qg_sim *s, int64_t n, const double *x, const double *v, const double *m,
                           const float *eps2, int64_t nsys, const int64_t *sys_off, void *stream) {
  if (!s || n < 1 || n >= INT32_MAX || !x || !v || !m || nsys < 1 || !sys_off) return QG_ERR_ARG;
  if (sys_off[0] != 0 || sys_off[nsys] != n) return QG_ERR_ARG;
  for (int64_t q = 0; q < nsys; q++)
    if (sys_off[q + 1] < sys_off[q]) return QG_ERR_ARG;
  if (eps2)
    for (int64_t i = 0; i < n; i++)
      if (!(eps2[i] >= 0.f) || !std::isfinite(eps2[i])) return QG_ERR_ARG;
  DeviceGuard g(s->device);
  cudaStream_t st = s->use(stream);
  s->has_state = false;
  s->n = n;
  s->sys_off.assign(sys_off, sys_off + nsys + 1);
  SIM_CUDA(s->x.reserve(3 * n));
  SIM_CUDA(s->v.reserve(3 * n));
  SIM_CUDA(s->a.reserve(3 * n));
  SIM_CUDA(s->a_s.reserve(3 * n));
  SIM_CUDA(s->m.reserve(n));
  SIM_CUDA(s->phi.reserve(n));
  SIM_CUDA(s->phi_s.reserve(n));
  SIM_CUDA(s->rank.reserve(n));
  SIM_CUDA(cudaMemcpyAsync(s->x.p, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  SIM_CUDA(cudaMemcpyAsync(s->v.p, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  SIM_CUDA(cudaMemcpyAsync(s->m.p, m, n * sizeof(double), cudaMemcpyHostToDevice, st));
  s->per_particle_eps = eps2 != nullptr;
  if (eps2) {
    SIM_CUDA(s->eps2.reserve(n));
    SIM_CUDA(s->eps2_s.reserve(n));
    SIM_CUDA(cudaMemcpyAsync(s->eps2.p, eps2, n * sizeof(float), cudaMemcpyHostToDevice, st));
  }
  SIM_CUDA(cudaStreamSynchronize(st));
  SIM_OK(evaluate(s, st, false, 0.0));
  s->has_state = true;
  return QG_OK;
}

qg_status qg_sim_step(qg_sim *s, double dt, int64_t nsteps, void *stream) {
  if (!s || !std::isfinite(dt) || nsteps < 0) return QG_ERR_ARG;
  if (!s->has_state) return QG_ERR_STATE;
  DeviceGuard g(s->device);
  cudaStream_t st = s->use(stream);
  for (int64_t k = 0; k < nsteps; k++) {
    const auto t0 = std::chrono::steady_clock::now();
    SIM_CUDA(cudaEventRecord(s->ev[0], st));
    kick_drift_kernel<<<blocks_for(3 * s->n), kThreads, 0, st>>>(3 * s->n, s->x.p, s->v.p, s->a.p, 0.5 * dt, dt);
    SIM_CUDA(cudaGetLastError());
    SIM_CUDA(cudaEventRecord(s->ev[1], st));
    const qg_status e = evaluate(s, st, true, 0.5 * dt);
    if (e != QG_OK) {
      s->has_state = false;  // positions have moved but the forces are not theirs
      return e;
    }
    float kd = 0.f, uk = 0.f;
    SIM_CUDA(cudaEventElapsedTime(&kd, s->ev[0], s->ev[1]));
    SIM_CUDA(cudaEventElapsedTime(&uk, s->ev[2], s->ev[3]));
    s->times.integrate_ms = kd + uk;
    s->times.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return QG_OK;
}

qg_status qg_sim_get_state(qg_sim *s, double *x, double *v, double *a, double *phi) {
  if (!s) return QG_ERR_ARG;
  if (!s->has_state) return QG_ERR_STATE;
  DeviceGuard g(s->device);
  SIM_CUDA(cudaStreamSynchronize(s->stream));
  const int64_t n = s->n;
  if (x) SIM_CUDA(cudaMemcpy(x, s->x.p, 3 * n * sizeof(double), cudaMemcpyDeviceToHost));
  if (v) SIM_CUDA(cudaMemcpy(v, s->v.p, 3 * n * sizeof(double), cudaMemcpyDeviceToHost));
  if (a) SIM_CUDA(cudaMemcpy(a, s->a.p, 3 * n * sizeof(double), cudaMemcpyDeviceToHost));
  if (phi) SIM_CUDA(cudaMemcpy(phi, s->phi.p, n * sizeof(double), cudaMemcpyDeviceToHost));
  return QG_OK;
}

qg_status qg_sim_state_dev(const qg_sim *s, const double **x, const double **v, const double **a, const double **phi,
                           const double **m) {
  if (!s) return QG_ERR_ARG;
  if (!s->has_state) return QG_ERR_STATE;
  if (x) *x = s->x.p;
  if (v) *v = s->v.p;
  if (a) *a = s->a.p;
  if (phi) *phi = s->phi.p;
  if (m) *m = s->m.p;
  return QG_OK;
}

qg_status qg_sim_energy(qg_sim *s, double *kinetic, double *potential, double *momentum, void *stream) {
  if (!s) return QG_ERR_ARG;
  if (!s->has_state) return QG_ERR_STATE;
  DeviceGuard g(s->device);
  cudaStream_t st = s->use(stream);
  const double inv_eps = s->prm.eps2 > 0.0 ? 1.0 / std::sqrt(s->prm.eps2) : 0.0;
  energy_partial_kernel<<<kRedBlocks, kThreads, 0, st>>>(s->n, s->v.p, s->m.p, s->phi.p, inv_eps,
                                                         s->per_particle_eps ? s->eps2.p : nullptr, s->red.p);
  energy_final_kernel<<<1, kThreads, 0, st>>>(s->red.p, s->red.p + kRedVals * kRedBlocks);
  SIM_CUDA(cudaGetLastError());
  double out[kRedVals];
  SIM_CUDA(cudaMemcpyAsync(out, s->red.p + kRedVals * kRedBlocks, sizeof(out), cudaMemcpyDeviceToHost, st));
  SIM_CUDA(cudaStreamSynchronize(st));
  if (kinetic) *kinetic = out[0];
  if (potential) *potential = out[1];
  if (momentum) std::memcpy(momentum, out + 2, 3 * sizeof(double));
  return QG_OK;
}

qg_status qg_sim_last_times(const qg_sim *s, qg_sim_times *out) {
  if (!s || !out) return QG_ERR_ARG;
  if (!s->has_state) return QG_ERR_STATE;
  *out = s->times;
  return QG_OK;
}

}  // extern "C"
