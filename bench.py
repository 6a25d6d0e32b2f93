#!/usr/bin/env python3
"""Benchmark of the GB300 monopole + quadrupole tree-force hot path.

One step = one qg_run over every sink group of the workload: device work-queue
build, then the persistent force kernel (FP64 group centring, list staging,
FP32 particle and cell loops, FP64 merges, outputs).  Inputs are resident in
HBM before the timed region; the L2 is flushed (a 256 MiB device write)
before every timed step and the flush is outside the per-step event pairs.

Printed (rank 0, one JSON line): interactions/s (particle-particle +
particle-cell), ms per step, the roofline of the force kernel (FP32 issue
bound), the FP64 oracle as a CPU baseline, an end-to-end number through the
C-ABI with host buffers, the clocks seen during the timed region, and the
quadrupole-vs-monopole force time at equal 99th-percentile force error.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "interactions/s; force time/step quad vs mono-only at equal 99th-pct force error"
UNIT = "interactions/s"
FLUSH_BYTES = 256 << 20
DESCR = {
    "cube_1m": "2^20 equal-mass particles uniform in the unit cube, eps=1/(20 N^(1/3)), leaf<=8, "
               "n_crit=256, quadrupole cells",
    "sphere_4k": "4096 particles uniform in the unit sphere, eps=1e-2, leaf<=8, n_crit=64",
    "plummer_4m": "2^22-particle Plummer sphere (a=1, r<=100), eps=1e-3, leaf<=8, n_crit=256",
    "batched_512": "512 independent Plummer/Hernquist systems, N log-uniform in [1024, 65536], eps=1e-2, "
                   "theta=0.5, one persistent launch (n_crit 64 unless --group-sizes tunes it)",
    "batched_64": "64 independent Plummer/Hernquist systems, N log-uniform in [1024, 65536], eps=1e-2, "
                  "n_crit=64 (the profiling-size case of batched_512)",
    "clumpy_16m": "2^24 particles in the unit cube, 70% in 2000 Plummer clumps + 30% uniform, eps=5e-5, "
                  "n_crit=256",
}
# The paper's own kernel speed, quoted as context (another machine, not a target): about 7e8
# particle-cell interactions/s at large N on one core of the CPU it names (Sec. 5.2).
PAPER_CONTEXT = {"cell_interactions_per_s": 7e8, "cpu": "Intel Xeon E5-2683 v4 (2.1 GHz), 1 core",
                 "code": "AVX2 FP32, approximate rsqrt, -ffast-math"}
# Workloads measured into the default line's 'configs' record, with their legs: group-size
# candidates, quadrupole thetas of the equal-error comparison, one launch per system vs batched.
CONFIGS = {"batched_512": {"group_sizes": [64, 128, 256], "ee_thetas": (), "batching": True},
           "clumpy_16m": {"group_sizes": None, "ee_thetas": (0.5,), "batching": False},
           "plummer_4m": {"group_sizes": None, "ee_thetas": (0.5,), "batching": False}}
# Algorithmic FP32 instructions per interaction (FMA = 1): quad 33, mono 13
OPS_QUAD, OPS_MONO = 33, 13
# FP32 forms of the force kernel (qg_stats.paired): name in the bench line and tag of the --launch flag
ARITH_NAMES = {0: "scalar f32", 1: "paired f32x2", 2: "entry-paired f32x2"}
ARITH_TAGS = {"scalar f32": "x1", "paired f32x2": "x2", "entry-paired f32x2": "xe"}
ARITH_CODES = {"scalar f32": 1, "paired f32x2": 2, "entry-paired f32x2": 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cube_1m")
    ap.add_argument("--theta", type=float, default=None)
    ap.add_argument("--no-equal-error", action="store_true", help="skip the monopole equal-error search")
    ap.add_argument("--equal-error-thetas", default="0.3,0.5,0.7",
                    help="quadrupole thetas of the equal-error comparison (comma separated)")
    ap.add_argument("--configs", default=None,
                    help="other workloads measured into the line's 'configs' record (comma separated, or 'none'); "
                         "default: %s for the default workload without --launch, else none" % ",".join(CONFIGS))
    ap.add_argument("--config-steps", type=int, default=20, help="timed steps of each 'configs' workload")
    ap.add_argument("--multi", choices=["shard", "replicas"], default="shard",
                    help="N > 1: shard = every rank evaluates its cost-balanced range of the workload's groups "
                         "(sources and cells replicated, no collective; total work fixed); replicas = every rank "
                         "evaluates the whole workload")
    ap.add_argument("--no-split-compare", action="store_true",
                    help="skip timing the step with long lists split into work items against the unsplit step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--batching-compare", action="store_true",
                    help="also time one launch per system against the single batched launch (multi-system sets)")
    ap.add_argument("--precision-compare", action="store_true",
                    help="also time the all-FP64 and the uncentred FP32 kernels and report their differences")
    ap.add_argument("--group-sizes", default=None,
                    help="candidate n_crit values (comma separated): time the step for each and use the fastest")
    ap.add_argument("--no-gpu-tree", action="store_true",
                    help="skip timing the tree build, moments, groups and walk on the GPU (whole step on the device)")
    ap.add_argument("--gpu-tree", action="store_true", help=argparse.SUPPRESS)  # the default; kept for old commands
    ap.add_argument("--launch", default=None,
                    help="R,W,T[,x1|x2|xe[,F]]: fixed sinks/thread (4a: chosen per item up to 4), warps/CTA, tile "
                         "(and scalar, sink-paired or entry-paired FP32, and entries between FP64 folds) instead of "
                         "the autotuner (profiling)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="qg_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = np.array([float(r[1]) for r in rows if r[1].replace(".", "").isdigit()])
        smax = float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if len(sm) else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ---------------------------------------------------------------- helpers

def build_case(name, theta):
    from paper_1812_07313_gb300 import tree as qtree
    from paper_1812_07313_gb300 import workloads
    wl = workloads.WORKLOADS[name]
    ps = wl.particles()
    t0 = time.perf_counter()
    tr = qtree.Tree(ps.x, ps.m, ps.sys_off, wl.leaf_max, wl.n_crit)
    t1 = time.perf_counter()
    L = tr.walk(wl.theta if theta is None else theta)
    t2 = time.perf_counter()
    eps2 = None
    eps2_all = float(ps.eps[0]) ** 2
    if ps.nsys > 1 and len(set(ps.eps.tolist())) > 1:
        eps2 = (ps.eps[tr.sink_sys] ** 2).astype(np.float32)
        eps2_all = 0.0
    return wl, ps, tr, L, eps2_all, eps2, {"construct_s": t1 - t0, "traverse_s": t2 - t1}


def load_ctx(ctx, tr, L, eps2_all, eps2):
    ctx.qg_set_sinks(tr.x, tr.group_off, eps2_all, eps2)
    ctx.qg_set_sources(tr.x, tr.m, L.plist_off, L.plist_idx)
    ctx.qg_set_cells(tr.cell_com, tr.cell_m, tr.cell_q, L.clist_off, L.clist_idx)


def timed_steps(torch, ctx, stream, flush, steps):
    """Per step: L2 flush (untimed), then events around qg_run; the force
    kernel's own time comes from the events inside the step's graph."""
    step_ms, force_ms = [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.add_(1)
            e0.record(stream)
            ctx.qg_run(stream.cuda_stream)
            e1.record(stream)
        _, f = ctx.qg_last_timing()  # synchronises the stream
        step_ms.append(e0.elapsed_time(e1))
        force_ms.append(f)
    return np.array(step_ms), np.array(force_ms)


def oracle_sample(tr, L, eps2_all, eps2, seconds, seed=0):
    """Groups in seeded random order until the oracle has about `seconds` of work."""
    import oracle
    rng = np.random.default_rng(seed)
    order = rng.permutation(tr.ngroups)
    ni = np.diff(tr.group_off)
    work = ni * (np.diff(L.plist_off) + np.diff(L.clist_off))
    # calibrate the oracle's rate on a few groups first
    probe = order[:8]
    t0 = time.perf_counter()
    oracle.expansion_forces(tr.group_off, tr.x, tr.x, tr.m, L.plist_off, L.plist_idx, tr.cell_com, tr.cell_m,
                            tr.cell_q, L.clist_off, L.clist_idx, eps2_all=eps2_all,
                            sink_eps2=None if eps2 is None else eps2.astype(np.float64), groups=probe)
    rate = max(work[probe].sum(), 1) / max(time.perf_counter() - t0, 1e-6)
    target = rate * seconds
    k = int(np.searchsorted(np.cumsum(work[order]), target)) + 1
    return order[:max(k, 1)], work


def run_oracle(tr, L, eps2_all, eps2, groups, threads=1):
    """Seconds the oracle takes on these groups (threads > 1: its groups split
    over that many host threads; the arithmetic of each group is unchanged)."""
    import oracle
    oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        oracle.expansion_forces(tr.group_off, tr.x, tr.x, tr.m, L.plist_off, L.plist_idx, tr.cell_com, tr.cell_m,
                                tr.cell_q, L.clist_off, L.clist_idx, eps2_all=eps2_all,
                                sink_eps2=None if eps2 is None else eps2.astype(np.float64), groups=groups)
        return time.perf_counter() - t0
    finally:
        oracle.set_threads(1)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    import subprocess
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The FP64 oracle as it stands, single-threaded on the host, on bounded
    samples of the same workload (rank 0 only)."""
    if rank != 0:
        return
    wl, ps, tr, L, eps2_all, eps2, _ = build_case(args.workload, args.theta)
    # about 150 s of oracle work in all, at most --cpu-seconds per step
    per_step = max(0.2, min(args.cpu_seconds, 150.0 / max(args.steps + args.warmup, 1)))
    total_int, total_t = 0, 0.0
    for s in range(args.warmup + args.steps):
        groups, work = oracle_sample(tr, L, eps2_all, eps2, per_step, seed=1000 + s)
        dt = run_oracle(tr, L, eps2_all, eps2, groups)
        if s >= args.warmup:
            total_int += int(work[groups].sum())
            total_t += dt
    value = total_int / total_t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "%s: %s" % (args.workload, DESCR.get(args.workload, "")),
                      "theta": L.theta, "sample": "seeded random groups, ~%.0f s of oracle work per step" % per_step},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "%d steps of seeded random group samples, %d interactions in total"
                                      % (args.steps, total_int)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- our arm

class GpuWorkload:
    """A workload's particles on the device and its tree, groups and lists
    built on the GPU (the same groups and lists as the host builder, in
    milliseconds): the legs below walk it at any theta and hand the lists to
    a force context."""

    def __init__(self, torch, name, n_crit=None):
        from paper_1812_07313_gb300 import gtree, workloads
        self.name = name
        self.wl = workloads.WORKLOADS[name]
        self.ps = self.wl.particles()
        if len(set(self.ps.eps.tolist())) != 1:
            raise ValueError("%s: one softening for every particle is needed here" % name)
        self.eps2_all = float(self.ps.eps[0]) ** 2
        self.dev = torch.cuda.current_device()
        self.x = torch.as_tensor(self.ps.x).cuda()
        self.m = torch.as_tensor(self.ps.m).cuda()
        self.tree = gtree.GpuTree(self.dev)
        self.n_crit = None
        self.theta = None
        if n_crit is not None:
            self.build(n_crit)

    def build(self, n_crit, stream=None):
        self.tree.build(self.x, self.m, self.ps.sys_off, self.wl.leaf_max, int(n_crit), stream)
        self.n_crit = int(n_crit)
        self.theta = None

    def load(self, ctx, theta, stream=None):
        """Walk at theta (unless the last walk was at it) and set ctx's inputs."""
        if self.theta != theta:
            self.tree.walk(theta, stream)
            self.theta = theta
        self.tree.attach(ctx, self.eps2_all, stream)

    def sorted_positions(self):
        return self.tree.host("xs"), self.tree.host("ms")

    def close(self):
        self.tree.close()


def time_context(torch, ctx, stream, flush, steps, warmup, local_rank=0, autotune=True):
    """Autotune (optional), warm up, then `steps` timed steps with the L2
    flushed before each and the clocks sampled: (step ms, force ms, clocks)."""
    if autotune:
        ctx.qg_autotune(stream.cuda_stream, reps=3)
    for _ in range(max(warmup, 1)):
        ctx.qg_run(stream.cuda_stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    step_ms, force_ms = timed_steps(torch, ctx, stream, flush, steps)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    return step_ms, force_ms, clocks


def roofline_of(i_pp, i_pc, force_ms, clocks, n_sm, stats, traffic=None):
    """FP32-issue roofline of the force kernel: algorithmic FP32
    lane-instructions (33 per particle-cell pair, 13 per particle pair, FMA =
    1) per second of force-kernel time, against SMs x 128 lanes x the median
    SM clock sampled during the timed region."""
    alg = OPS_QUAD * i_pc + OPS_MONO * i_pp
    achieved = alg / (force_ms * 1e-3) / 1e12
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = n_sm * 128 * sm_mhz * 1e6 / 1e12
    peak_max = n_sm * 128 * 2070e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s", "frac": achieved / peak,
            "traffic": traffic,
            "peak_basis": "FP32 lane-instructions/s = %d SMs x 128 x median SM clock %.0f MHz under load "
                          "(at the 2070 MHz maximum: %.1f Tinst/s, frac %.3f)"
                          % (n_sm, sm_mhz, peak_max, achieved / peak_max),
            "kernel": "force_kernel<float,R=%s,quad,%s>, %d threads, tile %d" % (
                ("1..%d per item" if stats.get("sinks_adaptive") else "%d") % stats["sinks_per_thread"],
                ARITH_NAMES[stats["paired"]], stats["block"], stats["tile_j"]),
            "force_kernel_ms": force_ms}


def equal_error(torch, qgrav, gw, thetas, flush, stream, steps, n_sample=4096):
    """For each quadrupole theta: time quadrupole steps and measure their p99
    of Eq. 8 against FP64 GPU direct summation on n_sample seeded sinks; find
    the largest monopole-only theta whose p99 is no larger (theta stepped down
    from the quadrupole's by factors of 0.8 until the p99 is met, then
    bisected between the last two), and time monopole-only steps there (both
    launch shapes autotuned).  Trees, groups and lists are built on the GPU
    (gw: GpuWorkload, already built)."""
    xs, ms = gw.sorted_positions()
    sys_off = np.asarray(gw.ps.sys_off)
    n = len(xs)
    rng = np.random.default_rng(12345)
    ns = min(n_sample, n)
    sample = np.sort(rng.choice(n, ns, replace=False))
    dev = torch.device("cuda")
    xs_d = torch.as_tensor(xs).to(dev)
    ms_d = torch.as_tensor(ms).to(dev)
    a_d = torch.empty((ns, 3), dtype=torch.float64, device=dev)
    p_d = torch.empty(ns, dtype=torch.float64, device=dev)
    # systems are independent (each sorted within itself): direct sums per system
    sys_of = np.searchsorted(sys_off, sample, side="right") - 1
    a_dir = np.empty((ns, 3))
    for s in np.unique(sys_of):
        sel = np.nonzero(sys_of == s)[0]
        b, e = int(sys_off[s]), int(sys_off[s + 1])
        qgrav.qg_direct_dev(xs_d[sample[sel]].contiguous(), xs_d[b:e], ms_d[b:e], gw.eps2_all, a_d[:len(sel)],
                            p_d[:len(sel)])
        a_dir[sel] = a_d[:len(sel)].cpu().numpy()

    def p99(a):
        e = np.linalg.norm(a[sample] - a_dir, axis=1) / np.linalg.norm(a_dir, axis=1)
        return float(np.percentile(e, 99))

    def timed(ctx, theta):
        gw.load(ctx, theta, stream.cuda_stream)
        ms, _, _ = time_context(torch, ctx, stream, flush, steps, 3)
        a, _ = ctx.qg_get_forces()
        st = ctx.qg_get_stats()
        return float(ms.mean()), a, int(st["i_pp"] + st["i_pc"])

    rows = []
    quad = qgrav.Context(gw.dev)
    mono = qgrav.Context(gw.dev, qgrav.Options(expansion=qgrav.QG_MONO))
    for theta_q in thetas:
        q_ms, a_q, q_int = timed(quad, theta_q)
        target = p99(a_q)
        cache = {}

        def mono_at(th):
            th = round(th, 5)
            if th not in cache:
                gw.load(mono, th, stream.cuda_stream)
                mono.qg_run(stream.cuda_stream)
                a, _ = mono.qg_get_forces()
                cache[th] = p99(a)
            return cache[th]

        # step down until the monopole code is at least as accurate, then bisect
        hi, lo = theta_q, theta_q
        while mono_at(lo) > target and lo > 0.02:
            hi, lo = lo, 0.8 * lo
        if mono_at(lo) <= target:
            for _ in range(6):
                mid = 0.5 * (lo + hi)
                if mono_at(mid) <= target:
                    lo = mid
                else:
                    hi = mid
        th_m = round(lo, 5)
        p_m = mono_at(th_m)
        m_ms, _, m_int = timed(mono, th_m)
        rows.append({"theta_quad": theta_q, "p99_quad": target, "quad_ms_per_step": q_ms, "quad_interactions": q_int,
                     "theta_mono": th_m, "p99_mono": p_m, "mono_ms_per_step": m_ms, "mono_interactions": m_int,
                     "quad_over_mono_time": q_ms / m_ms, "mono_meets_target": p_m <= target})
    quad.close()
    mono.close()
    return {"error_sample": "FP64 GPU direct summation on %d seeded sinks" % ns,
            "search": "monopole theta stepped down by 0.8 from the quadrupole theta until its p99 is no larger, "
                      "then 6 bisection steps; GPU-built trees and lists", "rows": rows}


def split_compare(torch, qgrav, ctx, chosen, stream, flush, steps=10):
    """The step at the chosen launch shape with long lists split into work
    items automatically (qg_options.split_j = -1) against the unsplit step,
    with the largest work item's share of one CTA's average load (work =
    the queue's cost measure; a share near 1 or above leaves the end of the
    persistent launch to a few CTAs)."""
    import dataclasses
    st = ctx.qg_get_stats()
    res = {}
    for name, sj in (("auto", -1), ("off", 0)):  # unsplit last: ctx keeps that step's results
        ctx.set_options(dataclasses.replace(chosen, split_j=sj))
        ms, fms, _ = time_context(torch, ctx, stream, flush, steps, 3, autotune=False)
        s = ctx.qg_get_stats()
        res[name] = {"ms_per_step": float(ms.mean()), "force_ms": float(fms.mean()), "items": int(s["n_items"]),
                     "split_groups": int(s["n_split"])}
    ctx.set_options(chosen)
    res["auto_over_off_time"] = res["auto"]["ms_per_step"] / res["off"]["ms_per_step"]
    res["grid"] = int(st["grid"])
    return res


def item_share(tr, L, grid, cell_ops=33.0):
    """Largest group's work (the queue's cost measure) over one CTA's average
    share of the step's work."""
    ni = np.diff(tr.group_off).astype(np.float64)
    npl, ncl = np.diff(L.plist_off).astype(np.float64), np.diff(L.clist_off).astype(np.float64)
    cost = ni * (13.0 * npl + cell_ops * ncl) + 64.0 * (npl + ncl) + 256.0
    return float(cost.max() / (cost.sum() / max(grid, 1)))


def config_record(torch, qgrav, name, steps, warmup, stream, flush, n_sm, local_rank=0, group_sizes=None,
                  ee_thetas=(), batching=False):
    """One workload measured as the main line is (GPU-built tree and lists,
    autotuned launch shape, L2 flushed before each timed step, clocks sampled
    during the timed region), with optional group-size tuning, quadrupole vs
    monopole-only at equal p99 error and the one-launch-per-system
    comparison."""
    from paper_1812_07313_gb300 import tuning
    t0 = time.perf_counter()
    gw = GpuWorkload(torch, name)
    theta = gw.wl.theta
    rec = {"workload": "%s: %s" % (name, DESCR.get(name, "")), "theta": theta}
    if group_sizes:
        best, table = tuning.tune_group_size_gpu(gw.tree, gw.x, gw.m, gw.ps.sys_off, gw.wl.leaf_max, theta,
                                                 group_sizes, gw.eps2_all, device=gw.dev, steps=3,
                                                 stream=stream.cuda_stream)
        gw.n_crit, gw.theta = best.n_crit, theta
        rec["group_size"] = {"n_crit": best.n_crit, "tuned": True,
                             "chosen_by": "shortest whole GPU step: tree build + walk + force step",
                             "candidates": [{"n_crit": r.n_crit, "groups": r.groups, "interactions": r.interactions,
                                             "step_ms": r.step_ms, "force_ms": r.force_ms,
                                             "tree_build_walk_ms": r.tree_ms,
                                             "whole_step_ms": r.step_ms + r.tree_ms, "launch": r.launch}
                                            for r in table]}
    else:
        gw.build(gw.wl.n_crit)
        rec["group_size"] = {"n_crit": gw.wl.n_crit, "tuned": False}
    ctx = qgrav.Context(gw.dev)
    gw.load(ctx, theta, stream.cuda_stream)
    t_tune = time.perf_counter()
    ctx.qg_autotune(stream.cuda_stream, reps=3)
    t_tune = time.perf_counter() - t_tune
    step_ms, force_ms, clocks = time_context(torch, ctx, stream, flush, steps, warmup, local_rank, autotune=False)
    st = ctx.qg_get_stats()
    i_pp, i_pc = int(st["i_pp"]), int(st["i_pc"])
    rec.update({"value": (i_pp + i_pc) / (float(step_ms.mean()) * 1e-3), "unit": UNIT,
                "ms_per_step": float(step_ms.mean()), "steps": steps,
                "interactions": {"i_pp": i_pp, "i_pc": i_pc}, "groups": int(st["n_groups"]),
                "launch": {"sinks_per_thread": st["sinks_per_thread"], "warps_per_group": st["warps_per_group"],
                           "tile_j": st["tile_j"], "grid": st["grid"], "block": st["block"],
                           "arith": ARITH_NAMES[st["paired"]], "sinks_adaptive": st["sinks_adaptive"],
                           "autotune_s": t_tune},
                "roofline": roofline_of(i_pp, i_pc, float(force_ms.mean()), clocks, n_sm, st),
                "clocks": clocks})
    if batching:
        rec["batching"] = batching_compare(torch, qgrav, gw, stream, flush, float(step_ms.mean()))
    ctx.close()
    if ee_thetas:
        rec["equal_error"] = equal_error(torch, qgrav, gw, list(ee_thetas), flush, stream, max(5, steps // 2),
                                         n_sample=2048 if gw.ps.x.shape[0] > (1 << 23) else 4096)
    gw.close()
    rec["wall_s"] = time.perf_counter() - t0
    return rec


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1812_07313_gb300 import qgrav

    torch.cuda.set_device(local_rank)
    qgrav.lib()
    wl, ps, tr, L, eps2_all, eps2, host_times = build_case(args.workload, args.theta)
    group_size = {"n_crit": wl.n_crit, "tuned": False}
    if args.group_sizes:
        from paper_1812_07313_gb300 import tuning
        cands = [int(v) for v in args.group_sizes.split(",")]
        best, table, (tr, L) = tuning.tune_group_size(
            ps.x, ps.m, ps.sys_off, wl.leaf_max, L.theta, cands, eps2_all=eps2_all,
            eps2_of_system=None if eps2 is None else ps.eps ** 2, device=torch.cuda.current_device())
        if eps2 is not None:
            eps2 = (ps.eps[tr.sink_sys] ** 2).astype(np.float32)
        group_size = {"n_crit": best.n_crit, "tuned": True,
                      "candidates": [{"n_crit": r.n_crit, "groups": r.groups, "interactions": r.interactions,
                                      "step_ms": r.step_ms, "force_ms": r.force_ms, "launch": r.launch}
                                     for r in table]}
    theta = L.theta
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    ctx = qgrav.Context(dev)
    sharded = world > 1 and args.multi == "shard"
    if sharded:
        # this rank's cost-balanced range of groups; sources and cells replicated
        from paper_1812_07313_gb300 import shard
        sh = shard.shards(tr.group_off, L.plist_off, L.plist_idx, L.clist_off, L.clist_idx, world)[rank]
        ctx.qg_set_sinks(tr.x[sh.s0:sh.s1], sh.group_off, eps2_all,
                         None if eps2 is None else eps2[sh.s0:sh.s1])
        ctx.qg_set_sources(tr.x, tr.m, sh.plist_off, sh.plist_idx)
        ctx.qg_set_cells(tr.cell_com, tr.cell_m, tr.cell_q, sh.clist_off, sh.clist_idx)
    else:
        load_ctx(ctx, tr, L, eps2_all, eps2)
    st = ctx.qg_get_stats()
    i_pp, i_pc = int(st["i_pp"]), int(st["i_pc"])
    inter = i_pp + i_pc
    stream = torch.cuda.Stream()
    flush = torch.zeros(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    t_tune = time.perf_counter()
    if args.launch:
        parts = args.launch.split(",")
        adapt = parts[0].endswith("a")  # e.g. 4a: sinks per thread chosen per item, up to 4
        R, W, T = int(parts[0].rstrip("a")), int(parts[1]), int(parts[2])
        arith = {"x1": qgrav.QG_ARITH_SCALAR, "x2": qgrav.QG_ARITH_PAIRED,
                 "xe": qgrav.QG_ARITH_ENTRY_PAIRED}[parts[3]] if len(parts) > 3 else 0
        flush_j = int(parts[4]) if len(parts) > 4 else 0
        ctx.set_options(qgrav.Options(sinks_per_thread=R, warps_per_group=W, tile_j=T, arith=arith,
                                      flush_j=flush_j, sinks_adaptive=int(adapt)))
    else:
        ctx.qg_autotune(stream.cuda_stream, reps=3)
    t_tune = time.perf_counter() - t_tune
    st = ctx.qg_get_stats()
    launch = {"sinks_per_thread": st["sinks_per_thread"], "warps_per_group": st["warps_per_group"],
              "tile_j": st["tile_j"], "flush_j": st["flush_j"], "grid": st["grid"], "block": st["block"],
              "autotune_s": t_tune, "autotuned": not args.launch}
    for _ in range(max(args.warmup, 0)):
        ctx.qg_run(stream.cuda_stream)
    torch.cuda.synchronize()
    a_quad, _ = ctx.qg_get_forces()
    st = ctx.qg_get_stats()
    launch.update({"sinks_per_thread": st["sinks_per_thread"], "warps_per_group": st["warps_per_group"],
                   "tile_j": st["tile_j"], "grid": st["grid"], "block": st["block"],
                   "arith": ARITH_NAMES[st["paired"]], "sinks_adaptive": st["sinks_adaptive"]})

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    t_wall0 = time.perf_counter()
    step_ms, force_ms = timed_steps(torch, ctx, stream, flush, args.steps)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms, value = aggregate_ranks(float(step_ms.sum()), args.steps, inter, world,
                                      dist if world > 1 else None, "cuda", summed=sharded)

    # roofline of the force kernel: FP32 issue bound (lane instructions, FMA = 1)
    roofline = roofline_of(i_pp, i_pc, float(force_ms.mean()), clocks, n_sm, st,
                           _recorded_traffic(args.workload, launch))

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "%s: %s" % (args.workload, DESCR.get(args.workload, "")),
                      "theta": theta, "expansion": "quad",
                      "precision": "fp32 pair arithmetic, offsets centred from float-pair records, "
                                   "float-float folds and stream merges, fp64 outputs",
                      "interactions": {"i_pp": i_pp, "i_pc": i_pc}, "groups": tr.ngroups,
                      "group_size": group_size, "launch": launch,
                      "l2": "flushed before every timed step (256 MiB device write, outside the step events)",
                      "parallelism": ("%d cost-balanced shards of the groups, sources and cells replicated, "
                                      "no collective" % world) if sharded else
                                     ("%d replicas" % world if world > 1 else "single GPU"),
                      "host_tree_s": host_times},
           "paper_context": PAPER_CONTEXT,
           "roofline": roofline, "gpu_launches": 3 * args.steps, "clocks": clocks,
           "wall_s_timed_loop": t_wall}

    gw = None
    solo = world == 1  # the legs below measure one GPU's step; at N > 1 only the main line and e2e run
    if solo and eps2 is None and ((not args.no_equal_error) or (args.batching_compare and ps.nsys > 1)):
        gw = GpuWorkload(torch, args.workload, n_crit=tr_n_crit(tr, wl))
    if solo and not args.no_equal_error and eps2 is None:
        thetas = [float(v) for v in args.equal_error_thetas.split(",")]
        ee_steps = max(5, args.steps // 2)
        out["equal_error"] = equal_error(torch, qgrav, gw, thetas, flush, stream, ee_steps)
    if solo and args.batching_compare and ps.nsys > 1 and gw is not None:
        gw.theta = None
        gw.tree.walk(theta)
        gw.theta = theta
        out["batching"] = batching_compare(torch, qgrav, gw, stream, flush, float(np.mean(step_ms)))
    if gw is not None:
        gw.close()
    # the chosen launch shape, for the legs below
    chosen = qgrav.Options(sinks_per_thread=launch["sinks_per_thread"], warps_per_group=launch["warps_per_group"],
                           tile_j=launch["tile_j"],
                           arith=ARITH_CODES[launch.get("arith", "scalar f32")],
                           sinks_adaptive=launch.get("sinks_adaptive", 0))
    if solo and not args.no_split_compare and not args.launch:
        sc = {args.workload: dict(split_compare(torch, qgrav, ctx, chosen, stream, flush),
                                  max_item_over_cta_share=item_share(tr, L, launch["grid"]))}
        if args.workload != "sphere_4k":
            # a small set: fewer groups than the GPU has CTA slots
            _, _, tr_s, L_s, e2_s, _, _ = build_case("sphere_4k", None)
            c_s = qgrav.Context(dev)
            load_ctx(c_s, tr_s, L_s, e2_s, None)
            best_s, _ = c_s.qg_autotune(stream.cuda_stream, reps=3)
            sc["sphere_4k"] = dict(split_compare(torch, qgrav, c_s, best_s, stream, flush),
                                   max_item_over_cta_share=item_share(tr_s, L_s, c_s.qg_get_stats()["grid"]),
                                   groups=int(tr_s.ngroups))
            c_s.close()
        out["split"] = sc
    if solo and not args.no_gpu_tree:
        out["gpu_tree"] = gpu_tree_step(torch, qgrav, ps, wl, tr, L, eps2_all, eps2, stream, chosen)
    if solo and args.precision_compare:
        out["precision"] = precision_compare(torch, qgrav, ctx, tr, L, eps2_all, eps2, stream, flush)

    # end to end through the C-ABI with host buffers (pinned), every step
    out["e2e"] = e2e(torch, qgrav, tr, L, eps2_all, eps2, inter, world, chosen,
                     shard_part=sh if sharded else None, dist=dist if world > 1 else None)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        groups, work = oracle_sample(tr, L, eps2_all, eps2, args.cpu_seconds)
        dt = run_oracle(tr, L, eps2_all, eps2, groups)
        out["cpu_baseline"] = {"value": float(work[groups].sum() / dt), "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": "%d of %d groups in seeded random order, %d interactions, %.1f s"
                                         % (len(groups), tr.ngroups, int(work[groups].sum()), dt)}
        # the same sample with the oracle's groups split over every host core
        ncores = os.cpu_count() or 1
        dtp = run_oracle(tr, L, eps2_all, eps2, groups, threads=ncores)
        out["cpu_baseline_all_cores"] = {"value": float(work[groups].sum() / dtp), "unit": UNIT, "cores": ncores,
                                         "kind": "oracle, groups split over host threads (OpenMP)",
                                         "cpu": cpu_model(), "sample": "the cpu_baseline sample, %.2f s" % dtp}
    ctx.close()

    # the other workloads, each measured as the main line is
    configs = args.configs
    if configs is None:
        configs = "none" if (args.launch or args.workload != "cube_1m") else ",".join(CONFIGS)
    if solo and configs != "none":
        out["configs"] = {}
        for name in configs.split(","):
            leg = CONFIGS.get(name, {"group_sizes": None, "ee_thetas": (), "batching": False})
            out["configs"][name] = config_record(torch, qgrav, name, args.config_steps, max(args.warmup, 3), stream,
                                                 flush, n_sm, local_rank, leg["group_sizes"], leg["ee_thetas"],
                                                 leg["batching"])
    if rank == 0:
        print(json.dumps(out))


def aggregate_ranks(total_ms, steps, units_per_step, world, dist=None, device="cpu", summed=False):
    """Whole-job throughput: the job took the slowest rank's time (max over
    ranks).  Replicas: every rank processed `units_per_step` per step;
    summed (shards): the ranks' own units per step are added up."""
    units = world * units_per_step
    if world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        if summed:
            u = torch.tensor([float(units_per_step)], dtype=torch.float64, device=device)
            dist.all_reduce(u, op=dist.ReduceOp.SUM)
            units = float(u.item())
    return total_ms, steps * units / (total_ms * 1e-3)


def batching_compare(torch, qgrav, gw, stream, flush, batched_ms, steps=5):
    """The same step as one qg_run per system (each system its own context,
    its own queue build and force launch, launched back to back on one
    stream) against the single batched launch.  Each system's sinks, lists
    and cells are cut out of the GPU-built tree (gw: GpuWorkload, built and
    walked): its nodes gathered and the cell-list entries renumbered."""
    t = gw.tree
    xs, ms = gw.sorted_positions()
    goff_all, po_all, pi_all = t.host("group_off"), t.host("plist_off"), t.host("plist_idx")
    co_all, ci_all = t.host("clist_off"), t.host("clist_idx")
    com, cm, cq, nr = t.host("cell_com"), t.host("cell_m"), t.host("cell_q"), t.host("node_range")
    sys_off = np.asarray(gw.ps.sys_off)
    sys_of_group = np.searchsorted(sys_off, goff_all[:-1], side="right") - 1
    node_sys = np.searchsorted(sys_off, nr[:, 0], side="right") - 1
    ctxs = []
    for s in range(len(sys_off) - 1):
        b, e = int(sys_off[s]), int(sys_off[s + 1])
        gsel = np.nonzero(sys_of_group == s)[0]
        if len(gsel) == 0:
            continue
        g0, g1 = int(gsel[0]), int(gsel[-1]) + 1
        nodes = np.nonzero(node_sys == s)[0]
        renum = np.full(len(nr), -1, dtype=np.int64)
        renum[nodes] = np.arange(len(nodes))
        goff = goff_all[g0:g1 + 1] - goff_all[g0]
        po = po_all[g0:g1 + 1] - po_all[g0]
        co = co_all[g0:g1 + 1] - co_all[g0]
        pi = (pi_all[po_all[g0]:po_all[g1]] - b).astype(np.int32)
        ci = renum[ci_all[co_all[g0]:co_all[g1]]].astype(np.int32)
        c = qgrav.Context(gw.dev)
        c.qg_set_sinks(xs[b:e], goff, gw.eps2_all)
        c.qg_set_sources(xs[b:e], ms[b:e], po, pi)
        c.qg_set_cells(com[nodes], cm[nodes], cq[nodes], co, ci)
        ctxs.append(c)
    # one launch shape for all systems: the batched step's autotuned shape would
    # favour the batched side, so each system keeps the default shape
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for c in ctxs:
        c.qg_run(stream.cuda_stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.add_(1)
            e0.record(stream)
            for c in ctxs:
                c.qg_run(stream.cuda_stream)
            e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    for c in ctxs:
        c.close()
    per_sys = float(np.mean(times))
    return {"systems": len(ctxs), "batched_ms_per_step": batched_ms, "per_system_ms_per_step": per_sys,
            "speedup": per_sys / batched_ms, "per_system_launches": 3 * len(ctxs),
            "note": "per-system contexts at the default launch shape, graphs replayed back to back on one stream"}


def gpu_tree_step(torch, qgrav, ps, wl, tr, L, eps2_all, eps2, stream, options, steps=5):
    """The whole step on the GPU: tree build with moments and groups, walk,
    attach, force kernel at the launch shape of the step above (the GPU
    builds the same groups and lists as the host); device times of each
    part."""
    from paper_1812_07313_gb300 import gtree
    x = torch.as_tensor(ps.x).cuda()
    m = torch.as_tensor(ps.m).cuda()
    t = gtree.GpuTree(torch.cuda.current_device())
    ctx = qgrav.Context(torch.cuda.current_device(), options)
    build, walk, force = [], [], []
    same = None
    for k in range(steps + 1):
        t.build(x, m, ps.sys_off, wl.leaf_max, tr_n_crit(tr, wl))
        t.walk(L.theta)
        b, w = t.timing()
        t.attach(ctx, eps2_all if eps2 is None else 0.0)
        if k == 0:
            sz = t.sizes()
            same = (sz["ngroups"] == tr.ngroups and sz["n_plist"] == len(L.plist_idx)
                    and sz["n_clist"] == len(L.clist_idx))  # list entries per group are tested in the suite
        ctx.qg_run(stream.cuda_stream)
        _, f = ctx.qg_last_timing()
        if k:
            build.append(b)
            walk.append(w)
            force.append(f)
    sz = t.sizes()
    ctx.close()
    t.close()
    return {"build_ms": float(np.mean(build)), "walk_ms": float(np.mean(walk)), "force_ms": float(np.mean(force)),
            "step_ms": float(np.mean(build) + np.mean(walk) + np.mean(force)), "nodes": sz["nnodes"],
            "groups": sz["ngroups"], "list_entries": sz["n_plist"] + sz["n_clist"], "same_list_sizes_as_host": same,
            "note": "device times; attach (device-to-device copies and list checks) not included"}


def tr_n_crit(tr, wl):
    return getattr(tr, "n_crit", wl.n_crit)


def precision_compare(torch, qgrav, ctx, tr, L, eps2_all, eps2, stream, flush, steps=3):
    """All-FP64 kernel and uncentred FP32 kernel on the same lists: device time
    per step and the relative differences |a - a_64| / |a_64| (and of phi)
    against the all-FP64 GPU result over every sink."""
    a32, p32 = ctx.qg_get_forces()
    res = {}
    for name, opt in (("fp64", qgrav.Options(precision=qgrav.QG_FP64, sinks_per_thread=2, warps_per_group=4,
                                              tile_j=256)),
                      ("fp32_raw", qgrav.Options(precision=qgrav.QG_FP32_RAW))):
        c = qgrav.Context(torch.cuda.current_device(), opt)
        load_ctx(c, tr, L, eps2_all, eps2)
        c.qg_run(stream.cuda_stream)
        torch.cuda.synchronize()
        ms, _ = timed_steps(torch, c, stream, flush, steps)
        a, p = c.qg_get_forces()
        c.close()
        res[name] = {"ms_per_step": float(ms.mean()), "a": a, "phi": p}
    a64, p64 = res["fp64"]["a"], res["fp64"]["phi"]

    def pct(x):
        return {"p50": float(np.percentile(x, 50)), "p90": float(np.percentile(x, 90)),
                "p99": float(np.percentile(x, 99)), "max": float(np.max(x))}

    out = {"fp64_ms_per_step": res["fp64"]["ms_per_step"], "fp32_raw_ms_per_step": res["fp32_raw"]["ms_per_step"]}
    for name, a, p in (("fp32_centred", a32, p32), ("fp32_raw", res["fp32_raw"]["a"], res["fp32_raw"]["phi"])):
        out[name + "_vs_fp64"] = {"a": pct(np.linalg.norm(a - a64, axis=1) / np.linalg.norm(a64, axis=1)),
                                  "phi": pct(np.abs(p - p64) / np.abs(p64))}
    return out


def e2e(torch, qgrav, tr, L, eps2_all, eps2, inter, world, options=None, steps=5, shard_part=None, dist=None):
    """The step through the C-ABI from pinned host arrays: qg_evaluate_host
    copies the sinks, sources and cells (the positions are one array, sinks
    and sources: copied once); on a coherent CPU-GPU link the force kernel
    then reads the lists from host memory and writes the results there,
    else the lists are copied in chunks while the kernel runs on the groups
    already there and the results copied back.  Either way every input byte
    crosses to the device and every result byte back, each step.  With
    shard_part (N > 1, sharded) each rank evaluates its range of groups from
    its own host arrays; the time is the slowest rank's."""
    tdt = {np.dtype("float64"): torch.float64, np.dtype("int64"): torch.int64,
           np.dtype("int32"): torch.int32, np.dtype("float32"): torch.float32}

    def pin(a):
        """A page-locked host copy of a (numpy view of a pinned torch tensor)."""
        t = torch.empty(a.shape, dtype=tdt[a.dtype], pin_memory=True)
        v = t.numpy()
        v[...] = a
        return v
    x, m = pin(tr.x), pin(tr.m)
    com, cm, cq = pin(tr.cell_com), pin(tr.cell_m), pin(tr.cell_q)
    if shard_part is None:
        xs, goff = x, pin(tr.group_off)
        po, pi, co, ci = pin(L.plist_off), pin(L.plist_idx), pin(L.clist_off), pin(L.clist_idx)
        e = None if eps2 is None else pin(eps2)
    else:
        sp = shard_part
        xs, goff = pin(tr.x[sp.s0:sp.s1]), pin(sp.group_off)
        po, pi, co, ci = pin(sp.plist_off), pin(sp.plist_idx), pin(sp.clist_off), pin(sp.clist_idx)
        e = None if eps2 is None else pin(eps2[sp.s0:sp.s1])
    n = len(xs)
    a_out, p_out = pin(np.empty((n, 3))), pin(np.empty(n))
    arrays = (x, goff, m, po, pi, com, cm, cq, co, ci) + (() if xs is x else (xs,))
    h2d = sum(v.nbytes for v in arrays) + (0 if e is None else e.nbytes)
    d2h = a_out.nbytes + p_out.nbytes
    ctx = qgrav.Context(torch.cuda.current_device(), options)

    def step():
        ctx.qg_evaluate_host(xs, goff, eps2_all, e, x, m, po, pi, com, cm, cq, co, ci, a_out, p_out)

    step()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = (time.perf_counter() - t0) / steps
    in_place = bool(ctx.qg_get_stats()["eval_in_place"])
    ctx.close()
    units = world * inter
    if dist is not None:
        t = torch.tensor([dt, float(inter)], dtype=torch.float64, device="cuda")
        tmax = t[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dt = float(tmax.item())
        if shard_part is not None:
            usum = t[1:].clone()
            dist.all_reduce(usum, op=dist.ReduceOp.SUM)
            units = float(usum.item())
    route = ("lists read and results written in place by the force kernel over the coherent CPU-GPU link"
             if in_place else "list copies overlapped with the force kernel, results copied back")
    return {"value": units / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": dt * 1e3, "lists_in_place": in_place,
            "api": "qg_evaluate_host (pinned host arrays in and out; %s), wall clock" % route}


# the translation units of the FP32 force kernels (the launch shape and form are part of the record key)
KERNEL_SOURCES = ("qg_force.cuh", "qg_force_f32.cu", "qg_force_f32ep.cu", "qg_internal.h")


def kernel_hash():
    """Hash of the sources the FP32 force kernel is compiled from, comments and
    blank space removed: a recorded DRAM traffic figure is used only while
    the code it was measured on is unchanged."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1812_07313_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:12]


def _recorded_traffic(workload, launch):
    """DRAM bytes (read + write) per force-kernel launch from the ncu summary in
    profiles/, when it was taken on this workload, launch shape and source
    (the file holds one record per captured shape, separated by blank lines)."""
    path = os.path.join(ROOT, "profiles", "force_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    recs, rec = [], {}
    with open(path) as f:
        for line in f:
            if not line.strip():
                if rec:
                    recs.append(rec)
                rec = {}
            elif "=" in line and not line.lstrip().startswith("#"):
                k, v = line.split("=", 1)
                rec[k.strip()] = v.strip()
    if rec:
        recs.append(rec)
    shape = "%d%s,%d,%d,%s" % (launch["sinks_per_thread"], "a" if launch.get("sinks_adaptive") else "",
                               launch["warps_per_group"], launch["tile_j"], ARITH_TAGS[launch.get("arith", "scalar f32")])
    for r in recs:
        if r.get("workload") == workload and r.get("kernel_hash") == kernel_hash() and r.get("launch") == shape:
            try:
                return float(r["bytes_per_launch"])
            except (KeyError, ValueError):
                return None
    return None


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
