"""The paper's accuracy study and its Table 3, on the GPU path.

``accuracy``: the force error of Eq. 8 for every particle of a 65,536-body
homogeneous sphere, Plummer model or exponential disk (Sec. 4, Figs. 1-2):
the tree forces from the GPU tree, walk and FP32 force kernel, the reference
from FP64 direct summation on the GPU; percentiles and the cumulative
distribution per theta, monopole-only and quadrupole cells, and the fitted
slope of the 90% error against theta (the paper finds about 5/2 and 7/2).

``table3``: the wall-clock split of one force evaluation for 4,194,304
particles (Table 3): T_construct (tree, moments, groups), T_traverse (group
walk), T_force (force kernel), monopole-only against quadrupole at the
paper's paired thetas, with the 90% error of each row on sampled sinks.

    python -m paper_1812_07313_gb300.study --accuracy --table3
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import gtree, qgrav, workloads

KINDS = {"sphere": "homogeneous sphere", "plummer": "Plummer model", "disk": "exponential disk"}
# Table 3's rows: (distribution, monopole theta, quadrupole theta)
TABLE3_PAIRS = [("sphere", 0.3, 0.65), ("sphere", 0.5, 0.75), ("plummer", 0.3, 0.4), ("plummer", 0.5, 0.6),
                ("disk", 0.3, 0.45), ("disk", 0.5, 0.65)]
# the paper's T_total [s] of those rows, monopole then quadrupole (Xeon E5-2683 v4, one core)
TABLE3_PAPER = {("sphere", 0.3): 23.99, ("sphere", 0.65): 10.88, ("sphere", 0.5): 10.26, ("sphere", 0.75): 8.35,
                ("plummer", 0.3): 41.23, ("plummer", 0.4): 44.65, ("plummer", 0.5): 15.13, ("plummer", 0.6): 22.26,
                ("disk", 0.3): 28.01, ("disk", 0.45): 24.86, ("disk", 0.5): 11.75, ("disk", 0.65): 12.67}


def _torch():
    import torch
    return torch


def _direct(torch, xs_dev, ms_dev, eps2, sinks=None):
    """FP64 direct forces on the GPU for the sorted particles (or a subset)."""
    sx = xs_dev if sinks is None else xs_dev[torch.as_tensor(sinks, device=xs_dev.device)].contiguous()
    k = sx.shape[0]
    a = torch.empty((k, 3), dtype=torch.float64, device=xs_dev.device)
    p = torch.empty(k, dtype=torch.float64, device=xs_dev.device)
    qgrav.qg_direct_dev(sx, xs_dev, ms_dev, eps2, a, p, device=xs_dev.device.index or 0)
    return a.cpu().numpy()


def _sorted_dev(torch, t):
    """The tree's sorted positions and masses as device tensors (copies)."""
    sz = t.sizes()
    xs = torch.as_tensor(t.host("xs")).cuda()
    ms = torch.as_tensor(t.host("ms")).cuda()
    return xs, ms, sz


def _forces(t, theta, eps2, expansion, tune=True):
    t.walk(theta)
    ctx = qgrav.Context(0, qgrav.Options(expansion=expansion))
    try:
        t.attach(ctx, eps2)
        if tune:
            ctx.qg_autotune(None, reps=2)
        ctx.qg_run()
        a, _ = ctx.qg_get_forces()
        _, f = ctx.qg_last_timing()
        st = ctx.qg_get_stats()
    finally:
        ctx.close()
    return a, f, st


# the paper's pairs of comparable accuracy (Sec. 4, Fig. 1): (monopole theta, quadrupole theta)
FIG1_PAIRS = {"sphere": ((0.3, 0.65), (0.5, 0.75)), "plummer": ((0.3, 0.4), (0.5, 0.6)),
              "disk": ((0.3, 0.45), (0.5, 0.65))}


def accuracy(kind, n=65536, seed=7, eps=1e-3, thetas=(0.3, 0.4, 0.45, 0.5, 0.6, 0.65, 0.7, 0.75, 0.8), n_crit=64,
             leaf_max=8):
    torch = _torch()
    ps = workloads.small_set(kind, n, seed, eps)
    t = gtree.GpuTree(0)
    t.build(torch.as_tensor(ps.x).cuda(), torch.as_tensor(ps.m).cuda(), None, leaf_max, n_crit)
    xs, ms, _ = _sorted_dev(torch, t)
    a_dir = _direct(torch, xs, ms, eps * eps)
    cdf_at = np.logspace(-6, -1, 21)
    rows = []
    for th in thetas:
        for name, ex in (("mono", qgrav.QG_MONO), ("quad", qgrav.QG_QUAD)):
            a, _, st = _forces(t, th, eps * eps, ex, tune=False)
            e = np.linalg.norm(a - a_dir, axis=1) / np.linalg.norm(a_dir, axis=1)
            rows.append({"theta": th, "cells": name, "p10": float(np.percentile(e, 10)),
                         "p50": float(np.percentile(e, 50)), "p90": float(np.percentile(e, 90)),
                         "p99": float(np.percentile(e, 99)),
                         "cdf": [float(np.mean(e <= c)) for c in cdf_at],
                         "i_pp": int(st["i_pp"]), "i_pc": int(st["i_pc"])})
    t.close()
    slopes = {}
    for name in ("mono", "quad"):
        th = np.array([r["theta"] for r in rows if r["cells"] == name])
        p = np.array([r["p90"] for r in rows if r["cells"] == name])
        slopes[name] = float(np.polyfit(np.log(th), np.log(p), 1)[0])
    pairs = []
    for tm, tq in FIG1_PAIRS[kind]:
        rm = next(r for r in rows if r["cells"] == "mono" and r["theta"] == tm)
        rq = next(r for r in rows if r["cells"] == "quad" and r["theta"] == tq)
        pairs.append({"theta_mono": tm, "theta_quad": tq,
                      "mono": {k: rm[k] for k in ("p10", "p50", "p90", "p99")},
                      "quad": {k: rq[k] for k in ("p10", "p50", "p90", "p99")}})
    return {"distribution": KINDS[kind], "n": n, "eps": eps, "n_crit": n_crit, "rows": rows,
            "cdf_error_levels": cdf_at.tolist(), "p90_slope": slopes, "fig1_pairs": pairs}


def table3(kind, theta_mono, theta_quad, n=1 << 22, seed=11, eps=1e-3, n_crit=256, leaf_max=8, reps=5,
           sample_groups=48):
    torch = _torch()
    ps = workloads.small_set(kind, n, seed, eps)
    x, m = torch.as_tensor(ps.x).cuda(), torch.as_tensor(ps.m).cuda()
    t = gtree.GpuTree(0)
    out = []
    sample = None
    for name, ex, th in (("monopole", qgrav.QG_MONO, theta_mono), ("quadrupole", qgrav.QG_QUAD, theta_quad)):
        ctx = qgrav.Context(0, qgrav.Options(expansion=ex))
        build, walk, force = [], [], []
        for k in range(reps + 1):
            t.build(x, m, None, leaf_max, n_crit)
            t.walk(th)
            b, w = t.timing()
            t.attach(ctx, eps * eps)
            if k == 0:
                ctx.qg_autotune(None, reps=2)
            ctx.qg_run()
            _, f = ctx.qg_last_timing()
            if k:
                build.append(b)
                walk.append(w)
                force.append(f)
        a, _ = ctx.qg_get_forces()
        st = ctx.qg_get_stats()
        ctx.close()
        if sample is None:
            go = t.host("group_off")
            g = np.sort(np.random.default_rng(3).choice(len(go) - 1, min(sample_groups, len(go) - 1), replace=False))
            sample = np.concatenate([np.arange(go[i], go[i + 1]) for i in g])
            xs, ms, _ = _sorted_dev(torch, t)
            a_dir = _direct(torch, xs, ms, eps * eps, sample)
        e = np.linalg.norm(a[sample] - a_dir, axis=1) / np.linalg.norm(a_dir, axis=1)
        tc, tt, tf = float(np.mean(build)), float(np.mean(walk)), float(np.mean(force))
        out.append({"program": name, "theta": th, "distribution": KINDS[kind], "T_construct_ms": tc,
                    "T_traverse_ms": tt, "T_force_ms": tf, "T_total_ms": tc + tt + tf,
                    "p90": float(np.percentile(e, 90)), "p99": float(np.percentile(e, 99)),
                    "sampled_sinks": int(len(sample)), "i_pp": int(st["i_pp"]), "i_pc": int(st["i_pc"]),
                    "paper_T_total_s": TABLE3_PAPER.get((kind, th))})
    t.close()
    base = out[0]["T_total_ms"]
    for r in out:
        r["ratio"] = r["T_total_ms"] / base
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--accuracy", action="store_true")
    ap.add_argument("--table3", action="store_true")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    res = {}
    if args.accuracy:
        res["accuracy"] = [accuracy(k) for k in KINDS]
        for r in res["accuracy"]:
            print(json.dumps({"distribution": r["distribution"], "p90_slope": r["p90_slope"],
                              "p90": {"%s %.2f" % (x["cells"], x["theta"]): x["p90"] for x in r["rows"]}}),
                  flush=True)
    if args.table3:
        res["table3"] = []
        for kind, tm, tq in TABLE3_PAIRS:
            rows = table3(kind, tm, tq)
            res["table3"].extend(rows)
            for r in rows:
                print(json.dumps(r), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    main()
