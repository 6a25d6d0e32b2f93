"""The cold-collapse runs of the paper (Sec. 5), on the GPU integrator.

A homogeneous sphere (G = M = R = 1, initial virial ratio 0.1) integrated
with the kick-drift-kick leapfrog at a fixed step; three settings:
    A: monopole-only cells, theta 0.3
    B: quadrupole cells,    theta 0.4
    C: quadrupole cells,    theta 0.65
The paper uses N = 2^22, Delta t = 2^-8 and eps = 2^-8, reports the mean
time per step (3.20, 3.70 and 2.05 s on 30 Xeon cores) and compares the
radial density profiles at t = 10 (they agree).  ``run`` reports the same
things: time per step (wall clock and its device parts), energy and virial
ratio along the run, and the density profile at the end.

    python -m paper_1812_07313_gb300.collapse --sims A,B,C --n 4194304 --t-end 10
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import qgrav, sim, workloads

SETTINGS = {"A": (qgrav.QG_MONO, 0.3), "B": (qgrav.QG_QUAD, 0.4), "C": (qgrav.QG_QUAD, 0.65)}
PAPER_S_PER_STEP = {"A": 3.20, "B": 3.70, "C": 2.05}


def density_centre(x, m, shrink=0.9, keep=1000):
    """Centre by shrinking spheres: the centre of mass of the particles within
    a sphere that shrinks by ``shrink`` each pass, until ``keep`` are left."""
    c = (m[:, None] * x).sum(axis=0) / m.sum()
    r = np.sqrt(((x - c) ** 2).sum(axis=1)).max()
    sel = np.arange(len(m))
    while len(sel) > keep:
        r *= shrink
        d2 = ((x[sel] - c) ** 2).sum(axis=1)
        nxt = sel[d2 < r * r]
        if len(nxt) < keep:
            break
        sel = nxt
        c = (m[sel, None] * x[sel]).sum(axis=0) / m[sel].sum()
    return c


def density_profile(x, m, rmin=0.01, rmax=2.0, nbins=24):
    """Spherically averaged density in log-spaced shells about the density
    centre: (shell edges, density, particles per shell)."""
    c = density_centre(x, m)
    r = np.sqrt(((x - c) ** 2).sum(axis=1))
    edges = np.logspace(np.log10(rmin), np.log10(rmax), nbins + 1)
    mass, _ = np.histogram(r, bins=edges, weights=m)
    count, _ = np.histogram(r, bins=edges)
    vol = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    return edges, mass / vol, count


def run(label, n=1 << 22, t_end=10.0, dt=2.0 ** -8, eps=2.0 ** -8, n_crit=256, seed=17, device=0,
        sample_every=64, log=None):
    expansion, theta = SETTINGS[label]
    x0, v0, m = workloads.cold_collapse(n, seed)
    s = sim.Simulation(sim.Params(theta=theta, eps2=eps * eps, n_crit=n_crit, leaf_max=8, expansion=expansion,
                                  autotune=True), device)
    s.set_state(x0, v0, m)
    K0, W0, _ = s.energy()
    nsteps = int(round(t_end / dt))
    wall, build, walk, force, integ, ipp, ipc = [], [], [], [], [], [], []
    launches = {}  # force launch (R, chosen per item, warps, tile, form) -> steps run with it
    track = [{"t": 0.0, "K": K0, "W": W0}]
    t0 = time.perf_counter()
    for k in range(1, nsteps + 1):
        s.step(dt, 1)
        tt = s.last_times()
        wall.append(tt["wall_ms"])
        build.append(tt["build_ms"])
        walk.append(tt["walk_ms"])
        force.append(tt["force_ms"])
        integ.append(tt["integrate_ms"])
        ipp.append(tt["i_pp"])
        ipc.append(tt["i_pc"])
        key = "%d%s,%d,%d,%s" % (tt["sinks_per_thread"], "a" if tt["sinks_adaptive"] else "", tt["warps_per_group"],
                                 tt["tile_j"], ("x1", "x2", "xe")[tt["form"]])
        launches[key] = launches.get(key, 0) + 1
        if k % sample_every == 0 or k == nsteps:
            K, W, _ = s.energy()
            track.append({"t": k * dt, "K": K, "W": W})
            if log:
                log("%s t=%.3f K=%.5f W=%.5f E=%.6f  %.1f ms/step" % (label, k * dt, K, W, K + W,
                                                                        np.mean(wall[-sample_every:])))
    total_s = time.perf_counter() - t0
    tunings = s.last_times()["retunes"]
    x, v, a, phi = s.state()
    s.close()
    edges, rho, count = density_profile(x, m)
    E0 = K0 + W0
    E = track[-1]["K"] + track[-1]["W"]
    return {
        "sim": label, "expansion": "mono" if expansion == qgrav.QG_MONO else "quad", "theta": theta,
        "n": n, "dt": dt, "eps": eps, "n_crit": n_crit, "steps": nsteps, "t_end": nsteps * dt,
        "s_per_step_wall": float(np.mean(wall)) / 1e3, "run_seconds": total_s,
        "ms_per_step_device": {"build": float(np.mean(build)), "walk": float(np.mean(walk)),
                               "force": float(np.mean(force)), "integrate": float(np.mean(integ))},
        "interactions_per_step": {"pp": float(np.mean(ipp)), "pc": float(np.mean(ipc))},
        "force_launch": {"tunings": int(tunings), "steps_per_shape": launches},
        "paper_s_per_step": PAPER_S_PER_STEP[label],
        "energy": {"E0": E0, "E_end": E, "rel_change": (E - E0) / abs(E0),
                   "max_rel_change": max(abs((p["K"] + p["W"] - E0) / E0) for p in track)},
        "virial_track": [(round(p["t"], 4), 2 * p["K"] / abs(p["W"])) for p in track],
        "profile": {"r_edges": edges.tolist(), "rho": rho.tolist(), "count": count.tolist()},
    }


def compare_profiles(results, rmin=0.01, rmax=1.0, min_count=100):
    """Largest |log10(rho_X / rho_A)| over shells in [rmin, rmax] holding at
    least ``min_count`` particles in both runs, for each run X against the first."""
    base = results[0]["profile"]
    e = np.asarray(base["r_edges"])
    mid = np.sqrt(e[1:] * e[:-1])
    out = {}
    for r in results[1:]:
        p = r["profile"]
        ok = ((mid >= rmin) & (mid <= rmax) & (np.asarray(base["count"]) >= min_count)
              & (np.asarray(p["count"]) >= min_count))
        d = np.abs(np.log10(np.asarray(p["rho"])[ok] / np.asarray(base["rho"])[ok]))
        out["%s_vs_%s" % (r["sim"], results[0]["sim"])] = float(d.max()) if d.size else None
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sims", default="A,B,C")
    ap.add_argument("--n", type=int, default=1 << 22)
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--dt", type=float, default=2.0 ** -8)
    ap.add_argument("--eps", type=float, default=2.0 ** -8)
    ap.add_argument("--n-crit", type=int, default=256)
    ap.add_argument("--out", default=None, help="write the results as JSON lines here")
    args = ap.parse_args()
    res = []
    for label in args.sims.split(","):
        r = run(label, args.n, args.t_end, args.dt, args.eps, args.n_crit,
                log=lambda s: print(s, flush=True))
        res.append(r)
        line = json.dumps({k: v for k, v in r.items() if k != "profile"})
        print(line, flush=True)
        if args.out:
            with open(args.out, "a") as f:
                f.write(json.dumps(r) + "\n")
    if len(res) > 1:
        print(json.dumps({"profile_max_abs_log10_ratio": compare_profiles(res)}), flush=True)


if __name__ == "__main__":
    main()
