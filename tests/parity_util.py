"""Shared helpers of the parity tests: seeded inputs -> tree lists -> the CUDA
path (through the qg_* C-ABI) and the FP64 oracle on the same lists."""
import numpy as np

import oracle
from paper_1812_07313_gb300 import qgrav
from paper_1812_07313_gb300 import tree as qtree
from paper_1812_07313_gb300 import workloads

# Tolerances for the FP32 mixed-precision path against the FP64 oracle:
# median and 99th percentile of |da|/|a| (and of |dphi|/|phi|).
TOL_MEDIAN = 1e-6
TOL_P99 = 1e-5
# The all-FP64 kernel differs from the oracle only by summation order.
TOL_FP64 = 1e-11


class Case:
    """A particle set, its tree and the lists of one walk."""

    def __init__(self, ps, theta, leaf_max=8, n_crit=64):
        self.ps = ps
        self.tree = qtree.Tree(ps.x, ps.m, ps.sys_off, leaf_max, n_crit)
        self.lists = self.tree.walk(theta)
        self.theta = theta
        # per-sink eps^2 when systems carry different softenings
        if ps.nsys > 1 and len(set(ps.eps.tolist())) > 1:
            self.eps2 = (ps.eps[self.tree.sink_sys] ** 2).astype(np.float32)
            self.eps2_all = 0.0
        else:
            self.eps2 = None
            self.eps2_all = float(ps.eps[0]) ** 2

    @classmethod
    def workload(cls, name, theta=None):
        wl = workloads.WORKLOADS[name]
        return cls(wl.particles(), wl.theta if theta is None else theta, wl.leaf_max, wl.n_crit)

    def gpu(self, options=None, ctx=None, autotune=False):
        """Forces from the CUDA path; autotune: at the launch shape qg_autotune
        picks (the benchmark's configuration)."""
        t, L = self.tree, self.lists
        own = ctx is None
        if own:
            ctx = qgrav.Context(0, options)
        elif options is not None:
            ctx.set_options(options)
        ctx.qg_set_sinks(t.x, t.group_off, self.eps2_all, self.eps2)
        ctx.qg_set_sources(t.x, t.m, L.plist_off, L.plist_idx)
        ctx.qg_set_cells(t.cell_com, t.cell_m, t.cell_q, L.clist_off, L.clist_idx)
        if autotune:
            ctx.qg_autotune(None, reps=1)
        ctx.qg_run()
        a, phi = ctx.qg_get_forces()
        stats = ctx.qg_get_stats()
        if own:
            ctx.close()
        return a, phi, stats

    def oracle(self, use_quad=True, groups=None):
        t, L = self.tree, self.lists
        eps2 = None if self.eps2 is None else self.eps2.astype(np.float64)
        return oracle.expansion_forces(t.group_off, t.x, t.x, t.m, L.plist_off, L.plist_idx,
                                       t.cell_com, t.cell_m, t.cell_q, L.clist_off, L.clist_idx,
                                       eps2_all=self.eps2_all, sink_eps2=eps2, use_quad=use_quad,
                                       groups=groups)

    def sample_groups(self, k, seed=0):
        rng = np.random.default_rng(seed)
        G = self.tree.ngroups
        if k >= G:
            return np.arange(G)
        # always include the largest group and the one with the longest list
        ni = np.diff(self.tree.group_off)
        nl = np.diff(self.lists.plist_off) + np.diff(self.lists.clist_off)
        pick = set(rng.choice(G, k - 2, replace=False).tolist()) | {int(np.argmax(ni)), int(np.argmax(nl))}
        return np.array(sorted(pick), dtype=np.int64)

    def sinks_of(self, groups):
        g = self.tree.group_off
        return np.concatenate([np.arange(g[i], g[i + 1]) for i in groups])


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if x.ndim == 2:
        return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)
    return np.abs(x - ref) / np.abs(ref)


def summary(e):
    return {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)), "max": float(np.max(e))}


def assert_parity(a, phi, a_ref, phi_ref, med=TOL_MEDIAN, p99=TOL_P99, label=""):
    ea, ep = rel_err(a, a_ref), rel_err(phi, phi_ref)
    sa, sp = summary(ea), summary(ep)
    print("%s |da|/|a| %s |dphi|/|phi| %s" % (label, sa, sp))
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(phi))
    assert sa["median"] <= med and sa["p99"] <= p99, (label, sa)
    assert sp["median"] <= med and sp["p99"] <= p99, (label, sp)
    return sa, sp
