"""Group-size tuning: the sink grouping of the modified tree algorithm
(Sec. 3.4: the particles of a cell with at most n_crit particles share one
interaction list) trades list length against how well a group fills the GPU.
Larger groups open more cells (more pairs per step) but amortise each staged
list entry over more sinks.  ``tune_group_size`` builds the tree and lists
for each candidate n_crit, lets ``qg_autotune`` pick the launch shape for
each, times the force step on the GPU, and returns the candidate with the
shortest step.  ``tune_group_size`` builds the trees on the host and ranks
the candidates by the force step alone; ``tune_group_size_gpu`` builds the
same groups and lists on the GPU and ranks them by the whole GPU step, tree
build + group walk + force (T_construct + T_traverse + T_force of the
paper's timing tables): smaller groups shorten the lists but lengthen the
walk, which visits the tree once per group.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import qgrav
from . import tree as qtree


@dataclass
class GroupSizeResult:
    n_crit: int
    groups: int
    i_pp: int
    i_pc: int
    step_ms: float
    force_ms: float
    launch: dict = field(default_factory=dict)
    host_s: float = 0.0   # host tree build + walk (tune_group_size), seconds
    tree_ms: float = 0.0  # GPU tree build + walk (tune_group_size_gpu), device milliseconds

    @property
    def interactions(self) -> int:
        return self.i_pp + self.i_pc


def _time_step(ctx, steps, stream):
    step, force = [], []
    for k in range(steps + 1):
        ctx.qg_run(stream)
        s, f = ctx.qg_last_timing()
        if k:
            step.append(s)
            force.append(f)
    return float(np.mean(step)), float(np.mean(force))


def tune_group_size(x, m, sys_off, leaf_max, theta, candidates, eps2_all=0.0, eps2_of_system=None,
                    device=0, options=None, steps=3, stream=None):
    """Time one force step for every n_crit in ``candidates``.

    eps2_of_system: optional per-system eps^2 (per-sink softening is then
    set from each sink's system).  Returns (best GroupSizeResult, all results,
    (tree, lists) of the best).
    """
    results, best, best_tl = [], None, None
    for n_crit in candidates:
        t0 = time.perf_counter()
        tr = qtree.Tree(x, m, sys_off, leaf_max, int(n_crit))
        L = tr.walk(theta)
        host_s = time.perf_counter() - t0
        eps2 = None if eps2_of_system is None else np.asarray(eps2_of_system)[tr.sink_sys].astype(np.float32)
        ctx = qgrav.Context(device, options)
        try:
            ctx.qg_set_sinks(tr.x, tr.group_off, eps2_all if eps2 is None else 0.0, eps2)
            ctx.qg_set_sources(tr.x, tr.m, L.plist_off, L.plist_idx)
            ctx.qg_set_cells(tr.cell_com, tr.cell_m, tr.cell_q, L.clist_off, L.clist_idx)
            ctx.qg_autotune(stream, reps=2)
            step_ms, force_ms = _time_step(ctx, steps, stream)
            st = ctx.qg_get_stats()
        finally:
            ctx.close()
        r = GroupSizeResult(int(n_crit), tr.ngroups, int(st["i_pp"]), int(st["i_pc"]), step_ms, force_ms,
                            {k: st[k] for k in ("sinks_per_thread", "sinks_adaptive", "warps_per_group", "tile_j", "paired")},
                            host_s)
        results.append(r)
        if best is None or r.step_ms < best.step_ms:
            best, best_tl = r, (tr, L)
    return best, results, best_tl


def tune_group_size_gpu(gtree_obj, x, m, sys_off, leaf_max, theta, candidates, eps2_all=0.0, device=0,
                        options=None, steps=3, stream=None):
    """As tune_group_size, with each candidate's tree, groups and lists built
    on the GPU (``gtree.GpuTree``; x, m are CUDA tensors, one softening for
    every sink), and the best candidate the one with the shortest whole step
    (tree build + walk + force step, device times).  Leaves the tree of the
    best candidate built and walked in ``gtree_obj``.  Returns (best
    GroupSizeResult, all results)."""
    results, best = [], None
    for n_crit in candidates:
        # built and walked twice, the second timed: the first pass of a size
        # grows the tree's buffers and may walk twice to size the lists
        for _ in range(2):
            gtree_obj.build(x, m, sys_off, leaf_max, int(n_crit), stream)
            gtree_obj.walk(theta, stream)
        build_ms, walk_ms = gtree_obj.timing()
        ctx = qgrav.Context(device, options)
        try:
            gtree_obj.attach(ctx, eps2_all, stream)
            ctx.qg_autotune(stream, reps=2)
            step_ms, force_ms = _time_step(ctx, steps, stream)
            st = ctx.qg_get_stats()
        finally:
            ctx.close()
        r = GroupSizeResult(int(n_crit), int(gtree_obj.sizes()["ngroups"]), int(st["i_pp"]), int(st["i_pc"]), step_ms,
                            force_ms, {k: st[k] for k in ("sinks_per_thread", "sinks_adaptive", "warps_per_group", "tile_j", "paired")},
                            tree_ms=build_ms + walk_ms)
        results.append(r)
        if best is None or r.step_ms + r.tree_ms < best.step_ms + best.tree_ms:
            best = r
    if best is not None and best.n_crit != results[-1].n_crit:
        gtree_obj.build(x, m, sys_off, leaf_max, best.n_crit, stream)
        gtree_obj.walk(theta, stream)
    return best, results
