"""Splitting one force step across ranks (one GPU each).

Sink groups are independent given read-only sources and cells, so the step
shards with no collective: every rank keeps the full source and cell arrays
and evaluates a contiguous range of groups, chosen so that the ranges carry
about equal cost (FP32 work of the pairs plus list staging, the same cost the
device work queue orders groups by).  Each rank writes the accelerations and
potentials of its own sinks; gathering them is needed only by a caller that
wants every sink on every rank (an integrator), and is not part of the step.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def group_costs(group_off, plist_off, clist_off, cell_ops=33.0):
    ni = np.diff(np.asarray(group_off, dtype=np.int64)).astype(np.float64)
    npl = np.diff(np.asarray(plist_off, dtype=np.int64)).astype(np.float64)
    ncl = np.diff(np.asarray(clist_off, dtype=np.int64)).astype(np.float64)
    return ni * (13.0 * npl + cell_ops * ncl) + 64.0 * (npl + ncl) + 256.0


def split_ranges(costs, world):
    """Contiguous group ranges [g0, g1) per rank with about equal total cost."""
    costs = np.asarray(costs, dtype=np.float64)
    G = len(costs)
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, cum[-1] * r / world, side="left")))
    cuts.append(G)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, G))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


@dataclass
class Shard:
    """One rank's part of a step: sinks [s0, s1) and their groups' lists,
    offsets rebased to start at 0; list entries keep indexing the full
    (replicated) source and cell arrays."""
    g0: int
    g1: int
    s0: int
    s1: int
    group_off: np.ndarray
    plist_off: np.ndarray
    plist_idx: np.ndarray
    clist_off: np.ndarray
    clist_idx: np.ndarray


def make_shard(group_off, plist_off, plist_idx, clist_off, clist_idx, g0, g1):
    group_off = np.asarray(group_off, dtype=np.int64)
    plist_off = np.asarray(plist_off, dtype=np.int64)
    clist_off = np.asarray(clist_off, dtype=np.int64)
    s0, s1 = int(group_off[g0]), int(group_off[g1])
    p0, p1 = int(plist_off[g0]), int(plist_off[g1])
    c0, c1 = int(clist_off[g0]), int(clist_off[g1])
    return Shard(g0, g1, s0, s1, group_off[g0:g1 + 1] - s0, plist_off[g0:g1 + 1] - p0,
                 np.ascontiguousarray(plist_idx[p0:p1]), clist_off[g0:g1 + 1] - c0,
                 np.ascontiguousarray(clist_idx[c0:c1]))


def shards(group_off, plist_off, plist_idx, clist_off, clist_idx, world, cell_ops=33.0):
    costs = group_costs(group_off, plist_off, clist_off, cell_ops)
    return [make_shard(group_off, plist_off, plist_idx, clist_off, clist_idx, g0, g1)
            for g0, g1 in split_ranges(costs, world)]
