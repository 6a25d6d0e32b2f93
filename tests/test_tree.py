"""Host oct-tree and group walk (the input generator of the force path)."""
import numpy as np
import pytest

import oracle
from paper_1812_07313_gb300 import tree as qtree
from paper_1812_07313_gb300 import workloads


@pytest.fixture(scope="module")
def sphere():
    ps = workloads.small_set("sphere", 4096, 1, 1e-2)
    return ps, qtree.Tree(ps.x, ps.m, ps.sys_off, 8, 64)


def test_groups_partition_and_respect_n_crit(sphere):
    ps, tr = sphere
    g = tr.group_off
    assert g[0] == 0 and g[-1] == tr.n and np.all(np.diff(g) > 0)
    assert np.diff(g).max() <= 64
    assert np.array_equal(np.sort(tr.perm), np.arange(tr.n))
    np.testing.assert_array_equal(tr.x, ps.x[tr.perm])


def _parents(tr):
    """Parent of each node: the node of twice the side whose range holds it."""
    rng, side = tr.cell_range, tr.cell_side
    parent = np.full(tr.nnodes, -1)
    for k in range(tr.nnodes):
        cand = np.nonzero((side == 2 * side[k]) & (rng[:, 0] <= rng[k, 0]) & (rng[:, 1] >= rng[k, 1])
                          & (tr.cell_sys == tr.cell_sys[k]))[0]
        assert len(cand) <= 1
        if len(cand):
            parent[k] = cand[0]
    return parent


def test_leaves_split_at_leaf_max_and_groups_are_maximal(sphere):
    """A node is split exactly when it holds more than leaf_max particles
    (Sec. 3.4's tree, leaf <= 8 here), and a group is a maximal node with at
    most n_crit particles: its parent holds more."""
    _, tr = sphere
    parent = _parents(tr)
    cnt = tr.cell_range[:, 1] - tr.cell_range[:, 0]
    internal = np.zeros(tr.nnodes, bool)
    internal[parent[parent >= 0]] = True
    assert np.all(cnt[internal] > tr.leaf_max)
    assert np.all(cnt[~internal] <= tr.leaf_max)
    node_of_range = {(int(b), int(e)): k for k, (b, e) in enumerate(tr.cell_range)}
    for g in range(tr.ngroups):
        b, e = int(tr.group_off[g]), int(tr.group_off[g + 1])
        k = node_of_range[(b, e)]  # a group is a node
        assert e - b <= tr.n_crit
        assert parent[k] < 0 or cnt[parent[k]] > tr.n_crit


def test_lattice_groups_and_leaves_in_closed_form():
    """A 16^3 lattice has nodes of exactly n_crit = 64 and leaf_max = 8
    particles: the groups are the 64 level-2 cubes of 64 points, and the
    tree stops at the 512 level-3 cubes of 8 points (1 + 8 + 64 + 512
    nodes)."""
    g = np.arange(16, dtype=np.float64)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) / 16.0
    tr = qtree.Tree(x, np.full(len(x), 1.0 / len(x)), None, 8, 64)
    assert tr.ngroups == 64 and np.all(np.diff(tr.group_off) == 64)
    assert tr.nnodes == 1 + 8 + 64 + 512
    cnt = tr.cell_range[:, 1] - tr.cell_range[:, 0]
    assert np.array_equal(np.sort(cnt), np.sort(np.repeat([4096, 512, 64, 8], [1, 8, 64, 512])))


def test_leaves_and_ranges(sphere):
    _, tr = sphere
    cnt = tr.cell_range[:, 1] - tr.cell_range[:, 0]
    assert np.all(cnt >= 1)
    assert cnt[0] == tr.n  # root
    np.testing.assert_allclose(tr.cell_m[0], 1.0, rtol=1e-12)


def test_moments_match_eq2_direct_sum(sphere):
    """Bottom-up parallel-axis moments equal the oracle's direct Eq. 2 sum."""
    _, tr = sphere
    rng = np.random.default_rng(0)
    for k in np.concatenate([[0], rng.choice(tr.nnodes, 60, replace=False)]):
        b, e = tr.cell_range[k]
        M, com, q = oracle.cell_moments(tr.x[b:e], tr.m[b:e])
        np.testing.assert_allclose(tr.cell_m[k], M, rtol=1e-12)
        np.testing.assert_allclose(tr.cell_com[k], com, rtol=1e-12, atol=1e-14)
        scale = M * tr.cell_side[k] ** 2
        np.testing.assert_allclose(tr.cell_q[k], q, rtol=1e-9, atol=1e-11 * scale)


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 0.8])
def test_lists_cover_all_mass_exactly_once(sphere, theta):
    _, tr = sphere
    L = tr.walk(theta)
    assert L.plist_off[-1] == len(L.plist_idx) and L.clist_off[-1] == len(L.clist_idx)
    for g in range(tr.ngroups):
        pi = L.plist_idx[L.plist_off[g]:L.plist_off[g + 1]]
        ci = L.clist_idx[L.clist_off[g]:L.clist_off[g + 1]]
        # every particle is covered exactly once, by itself or by one accepted cell
        cover = np.zeros(tr.n, dtype=np.int64)
        np.add.at(cover, pi, 1)
        for c in ci:
            b, e = tr.cell_range[c]
            cover[b:e] += 1
        assert np.all(cover == 1), g


def test_accepted_cells_satisfy_opening_test(sphere):
    _, tr = sphere
    theta = 0.6
    L = tr.walk(theta)
    for g in range(0, tr.ngroups, 7):
        b, e = tr.group_off[g], tr.group_off[g + 1]
        lo, hi = tr.x[b:e].min(0), tr.x[b:e].max(0)
        for c in L.clist_idx[L.clist_off[g]:L.clist_off[g + 1]]:
            cb, ce = tr.cell_range[c]
            assert ce <= b or cb >= e  # never holds the group's own particles
            d = np.linalg.norm(np.maximum(0, np.maximum(lo - tr.cell_com[c], tr.cell_com[c] - hi)))
            assert tr.cell_side[c] < theta * d


def _acceptable(tr, k, b, e, lo, hi, theta):
    """The walk's acceptance test for node k and the group of sinks [b, e) with
    bounding box [lo, hi]: k holds none of the group's particles, its cube
    does not meet the box, and side < theta * (distance of its centre of mass
    from the box)."""
    cb, ce = tr.cell_range[k]
    if cb < e and ce > b:
        return False
    h = 0.5 * tr.cell_side[k]
    c = tr.cell_centre[k]
    if np.all(c + h >= lo) and np.all(c - h <= hi):
        return False
    d = np.linalg.norm(np.maximum(0, np.maximum(lo - tr.cell_com[k], tr.cell_com[k] - hi)))
    return tr.cell_side[k] ** 2 < theta ** 2 * d ** 2


def test_cells_are_opened_only_when_the_test_requires_it(sphere):
    """The other direction of the opening test: the parent of every accepted
    cell, and the leaf of every listed particle outside the group, failed the
    acceptance test (the walk is not more conservative than theta asks)."""
    _, tr = sphere
    theta = 0.6
    L = tr.walk(theta)
    rng = tr.cell_range
    parent = _parents(tr)
    leaf_of = np.full(tr.n, -1)
    is_parent = np.zeros(tr.nnodes, bool)
    is_parent[parent[parent >= 0]] = True
    for k in np.nonzero(~is_parent)[0]:
        leaf_of[rng[k, 0]:rng[k, 1]] = k
    assert np.all(leaf_of >= 0)
    for g in range(0, tr.ngroups, 5):
        b, e = tr.group_off[g], tr.group_off[g + 1]
        lo, hi = tr.x[b:e].min(0), tr.x[b:e].max(0)
        for c in L.clist_idx[L.clist_off[g]:L.clist_off[g + 1]]:
            assert _acceptable(tr, c, b, e, lo, hi, theta)
            assert parent[c] >= 0 and not _acceptable(tr, parent[c], b, e, lo, hi, theta)
        for i in L.plist_idx[L.plist_off[g]:L.plist_off[g + 1]]:
            if not b <= i < e:
                assert not _acceptable(tr, leaf_of[i], b, e, lo, hi, theta)


def test_multi_system_lists_stay_inside_their_system():
    ps = workloads.batched_systems(nsys=6, seed=9, n_lo=200, n_hi=900)
    tr = qtree.Tree(ps.x, ps.m, ps.sys_off, 8, 64)
    L = tr.walk(0.5)
    for g in range(tr.ngroups):
        s = tr.sink_sys[tr.group_off[g]]
        assert np.all(tr.sink_sys[tr.group_off[g]:tr.group_off[g + 1]] == s)
        pi = L.plist_idx[L.plist_off[g]:L.plist_off[g + 1]]
        ci = L.clist_idx[L.clist_off[g]:L.clist_off[g + 1]]
        assert np.all(tr.sink_sys[pi] == s)
        assert np.all(tr.cell_sys[ci] == s)
        mass = tr.m[pi].sum() + tr.cell_m[ci].sum()
        np.testing.assert_allclose(mass, 1.0, rtol=1e-12)


def test_bad_input_is_rejected():
    with pytest.raises(ValueError):
        qtree.Tree(np.array([[0.0, np.nan, 0.0]]), np.ones(1))
    with pytest.raises(ValueError):
        qtree.Tree(np.zeros((4, 3)), np.ones(4), sys_off=np.array([0, 3]))


def test_degenerate_sets():
    # one particle, and many coincident particles (depth limit)
    tr = qtree.Tree(np.zeros((1, 3)), np.ones(1))
    assert tr.ngroups == 1
    L = tr.walk(0.5)
    assert list(L.plist_idx) == [0]
    x = np.zeros((50, 3))
    tr = qtree.Tree(x, np.full(50, 0.02), leaf_max=8, n_crit=16)
    L = tr.walk(0.5)
    assert tr.group_off[-1] == 50
    assert len(L.clist_idx) == 0
