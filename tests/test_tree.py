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
