"""GPU tree build, moments, groups and walk (include/qg_gtree.h) against the
host builder: the same sorted order, nodes, moments (bit for bit: both sides
evaluate the same FP64 expressions without contraction), groups and list
entries (each group's list holds the same entries as the host's depth-first
walk, in the GPU walk's own order); and a force step built entirely on the
GPU against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1812_07313_gb300 import gtree, qgrav, workloads
from paper_1812_07313_gb300 import tree as qtree
from tests.parity_util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qgrav.lib()


def _sets():
    yield "sphere_4k", workloads.small_set("sphere", 4096, 1, 1e-2), 8, 64, 0.5
    yield "plummer_20k", workloads.small_set("plummer", 20000, 5, 1e-2), 8, 32, 0.6
    yield "cube_30k", workloads.small_set("cube", 30000, 6, 1e-3), 8, 256, 0.5
    yield "batched_6", workloads.batched_systems(nsys=6, seed=9, n_lo=300, n_hi=5000), 8, 64, 0.5
    x = np.concatenate([np.zeros((40, 3)), np.random.default_rng(2).random((200, 3))])
    yield "coincident", workloads.single_system("coincident", x, 1e-3), 8, 16, 0.5
    yield "one", workloads.single_system("one", np.array([[0.5, 0.25, 0.125]]), 1e-2), 8, 64, 0.5
    # a lattice: many opening tests with side / d at theta up to rounding
    # (near-ties, decided by the walk's FP64 test)
    g = np.arange(16, dtype=np.float64)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) / 16.0
    yield "lattice_t05", workloads.single_system("lattice", lat, 1e-3), 8, 64, 0.5
    yield "lattice_t1", workloads.single_system("lattice", lat, 1e-3), 1, 8, 1.0
    yield "lattice_far", workloads.single_system("lattice", lat + 1.0e4, 1e-3), 8, 64, 0.5
    # systems that are empty (first, middle and last) next to populated ones
    pe = workloads.small_set("plummer", 3000, 17, 1e-2)
    pe.sys_off = np.array([0, 0, 1200, 1200, 3000, 3000], dtype=np.int64)
    yield "empty_systems", pe, 8, 64, 0.5


CASES = list(_sets())


def _gpu_tree(ps, leaf, ncrit, theta):
    import torch
    t = gtree.GpuTree(0)
    t.build(torch.as_tensor(ps.x).cuda(), torch.as_tensor(ps.m).cuda(), ps.sys_off, leaf, ncrit)
    t.walk(theta)
    return t


def _per_group_sorted(off, idx):
    """Each group's list segment sorted (list order is not part of the result)."""
    gid = np.repeat(np.arange(len(off) - 1), np.diff(off))
    return idx[np.lexsort((idx, gid))]


def _node_keys(rng, side):
    return [(int(b), int(e), float(s)) for (b, e), s in zip(rng, side)]


@pytest.mark.parametrize("name,ps,leaf,ncrit,theta", CASES, ids=[c[0] for c in CASES])
def test_gpu_tree_equals_host_builder(name, ps, leaf, ncrit, theta):
    h = qtree.Tree(ps.x, ps.m, ps.sys_off, leaf, ncrit)
    L = h.walk(theta)
    t = _gpu_tree(ps, leaf, ncrit, theta)
    sz = t.sizes()
    assert sz["n"] == h.n and sz["nnodes"] == h.nnodes and sz["ngroups"] == h.ngroups
    assert np.array_equal(t.host("perm"), h.perm)
    assert np.array_equal(t.host("xs"), h.x)
    assert np.array_equal(t.host("group_off"), h.group_off)
    # nodes: the same set, keyed by (sorted particle range, side length)
    gk = _node_keys(t.host("node_range"), t.host("cell_side"))
    hk = _node_keys(h.cell_range, h.cell_side)
    assert len(set(gk)) == len(gk) and set(gk) == set(hk)
    g_of = {k: i for i, k in enumerate(gk)}
    h2g = np.array([g_of[k] for k in hk], dtype=np.int64)
    assert np.array_equal(t.host("cell_m")[h2g], h.cell_m)
    assert np.array_equal(t.host("cell_com")[h2g], h.cell_com)
    assert np.array_equal(t.host("cell_q")[h2g], h.cell_q)
    # lists: the same entries per group (cells mapped to the GPU numbering)
    assert np.array_equal(t.host("plist_off"), L.plist_off)
    assert np.array_equal(t.host("clist_off"), L.clist_off)
    gp, gc = t.host("plist_idx"), t.host("clist_idx")
    assert np.array_equal(_per_group_sorted(L.plist_off, gp), _per_group_sorted(L.plist_off, L.plist_idx))
    assert np.array_equal(_per_group_sorted(L.clist_off, gc), _per_group_sorted(L.clist_off, h2g[L.clist_idx]))
    # no entry twice within a group
    for off, idx in ((L.plist_off, gp), (L.clist_off, gc)):
        srt = _per_group_sorted(off, idx)
        gid = np.repeat(np.arange(len(off) - 1), np.diff(off))
        assert not np.any((srt[1:] == srt[:-1]) & (gid[1:] == gid[:-1]))
    build_ms, walk_ms = t.timing()
    assert build_ms > 0 and walk_ms > 0
    t.close()


@pytest.mark.parametrize("seed", range(6))
def test_random_parameters_match_the_host(seed):
    """Seeded random distributions, leaf sizes, group sizes, opening angles
    and system splits: nodes, moments and per-group lists as on the host."""
    rng = np.random.default_rng(100 + seed)
    kind = ["sphere", "cube", "plummer", "hernquist", "clumpy", "disk"][seed]
    n = int(rng.integers(500, 20000))
    ps = workloads.small_set(kind, n, 200 + seed, 1e-3)
    nsys = int(rng.integers(1, 4))
    cuts = np.sort(rng.choice(np.arange(1, n), nsys - 1, replace=False)) if nsys > 1 else np.zeros(0, np.int64)
    sys_off = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    leaf = int(rng.integers(1, 17))
    ncrit = int(rng.integers(leaf, 300))
    theta = float(rng.uniform(0.2, 1.0))
    h = qtree.Tree(ps.x, ps.m, sys_off, leaf, ncrit)
    L = h.walk(theta)
    import torch
    t = gtree.GpuTree(0)
    t.build(torch.as_tensor(ps.x).cuda(), torch.as_tensor(ps.m).cuda(), sys_off, leaf, ncrit)
    t.walk(theta)
    assert t.sizes()["nnodes"] == h.nnodes and t.sizes()["ngroups"] == h.ngroups
    assert np.array_equal(t.host("perm"), h.perm) and np.array_equal(t.host("group_off"), h.group_off)
    gk = _node_keys(t.host("node_range"), t.host("cell_side"))
    g_of = {k: i for i, k in enumerate(gk)}
    h2g = np.array([g_of[k] for k in _node_keys(h.cell_range, h.cell_side)], dtype=np.int64)
    assert np.array_equal(t.host("cell_q")[h2g], h.cell_q)
    assert np.array_equal(t.host("plist_off"), L.plist_off) and np.array_equal(t.host("clist_off"), L.clist_off)
    assert np.array_equal(_per_group_sorted(L.plist_off, t.host("plist_idx")),
                          _per_group_sorted(L.plist_off, L.plist_idx))
    assert np.array_equal(_per_group_sorted(L.clist_off, t.host("clist_idx")),
                          _per_group_sorted(L.clist_off, h2g[L.clist_idx]))
    t.close()


@pytest.mark.parametrize("n", [3000, 40000])
def test_walk_that_opens_everything(n):
    """theta = 0 opens every node: each group's particle list is all n
    particles.  Far more entries than the walk's first guess of the list
    size (it walks again with the exact totals), and at n = 40000 longer
    lists than a warp's staging area (it falls back to two passes); a later
    walk of the same tree at theta 0.5 still matches the host."""
    ps = workloads.small_set("plummer", n, 23, 1e-2)
    h = qtree.Tree(ps.x, ps.m, ps.sys_off, 8, 64)
    t = _gpu_tree(ps, 8, 64, 0.0)
    L0 = h.walk(0.0)
    assert t.sizes()["n_plist"] == len(L0.plist_idx) == h.ngroups * n
    assert np.array_equal(t.host("plist_off"), L0.plist_off)
    assert np.array_equal(_per_group_sorted(L0.plist_off, t.host("plist_idx")),
                          _per_group_sorted(L0.plist_off, L0.plist_idx))
    assert t.sizes()["n_clist"] == 0
    t.walk(0.5)
    L = h.walk(0.5)
    assert np.array_equal(t.host("plist_off"), L.plist_off) and np.array_equal(t.host("clist_off"), L.clist_off)
    assert np.array_equal(_per_group_sorted(L.plist_off, t.host("plist_idx")),
                          _per_group_sorted(L.plist_off, L.plist_idx))
    t.close()


def test_gpu_built_step_matches_oracle_and_host_lists():
    import torch
    ps = workloads.small_set("plummer", 30000, 11, 1e-2)
    eps2 = 1e-4
    t = _gpu_tree(ps, 8, 64, 0.5)
    ctx = qgrav.Context(0)
    t.attach(ctx, eps2)
    ctx.qg_run()
    a, phi = ctx.qg_get_forces()
    # the same step from the host builder's lists
    h = qtree.Tree(ps.x, ps.m, ps.sys_off, 8, 64)
    L = h.walk(0.5)
    ctx2 = qgrav.Context(0)
    ctx2.qg_set_sinks(h.x, h.group_off, eps2)
    ctx2.qg_set_sources(h.x, h.m, L.plist_off, L.plist_idx)
    ctx2.qg_set_cells(h.cell_com, h.cell_m, h.cell_q, L.clist_off, L.clist_idx)
    ctx2.qg_run()
    a2, phi2 = ctx2.qg_get_forces()
    a_ref, phi_ref = oracle.expansion_forces(h.group_off, h.x, h.x, h.m, L.plist_off, L.plist_idx, h.cell_com,
                                             h.cell_m, h.cell_q, L.clist_off, L.clist_idx, eps2_all=eps2)
    assert_parity(a, phi, a_ref, phi_ref, label="gpu-built step")
    assert_parity(a2, phi2, a_ref, phi_ref, label="host-built step")
    # the oracle on the GPU's own lists and cells as well
    a_g, phi_g = oracle.expansion_forces(t.host("group_off"), t.host("xs"), t.host("xs"), t.host("ms"),
                                         t.host("plist_off"), t.host("plist_idx"), t.host("cell_com"),
                                         t.host("cell_m"), t.host("cell_q"), t.host("clist_off"),
                                         t.host("clist_idx"), eps2_all=eps2)
    assert_parity(a, phi, a_g, phi_g, label="gpu-built step, oracle on gpu lists")
    # back to input order
    ad = torch.empty((ps.n, 3), dtype=torch.float64, device="cuda")
    pd = torch.empty(ps.n, dtype=torch.float64, device="cuda")
    cs = torch.cuda.current_stream().cuda_stream  # one stream for the copy and the unsort
    ctx.qg_get_forces_dev(ad, pd, cs)
    a_in = torch.empty_like(ad)
    t.unsort(ad, a_in, 3, cs)
    torch.cuda.synchronize()
    expect = np.empty_like(a)
    expect[h.perm] = a
    assert np.array_equal(a_in.cpu().numpy(), expect)
    ctx.close()
    ctx2.close()
    t.close()


def test_attach_move_equals_attach():
    """qg_gtree_attach_move hands the walk's lists to a context without copies:
    the step equals the one from the copying attach bit for bit; the tree then
    holds no lists (NULL pointers, QG_ERR_STATE on a second attach) until its
    next walk; the buffers it got back serve that walk; and a context that
    takes lists twice in a row (as the integrator does every step) keeps
    giving the copying attach's results."""
    import torch
    ps = workloads.small_set("plummer", 30000, 11, 1e-2)
    eps2 = 1e-4
    t = _gpu_tree(ps, 8, 64, 0.5)
    ctx_copy, ctx_move = qgrav.Context(0), qgrav.Context(0)
    t.attach(ctx_copy, eps2)
    ctx_copy.qg_run()
    a0, p0 = ctx_copy.qg_get_forces()
    st0 = ctx_copy.qg_get_stats()
    t.attach_move(ctx_move, eps2)
    assert t.pointers()["plist_idx"] is None and t.pointers()["clist_off"] is None
    for attach in (t.attach, t.attach_move):
        with pytest.raises(qgrav.QGError) as e:
            attach(qgrav.Context(0), eps2)
        assert e.value.status == qgrav.QG_ERR_STATE
    ctx_move.qg_run()
    a1, p1 = ctx_move.qg_get_forces()
    st1 = ctx_move.qg_get_stats()
    assert np.array_equal(a1, a0) and np.array_equal(p1, p0)
    for k in ("n_sinks", "n_groups", "n_plist", "n_clist", "i_pp", "i_pc"):
        assert st1[k] == st0[k], k
    # a second system through the same tree and the same two contexts
    ps2 = workloads.small_set("sphere", 12000, 3, 1e-2)
    t.build(torch.as_tensor(ps2.x).cuda(), torch.as_tensor(ps2.m).cuda(), ps2.sys_off, 8, 32)
    t.walk(0.6)
    t.attach(ctx_copy, eps2)
    ctx_copy.qg_run()
    a2, p2 = ctx_copy.qg_get_forces()
    t.attach_move(ctx_move, eps2)
    ctx_move.qg_run()
    a3, p3 = ctx_move.qg_get_forces()
    assert np.array_equal(a3, a2) and np.array_equal(p3, p2)
    # and the first system again: the walk refills the buffers the tree got back
    t.build(torch.as_tensor(ps.x).cuda(), torch.as_tensor(ps.m).cuda(), ps.sys_off, 8, 64)
    t.walk(0.5)
    assert t.pointers()["plist_idx"] is not None
    t.attach_move(ctx_move, eps2)
    ctx_move.qg_run()
    a4, p4 = ctx_move.qg_get_forces()
    assert np.array_equal(a4, a0) and np.array_equal(p4, p0)
    for c in (ctx_copy, ctx_move):
        c.close()
    t.close()


@pytest.mark.parametrize("name", ["cube_1m", "plummer_4m"])
def test_full_size_gpu_built_step_sampled(name):
    """The whole step on the GPU at full size (tree, moments, groups, walk,
    force kernel), against the oracle on the GPU's own lists for sampled
    groups (the largest and the longest-listed among them)."""
    import torch
    wl = workloads.WORKLOADS[name]
    ps = wl.particles()
    eps2 = float(ps.eps[0]) ** 2
    t = gtree.GpuTree(0)
    t.build(torch.as_tensor(ps.x).cuda(), torch.as_tensor(ps.m).cuda(), ps.sys_off, wl.leaf_max, wl.n_crit)
    t.walk(wl.theta)
    ctx = qgrav.Context(0)
    t.attach(ctx, eps2)
    ctx.qg_autotune(None, reps=1)
    ctx.qg_run()
    a, phi = ctx.qg_get_forces()
    ctx.close()
    h = {k: t.host(k) for k in ("group_off", "xs", "ms", "plist_off", "plist_idx", "cell_com", "cell_m", "cell_q",
                                "clist_off", "clist_idx")}
    t.close()
    G = len(h["group_off"]) - 1
    ni = np.diff(h["group_off"])
    nl = np.diff(h["plist_off"]) + np.diff(h["clist_off"])
    rng = np.random.default_rng(4)
    groups = np.array(sorted(set(rng.choice(G, 46, replace=False).tolist()) | {int(np.argmax(ni)), int(np.argmax(nl))}))
    a_ref, phi_ref = oracle.expansion_forces(h["group_off"], h["xs"], h["xs"], h["ms"], h["plist_off"],
                                             h["plist_idx"], h["cell_com"], h["cell_m"], h["cell_q"],
                                             h["clist_off"], h["clist_idx"], eps2_all=eps2, groups=groups)
    sinks = np.concatenate([np.arange(h["group_off"][g], h["group_off"][g + 1]) for g in groups])
    assert_parity(a[sinks], phi[sinks], a_ref[sinks], phi_ref[sinks], label="%s gpu-built" % name)


def test_gpu_tree_rejects_bad_arguments():
    import torch
    t = gtree.GpuTree(0)
    x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    m = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(qgrav.QGError):
        t.build(x, m, np.array([0, 3]), 8, 64)  # offsets do not cover n
    with pytest.raises(qgrav.QGError):
        t.walk(0.5)  # nothing built
    t.build(x, m, None, 8, 64)
    t.walk(0.5)
    assert t.sizes()["ngroups"] == 1
    t.close()
