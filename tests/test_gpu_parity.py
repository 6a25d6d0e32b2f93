"""CUDA path (through the qg_* C-ABI) against the FP64 oracle, element by element
on the same seeded inputs and lists."""
import zlib

import numpy as np
import pytest

import oracle
from paper_1812_07313_gb300 import qgrav, workloads
from tests.parity_util import Case, assert_parity, rel_err, summary, TOL_FP64, TOL_MEDIAN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qgrav.lib()  # a GPU without the built library is a failure, not a skip


@pytest.fixture(scope="module")
def sphere4k():
    return Case.workload("sphere_4k")


def test_sphere_4k_quad_all_sinks(sphere4k):
    """4096 particles in a sphere, theta = 0.5, n_crit = 64: every sink."""
    a, phi, st = sphere4k.gpu()
    a_ref, phi_ref = sphere4k.oracle()
    assert st["i_pc"] > 0 and st["i_pp"] > 0
    assert_parity(a, phi, a_ref, phi_ref, label="sphere_4k quad")


def test_sphere_4k_mono(sphere4k):
    a, phi, _ = sphere4k.gpu(qgrav.Options(expansion=qgrav.QG_MONO))
    a_ref, phi_ref = sphere4k.oracle(use_quad=False)
    assert_parity(a, phi, a_ref, phi_ref, label="sphere_4k mono")


@pytest.mark.parametrize("theta", [0.3, 0.65])
def test_exponential_disk_quad_and_mono(theta):
    """A thin exponential disk (the third distribution of the accuracy study)."""
    case = Case(workloads.small_set("disk", 20000, 19, 1e-3), theta, 8, 64)
    for exp, uq in ((qgrav.QG_QUAD, True), (qgrav.QG_MONO, False)):
        a, phi, _ = case.gpu(qgrav.Options(expansion=exp))
        a_ref, phi_ref = case.oracle(use_quad=uq)
        assert_parity(a, phi, a_ref, phi_ref, label="disk theta %.2f %s" % (theta, "quad" if uq else "mono"))


def _pin(x):
    import torch
    tdt = {np.dtype(np.float64): torch.float64, np.dtype(np.int32): torch.int32, np.dtype(np.int64): torch.int64}
    t = torch.empty(tuple(x.shape), dtype=tdt[np.asarray(x).dtype], pin_memory=True)
    t.numpy()[...] = x
    return t


def _evaluate_host(case, ctx, same_x=True, idx_fix=None, pinned=False):
    """qg_evaluate_host on the case's inputs; pinned: lists and outputs in
    page-locked memory (the in-place route on a coherent link)."""
    t, L = case.tree, case.lists
    pi, ci = L.plist_idx, L.clist_idx
    if idx_fix is not None:
        pi, ci = idx_fix(pi.copy(), ci.copy())
    src_x = t.x if same_x else t.x.copy()
    keep = []
    a_out = phi_out = None
    if pinned:
        keep = [_pin(pi), _pin(ci), _pin(np.zeros((t.n, 3))), _pin(np.zeros(t.n))]
        pi, ci, a_out, phi_out = (k.numpy() for k in keep)
    out = ctx.qg_evaluate_host(t.x, t.group_off, case.eps2_all, case.eps2, src_x, t.m, L.plist_off, pi,
                               t.cell_com, t.cell_m, t.cell_q, L.clist_off, ci, a_out, phi_out)
    if pinned:
        out = tuple(np.array(o) for o in out)  # off the pinned buffers before they are freed
    return out


@pytest.mark.parametrize("form", ["entry-paired", "entry-paired, R per item", "scalar, R per item"])
@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("name", ["sphere", "batched"])
def test_pipelined_host_evaluation_equals_the_separate_calls(name, pinned, form):
    """qg_evaluate_host gives bit for bit the results of qg_set_* + qg_run at
    the same options, with the positions copied once or twice, and leaves
    the context holding the inputs: by both routes, list copies overlapped
    with the kernel in four chunks of groups (pageable lists) and lists read
    in place by the kernel (page-locked lists and outputs), for each FP32
    form with an in-place variant (sinks per thread fixed or chosen per
    work item)."""
    if name == "sphere":
        case = Case(workloads.small_set("sphere", 6000, 31, 1e-2), 0.5, 8, 64)
    else:
        case = Case(workloads.batched_systems(nsys=6, seed=9, n_lo=300, n_hi=5000), 0.5, 8, 64)
    arith = qgrav.QG_ARITH_SCALAR if form.startswith("scalar") else qgrav.QG_ARITH_ENTRY_PAIRED
    opts = qgrav.Options(sinks_per_thread=4, warps_per_group=2, tile_j=128, arith=arith,
                         sinks_adaptive=1 if "per item" in form else 0)
    a_ref, phi_ref, st_ref = case.gpu(opts)
    ctx = qgrav.Context(0, opts)
    for same in (True, False):
        a, phi = _evaluate_host(case, ctx, same_x=same, pinned=pinned)
        assert np.array_equal(a, a_ref) and np.array_equal(phi, phi_ref)
    st = ctx.qg_get_stats()
    assert st["i_pp"] == st_ref["i_pp"] and st["i_pc"] == st_ref["i_pc"]
    assert st["eval_in_place"] == (1 if pinned else 0)
    assert st["sinks_adaptive"] == opts.sinks_adaptive
    a_d, phi_d = ctx.qg_get_forces()  # the device holds the same results
    assert np.array_equal(a_d, a_ref) and np.array_equal(phi_d, phi_ref)
    ctx.qg_run()  # the context holds the inputs: a graph step on them
    a2, phi2 = ctx.qg_get_forces()
    assert np.array_equal(a2, a_ref) and np.array_equal(phi2, phi_ref)
    ctx.qg_last_timing()
    a_o, phi_o = case.oracle()
    assert_parity(a, phi, a_o, phi_o, label="%s pipelined" % name)
    ctx.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_pipelined_host_evaluation_edge_cases(pinned):
    ctx = qgrav.Context(0)
    z3, z1 = np.zeros((0, 3)), np.zeros(0)
    off0 = np.zeros(1, dtype=np.int64)
    i0 = np.zeros(0, dtype=np.int32)
    # nothing at all
    a, phi = ctx.qg_evaluate_host(z3, off0, 1e-4, None, z3, z1, off0, i0, z3, z1, np.zeros((0, 6)), off0, i0)
    assert a.shape == (0, 3) and phi.shape == (0,)
    # sinks in groups whose lists are all empty (and an empty group): zero force and potential
    x = np.random.default_rng(1).random((50, 3))
    goff = np.array([0, 20, 20, 50], dtype=np.int64)
    lo = np.zeros(4, dtype=np.int64)
    outs = (_pin(np.ones((50, 3))), _pin(np.ones(50))) if pinned else (None, None)
    a, phi = ctx.qg_evaluate_host(x, goff, 1e-4, None, x, np.full(50, 0.02), lo, i0, z3, z1, np.zeros((0, 6)),
                                  lo, i0, *(o.numpy() if pinned else o for o in outs))
    assert np.all(a == 0.0) and np.all(phi == 0.0)
    assert ctx.qg_get_stats()["eval_in_place"] == (1 if pinned else 0)
    # one group only (fewer groups than chunks), zero softening on the guarded path
    ps = workloads.small_set("sphere", 300, 3, 0.0)
    case = Case(ps, 0.5, 8, 512)
    assert case.tree.ngroups == 1
    a, phi = _evaluate_host(case, ctx, pinned=pinned)
    a_o, phi_o = case.oracle()
    assert_parity(a, phi, a_o, phi_o, label="one group, eps 0")
    # a group larger than one pass of the CTA (several sink chunks re-read its list)
    ps = workloads.small_set("plummer", 3000, 4, 1e-2)
    case = Case(ps, 0.5, 8, 3000)
    assert case.tree.ngroups == 1
    a_ref, phi_ref, _ = case.gpu(qgrav.Options(sinks_per_thread=2, warps_per_group=2), ctx=ctx)
    a, phi = _evaluate_host(case, ctx, pinned=pinned)
    assert np.array_equal(a, a_ref) and np.array_equal(phi, phi_ref)
    ctx.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_pipelined_host_evaluation_rejects_bad_entries(pinned):
    case = Case(workloads.small_set("plummer", 3000, 5, 1e-2), 0.5, 8, 64)
    ctx = qgrav.Context(0)

    def bad_cell(pi, ci):
        ci[len(ci) // 2] = len(case.tree.cell_m) + 5
        return pi, ci

    def bad_particle(pi, ci):
        pi[-1] = -1
        return pi, ci

    for fix in (bad_cell, bad_particle):
        with pytest.raises(qgrav.QGError) as e:
            _evaluate_host(case, ctx, idx_fix=fix, pinned=pinned)
        assert e.value.status == qgrav.QG_ERR_ARG
        with pytest.raises(qgrav.QGError):
            ctx.qg_run()  # the failed call left no runnable inputs
    a, phi = _evaluate_host(case, ctx, pinned=pinned)  # and the context is still usable
    assert ctx.qg_get_stats()["eval_in_place"] == (1 if pinned else 0)
    a_o, phi_o = case.oracle()
    assert_parity(a, phi, a_o, phi_o, label="after rejected inputs")
    # a bad entry in the list of a group with no sinks is found too
    x = np.random.default_rng(2).random((40, 3))
    goff = np.array([0, 40, 40], dtype=np.int64)
    po = np.array([0, 5, 8], dtype=np.int64)
    pi = np.array([0, 1, 2, 3, 4, 5, 6, 40], dtype=np.int32)
    co = np.zeros(3, dtype=np.int64)
    i0 = np.zeros(0, dtype=np.int32)
    if pinned:
        kp = [_pin(pi), _pin(np.zeros((40, 3))), _pin(np.zeros(40))]
        args = (kp[0].numpy(), kp[1].numpy(), kp[2].numpy())
    else:
        args = (pi, None, None)
    with pytest.raises(qgrav.QGError) as e:
        ctx.qg_evaluate_host(x, goff, 1e-4, None, x, np.full(40, 0.025), po, args[0], np.zeros((0, 3)),
                             np.zeros(0), np.zeros((0, 6)), co, i0, args[1], args[2])
    assert e.value.status == qgrav.QG_ERR_ARG
    # list entries with no sources at all are refused on the host
    with pytest.raises(qgrav.QGError) as e:
        ctx.qg_evaluate_host(x, goff, 1e-4, None, np.zeros((0, 3)), np.zeros(0), po, pi, np.zeros((0, 3)),
                             np.zeros(0), np.zeros((0, 6)), co, i0)
    assert e.value.status == qgrav.QG_ERR_ARG
    # offsets that decrease, and an invalid softening, are found on the host
    # (while the first copies run) before any kernel is queued
    pi_ok = np.array([0, 1, 2, 3, 4, 5, 6, 7], dtype=np.int32)
    for go, pof, e2 in ((np.array([0, 41, 40], dtype=np.int64), po, None),
                        (goff, np.array([0, 9, 8], dtype=np.int64), None),
                        (goff, po, np.where(np.arange(40) == 17, -1.0, 0.01).astype(np.float32))):
        with pytest.raises(qgrav.QGError) as e:
            ctx.qg_evaluate_host(x, go, 1e-4, e2, x, np.full(40, 0.025), pof, pi_ok, np.zeros((0, 3)), np.zeros(0),
                                 np.zeros((0, 6)), co, i0)
        assert e.value.status == qgrav.QG_ERR_ARG
    a, phi = ctx.qg_evaluate_host(x, goff, 1e-4, None, x, np.full(40, 0.025), po, pi_ok, np.zeros((0, 3)),
                                  np.zeros(0), np.zeros((0, 6)), co, i0)
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(phi))
    ctx.close()


def test_sphere_4k_fp64_kernel(sphere4k):
    for exp, uq in ((qgrav.QG_QUAD, True), (qgrav.QG_MONO, False)):
        a, phi, _ = sphere4k.gpu(qgrav.Options(precision=qgrav.QG_FP64, expansion=exp))
        a_ref, phi_ref = sphere4k.oracle(use_quad=uq)
        assert_parity(a, phi, a_ref, phi_ref, med=TOL_FP64, p99=TOL_FP64, label="sphere_4k fp64")


# the FP32 forms: scalar, two sinks per float2, two list entries per float2
FORMS = [qgrav.QG_ARITH_SCALAR, qgrav.QG_ARITH_PAIRED, qgrav.QG_ARITH_ENTRY_PAIRED]
FORM_STAT = {qgrav.QG_ARITH_SCALAR: 0, qgrav.QG_ARITH_PAIRED: 1, qgrav.QG_ARITH_ENTRY_PAIRED: 2}


@pytest.mark.parametrize("arith", FORMS)
@pytest.mark.parametrize("R,warps,tile,flush", [
    (2, 2, 32, 16), (2, 8, 96, 0), (4, 2, 64, 40), (4, 4, 256, 0), (4, 8, 1024, 1000),
    (8, 2, 128, 0), (8, 4, 512, 8)])
def test_launch_shapes_and_ragged_tiles(sphere4k, R, warps, tile, flush, arith):
    """Every supported launch shape in every FP32 form (scalar; two sinks per
    float2; two list entries per float2, with f32x2 instructions), tiles that
    leave ragged tails (odd ones pad the entry-paired form), and FP64 folds
    from every entry to never."""
    if arith == qgrav.QG_ARITH_ENTRY_PAIRED and R > 4:
        pytest.skip("the entry-paired form holds at most 4 sinks per thread")
    o = qgrav.Options(tile_j=tile, warps_per_group=warps, sinks_per_thread=R, flush_j=flush, arith=arith)
    a, phi, st = sphere4k.gpu(o)
    assert st["sinks_per_thread"] == R and st["tile_j"] == tile
    assert st["paired"] == FORM_STAT[arith]
    a_ref, phi_ref = sphere4k.oracle()
    assert_parity(a, phi, a_ref, phi_ref, label="shape %s" % ((R, warps, tile, flush, arith),))


@pytest.mark.parametrize("arith", FORMS)
def test_mono_and_guard_in_every_form(arith):
    """Monopole-only cells and the zero-softening guard in every FP32 form,
    at the stated tolerance."""
    ps = workloads.small_set("sphere", 1500, 14, 0.0)
    case = Case(ps, 0.6)
    for exp, uq in ((qgrav.QG_QUAD, True), (qgrav.QG_MONO, False)):
        a, phi, _ = case.gpu(qgrav.Options(expansion=exp, arith=arith))
        a_ref, phi_ref = case.oracle(use_quad=uq)
        assert_parity(a, phi, a_ref, phi_ref, label="eps=0 %s %s" % (exp, arith))


def test_autotuner_picks_a_supported_shape_and_keeps_parity(sphere4k):
    t, L = sphere4k.tree, sphere4k.lists
    ctx = qgrav.Context(0)
    ctx.qg_set_sinks(t.x, t.group_off, sphere4k.eps2_all)
    ctx.qg_set_sources(t.x, t.m, L.plist_off, L.plist_idx)
    ctx.qg_set_cells(t.cell_com, t.cell_m, t.cell_q, L.clist_off, L.clist_idx)
    best, ms = ctx.qg_autotune(reps=2)
    assert best.sinks_per_thread in (2, 4, 8) and best.warps_per_group in (2, 4, 8)
    assert best.tile_j in (128, 256, 512, 1024) and ms > 0
    st = ctx.qg_get_stats()
    assert st["sinks_per_thread"] == best.sinks_per_thread and st["tile_j"] == best.tile_j
    a0, p0 = ctx.qg_get_forces()
    ctx.qg_run()
    a, phi = ctx.qg_get_forces()
    ctx.close()
    assert np.array_equal(a, a0) and np.array_equal(phi, p0)
    a_ref, phi_ref = sphere4k.oracle()
    assert_parity(a, phi, a_ref, phi_ref, label="autotuned %s" % best)


def test_group_size_tuning_picks_the_fastest_and_keeps_parity():
    from paper_1812_07313_gb300 import tuning
    ps = workloads.batched_systems(nsys=6, seed=13, n_lo=800, n_hi=4000)
    best, table, (tr, L) = tuning.tune_group_size(ps.x, ps.m, ps.sys_off, 8, 0.5, [16, 64, 256],
                                                  eps2_all=1e-4, steps=2)
    assert [r.n_crit for r in table] == [16, 64, 256]
    assert best.step_ms == min(r.step_ms for r in table)
    assert np.diff(tr.group_off).max() <= best.n_crit
    ctx = qgrav.Context(0)
    ctx.qg_set_sinks(tr.x, tr.group_off, 1e-4)
    ctx.qg_set_sources(tr.x, tr.m, L.plist_off, L.plist_idx)
    ctx.qg_set_cells(tr.cell_com, tr.cell_m, tr.cell_q, L.clist_off, L.clist_idx)
    ctx.qg_run()
    a, phi = ctx.qg_get_forces()
    ctx.close()
    a_ref, phi_ref = oracle.expansion_forces(tr.group_off, tr.x, tr.x, tr.m, L.plist_off, L.plist_idx,
                                             tr.cell_com, tr.cell_m, tr.cell_q, L.clist_off, L.clist_idx,
                                             eps2_all=1e-4)
    assert_parity(a, phi, a_ref, phi_ref, label="tuned n_crit %d" % best.n_crit)


@pytest.mark.parametrize("arith", FORMS)
def test_deterministic_and_repeatable(sphere4k, arith):
    ctx = qgrav.Context(0, qgrav.Options(arith=arith))
    a1, p1, _ = sphere4k.gpu(ctx=ctx)
    ctx.qg_run()
    a2, p2 = ctx.qg_get_forces()
    ctx.close()
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)


def test_device_pointer_entry_points_match_host(sphere4k):
    import torch
    t, L = sphere4k.tree, sphere4k.lists
    a_h, phi_h, _ = sphere4k.gpu()
    d = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)
    ctx = qgrav.Context(0)
    ctx.qg_set_sinks_dev(d(t.x, torch.float64), d(t.group_off, torch.int64), sphere4k.eps2_all)
    ctx.qg_set_sources_dev(d(t.x, torch.float64), d(t.m, torch.float64), d(L.plist_off, torch.int64),
                           d(L.plist_idx, torch.int32))
    ctx.qg_set_cells_dev(d(t.cell_com, torch.float64), d(t.cell_m, torch.float64), d(t.cell_q, torch.float64),
                         d(L.clist_off, torch.int64), d(L.clist_idx, torch.int32))
    stream = torch.cuda.current_stream().cuda_stream
    ctx.qg_run(stream)
    a = torch.empty((t.n, 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(t.n, dtype=torch.float64, device="cuda")
    ctx.qg_get_forces_dev(a, phi, stream)
    torch.cuda.synchronize()
    ctx.close()
    assert np.array_equal(a.cpu().numpy(), a_h) and np.array_equal(phi.cpu().numpy(), phi_h)


def test_gpu_direct_sum_matches_oracle():
    import torch
    ps = workloads.small_set("plummer", 3000, 4, 0.01)
    sinks = ps.x[::7]
    a_ref, phi_ref = oracle.direct_forces(sinks, ps.x, ps.m, eps2_all=1e-4)
    d = lambda x: torch.as_tensor(np.ascontiguousarray(x)).cuda()
    a = torch.empty((len(sinks), 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(len(sinks), dtype=torch.float64, device="cuda")
    qgrav.qg_direct_dev(d(sinks), d(ps.x), d(ps.m), 1e-4, a, phi)
    assert np.max(rel_err(a.cpu().numpy(), a_ref)) < 1e-12
    assert np.max(rel_err(phi.cpu().numpy(), phi_ref)) < 1e-12


# ------------------------------------------------------------------ edge cases

def _explicit(sink_x, group_off, src_x, src_m, plist_off, plist_idx, com, cm, cq, clist_off, clist_idx,
              eps2_all, eps2=None, options=None):
    ctx = qgrav.Context(0, options)
    ctx.qg_set_sinks(sink_x, group_off, eps2_all, eps2)
    ctx.qg_set_sources(src_x, src_m, plist_off, plist_idx)
    ctx.qg_set_cells(com, cm, cq, clist_off, clist_idx)
    ctx.qg_run()
    a, phi = ctx.qg_get_forces()
    ctx.close()
    e = None if eps2 is None else np.asarray(eps2, dtype=np.float64)
    a_ref, phi_ref = oracle.expansion_forces(group_off, sink_x, src_x, src_m, plist_off, plist_idx, com, cm, cq,
                                             clist_off, clist_idx, eps2_all=eps2_all, sink_eps2=e,
                                             use_quad=(options is None or options.expansion == qgrav.QG_QUAD))
    return a, phi, a_ref, phi_ref


def _random_cells(rng, nc, centre, spread):
    com = centre + rng.uniform(-spread, spread, (nc, 3))
    cm = rng.uniform(0.5, 2.0, nc)
    q = np.empty((nc, 6))
    for c in range(nc):
        xs = rng.uniform(-0.3, 0.3, (5, 3))
        _, _, q[c] = oracle.cell_moments(xs, rng.uniform(0.1, 1, 5))
    return com, cm, q


def test_empty_lists_single_sinks_and_empty_groups():
    """Groups with no list entries get zero force; one-sink groups; a group
    with no sinks at all; lists of every length 0..70 (ragged tails)."""
    rng = np.random.default_rng(1)
    G = 72
    sizes = rng.integers(0, 4, G)
    sizes[5] = 0
    sizes[6] = 1
    group_off = np.concatenate([[0], np.cumsum(sizes)])
    n = int(group_off[-1])
    sink_x = rng.uniform(-1, 1, (n, 3))
    src_x = rng.uniform(-5, 5, (300, 3))
    src_m = rng.uniform(0.1, 1, 300)
    com, cm, cq = _random_cells(rng, 90, np.array([10.0, 0, 0]), 3.0)
    plen = np.arange(G) % 71
    clen = (np.arange(G) * 7) % 67
    plen[3] = 0
    clen[3] = 0
    plist_off = np.concatenate([[0], np.cumsum(plen)])
    clist_off = np.concatenate([[0], np.cumsum(clen)])
    plist_idx = rng.integers(0, 300, plist_off[-1]).astype(np.int32)
    clist_idx = rng.integers(0, 90, clist_off[-1]).astype(np.int32)
    for arith in FORMS:
        a, phi, a_ref, phi_ref = _explicit(sink_x, group_off, src_x, src_m, plist_off, plist_idx, com, cm, cq,
                                           clist_off, clist_idx, 1e-3, options=qgrav.Options(tile_j=32, arith=arith))
        no_list = np.nonzero((plen == 0) & (clen == 0))[0]
        assert 3 in no_list
        empty = np.concatenate([np.arange(group_off[g], group_off[g + 1]) for g in no_list])
        assert len(empty) > 0
        assert np.all(a[empty] == 0.0) and np.all(phi[empty] == 0.0)
        live = np.setdiff1d(np.arange(n), empty)
        assert_parity(a[live], phi[live], a_ref[live], phi_ref[live], label="edges form %d" % arith)


def test_group_larger_than_one_cta_pass():
    """A group of 1500 sinks is evaluated in several sink chunks of one CTA."""
    ps = workloads.small_set("cube", 6000, 8, 2e-3)
    case = Case(ps, 0.5, leaf_max=8, n_crit=1500)
    assert np.diff(case.tree.group_off).max() > 512
    a_ref, phi_ref = case.oracle()
    for arith in FORMS:
        for R in (2, 4):
            a, phi, _ = case.gpu(qgrav.Options(sinks_per_thread=R, arith=arith))
            assert_parity(a, phi, a_ref, phi_ref, label="big groups R=%d form %d" % (R, arith))


def test_zero_softening_skips_coincident_pairs():
    """eps = 0: the self pair of every sink has rhat = 0 and is skipped by both."""
    ps = workloads.small_set("sphere", 2000, 12, 0.0)
    case = Case(ps, 0.5)
    assert case.eps2_all == 0.0
    a_ref, phi_ref = case.oracle()
    for arith in FORMS:
        a, phi, _ = case.gpu(qgrav.Options(arith=arith))
        assert np.all(np.isfinite(a))
        assert_parity(a, phi, a_ref, phi_ref, label="eps=0 form %d" % arith)


@pytest.mark.parametrize("adaptive", [0, 1])
@pytest.mark.parametrize("arith", [qgrav.QG_ARITH_SCALAR, qgrav.QG_ARITH_ENTRY_PAIRED])
@pytest.mark.parametrize("n", [96, 97])
@pytest.mark.parametrize("origin", [0.0, 3000.0])
def test_self_pair_adds_no_force_at_tiny_softening(origin, n, arith, adaptive):
    """Every sink is also an entry of its own group's list.  With eps = 1e-9
    its own pair must give dx = 0 exactly (sink and entry offsets rounded by
    the same operations), else it adds a force of order m dx / eps^3; the
    potential keeps the pair's -m/eps, as the oracle does.  An odd list (97
    entries) gives the entry-paired form a padding entry next to these
    near-singular pairs."""
    rng = np.random.default_rng(41)
    x = origin + rng.random((n, 3))
    m = rng.uniform(0.5, 1.5, n) / n
    goff = np.array([0, 40, n], dtype=np.int64)   # two groups; each lists every particle
    off = np.array([0, n, 2 * n], dtype=np.int64)
    idx = np.concatenate([np.arange(n), np.arange(n)]).astype(np.int32)
    eps2 = 1e-18
    ctx = qgrav.Context(0, qgrav.Options(arith=arith, sinks_adaptive=adaptive))
    ctx.qg_set_sinks(x, goff, eps2)
    ctx.qg_set_sources(x, m, off, idx)
    ctx.qg_set_cells(np.zeros((0, 3)), np.zeros(0), np.zeros((0, 6)), np.zeros(3, dtype=np.int64),
                     np.zeros(0, dtype=np.int32))
    ctx.qg_run()
    a, phi = ctx.qg_get_forces()
    ctx.close()
    a_ref, phi_ref = oracle.expansion_forces(goff, x, x, m, off, idx, np.zeros((0, 3)), np.zeros(0),
                                             np.zeros((0, 6)), np.zeros(3, dtype=np.int64),
                                             np.zeros(0, dtype=np.int32), eps2_all=eps2)
    assert_parity(a, phi, a_ref, phi_ref, med=1e-6, p99=1e-5, label="self pair, origin %g" % origin)


def test_per_sink_softening():
    rng = np.random.default_rng(3)
    ps = workloads.small_set("plummer", 3000, 13, 0.02)
    case = Case(ps, 0.6)
    case.eps2 = rng.uniform(1e-4, 4e-3, case.tree.n).astype(np.float32)
    a, phi, _ = case.gpu()
    a_ref, phi_ref = case.oracle()
    assert_parity(a, phi, a_ref, phi_ref, label="per-sink eps")
    # the one-call entry point by both routes, per-sink softening included
    ctx = qgrav.Context(0)
    for pinned in (False, True):
        a2, phi2 = _evaluate_host(case, ctx, pinned=pinned)
        assert ctx.qg_get_stats()["eval_in_place"] == (1 if pinned else 0)
        assert np.array_equal(a2, a) and np.array_equal(phi2, phi)
    ctx.close()


def test_uncentred_fp32_holds_the_tolerance_near_the_origin(sphere4k):
    """The ablation kernel (absolute coordinates cast to FP32, no centring)
    on a set about the origin: the casts lose no more than the offsets'
    rounding would, and the tolerance holds."""
    a_ref, phi_ref = sphere4k.oracle()
    a, phi, _ = sphere4k.gpu(qgrav.Options(precision=qgrav.QG_FP32_RAW))
    assert_parity(a, phi, a_ref, phi_ref, label="raw fp32 near the origin")


def test_far_from_origin_needs_centring():
    """Systems thousands of units from the origin: the centred FP32 path holds
    the tolerance; casting absolute coordinates (QG_FP32_RAW) cannot."""
    ps = workloads.batched_systems(nsys=4, seed=21, n_lo=1500, n_hi=3000, spacing=4096.0)
    case = Case(ps, 0.5)
    a_ref, phi_ref = case.oracle()
    for arith in (qgrav.QG_ARITH_ENTRY_PAIRED, qgrav.QG_ARITH_SCALAR):
        a, phi, _ = case.gpu(qgrav.Options(arith=arith))
        assert_parity(a, phi, a_ref, phi_ref, label="far, centred, form %d" % arith)
    a_raw, phi_raw, _ = case.gpu(qgrav.Options(precision=qgrav.QG_FP32_RAW))
    e_raw, e_c = np.median(rel_err(a_raw, a_ref)), np.median(rel_err(a, a_ref))
    print("far: median |da|/|a| raw %.2e centred %.2e" % (e_raw, e_c))
    assert e_raw > 100 * TOL_MEDIAN and e_raw > 100 * e_c


def test_invalid_lists_are_rejected_before_any_kernel_reads_them():
    import torch
    case = Case(workloads.small_set("sphere", 500, 2, 0.01), 0.5)
    t, L = case.tree, case.lists
    ctx = qgrav.Context(0)
    ctx.qg_set_sinks(t.x, t.group_off, case.eps2_all)
    bad = L.plist_idx.copy()
    bad[len(bad) // 2] = t.n + 5
    with pytest.raises(qgrav.QGError) as e:
        ctx.qg_set_sources(t.x, t.m, L.plist_off, bad)
    assert e.value.status == qgrav.QG_ERR_ARG
    with pytest.raises(qgrav.QGError) as e:
        ctx.qg_set_sources_dev(torch.as_tensor(t.x).cuda(), torch.as_tensor(t.m).cuda(),
                               torch.as_tensor(L.plist_off).cuda(), torch.as_tensor(bad).cuda())
    assert e.value.status == qgrav.QG_ERR_ARG
    with pytest.raises(qgrav.QGError) as e:
        ctx.qg_run()
    assert e.value.status == qgrav.QG_ERR_STATE
    ctx.qg_set_sources(t.x, t.m, L.plist_off, L.plist_idx)
    ctx.qg_set_cells(t.cell_com, t.cell_m, t.cell_q, L.clist_off, L.clist_idx)
    ctx.qg_run()
    a, phi = ctx.qg_get_forces()
    # lists set for another group count are refused by the binding
    with pytest.raises(ValueError):
        ctx.qg_set_cells(t.cell_com, t.cell_m, t.cell_q, L.clist_off[:-1], L.clist_idx)
    # and offsets that do not start at 0 by the library
    off = L.clist_off.copy()
    off[0] = 1
    with pytest.raises(qgrav.QGError) as e:
        ctx.qg_set_cells(t.cell_com, t.cell_m, t.cell_q, off, np.zeros(off[-1], dtype=np.int32))
    assert e.value.status == qgrav.QG_ERR_ARG
    ctx.close()
    assert np.all(np.isfinite(a))


@pytest.mark.parametrize("arith", [qgrav.QG_ARITH_SCALAR, qgrav.QG_ARITH_ENTRY_PAIRED])
@pytest.mark.parametrize("split", [7, 64, 500, -1])
def test_split_lists_are_repeatable_and_keep_parity(sphere4k, split, arith):
    """Long lists cut into work items (group, entry range): each part's FP64
    partial sums merged by the group's last part in a fixed order.  Results
    are bitwise repeatable (twice in one context and in a fresh one), match
    the oracle at the stated tolerance, and agree with the unsplit step to
    FP32 rounding.  split 7 cuts every list (up to the maximum of 64 parts);
    -1 is the automatic mode (on this small set nearly every group is above a
    quarter of its share of the persistent grid's CTAs, so nearly every list
    is cut)."""
    o = qgrav.Options(arith=arith, split_j=split)
    ctx = qgrav.Context(0, o)
    a1, p1, st = sphere4k.gpu(ctx=ctx)
    ctx.qg_run()
    a2, p2 = ctx.qg_get_forces()
    ctx.close()
    a3, p3, st3 = sphere4k.gpu(o)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
    assert np.array_equal(a1, a3) and np.array_equal(p1, p3)
    G = sphere4k.tree.ngroups
    assert st["n_split"] > 0 and st["n_items"] > G, st
    if split == 7:
        assert st["n_split"] == G, st        # every list has more than 7 entries
    if split == -1:
        assert st["n_split"] >= 0.9 * G, st  # all but the cheapest groups
    a_ref, phi_ref = sphere4k.oracle()
    assert_parity(a1, p1, a_ref, phi_ref, label="split %d form %d" % (split, arith))
    a0, p0, st0 = sphere4k.gpu(qgrav.Options(arith=arith))
    assert st0["n_split"] == 0 and st0["n_items"] == G
    assert np.max(rel_err(a1, a0)) < 1e-5 and np.max(rel_err(p1, p0)) < 1e-5


def test_split_lists_with_empty_and_single_entry_lists():
    """Splitting leaves groups with no list entries, one entry or no sinks
    alone, and cuts lists that end in ragged tails; every part of a group of
    more sinks than one CTA pass holds (sink chunks) adds up too."""
    rng = np.random.default_rng(8)
    G = 40
    sizes = rng.integers(0, 6, G)
    sizes[3] = 0
    sizes[11] = 2
    sizes[7] = 700   # more sinks than one pass of 128 threads x 4 sinks
    group_off = np.concatenate([[0], np.cumsum(sizes)])
    n = int(group_off[-1])
    sink_x = rng.uniform(-1, 1, (n, 3))
    src_x = rng.uniform(-5, 5, (400, 3))
    src_m = rng.uniform(0.1, 1, 400)
    com, cm, cq = _random_cells(rng, 120, np.array([10.0, 0, 0]), 3.0)
    plen = (np.arange(G) * 13) % 97
    clen = (np.arange(G) * 7) % 89
    plen[5], clen[5] = 1, 0
    plen[9], clen[9] = 0, 1
    plen[11], clen[11] = 0, 0
    plist_off = np.concatenate([[0], np.cumsum(plen)])
    clist_off = np.concatenate([[0], np.cumsum(clen)])
    plist_idx = rng.integers(0, 400, plist_off[-1]).astype(np.int32)
    clist_idx = rng.integers(0, 120, clist_off[-1]).astype(np.int32)
    for arith in (qgrav.QG_ARITH_SCALAR, qgrav.QG_ARITH_ENTRY_PAIRED):
        a, phi, a_ref, phi_ref = _explicit(sink_x, group_off, src_x, src_m, plist_off, plist_idx, com, cm, cq,
                                           clist_off, clist_idx, 1e-3,
                                           options=qgrav.Options(tile_j=32, split_j=5, arith=arith))
        no_list = np.nonzero((plen == 0) & (clen == 0))[0]
        assert 11 in no_list
        empty = np.concatenate([np.arange(group_off[g], group_off[g + 1]) for g in no_list])
        assert np.all(a[empty] == 0.0) and np.all(phi[empty] == 0.0)
        live = np.setdiff1d(np.arange(n), empty)
        assert_parity(a[live], phi[live], a_ref[live], phi_ref[live], label="split edges form %d" % arith)


def test_split_option_is_checked():
    ctx = qgrav.Context(0)
    with pytest.raises(qgrav.QGError) as e:
        ctx.set_options(qgrav.Options(split_j=-2))
    assert e.value.status == qgrav.QG_ERR_ARG
    ctx.close()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_contexts_concatenate_to_the_unsharded_step(sphere4k, world):
    """The multi-GPU split of a step (contiguous cost-balanced ranges of
    groups, sources and cells replicated, no collective), run as one context
    per shard on one GPU: the shards' results, concatenated, are the
    unsharded step's bit for bit (same launch shape)."""
    from paper_1812_07313_gb300 import shard
    t, L = sphere4k.tree, sphere4k.lists
    for opt in (qgrav.Options(sinks_per_thread=4, warps_per_group=2, tile_j=256, arith=qgrav.QG_ARITH_ENTRY_PAIRED),
                qgrav.Options(sinks_per_thread=2, warps_per_group=4, tile_j=128, arith=qgrav.QG_ARITH_SCALAR)):
        a0, p0, _ = sphere4k.gpu(opt)
        parts = shard.shards(t.group_off, L.plist_off, L.plist_idx, L.clist_off, L.clist_idx, world)
        assert len(parts) == world and parts[0].s0 == 0 and parts[-1].s1 == t.n
        a_parts, p_parts = [], []
        for sh in parts:
            ctx = qgrav.Context(0, opt)
            ctx.qg_set_sinks(t.x[sh.s0:sh.s1], sh.group_off, sphere4k.eps2_all)
            ctx.qg_set_sources(t.x, t.m, sh.plist_off, sh.plist_idx)
            ctx.qg_set_cells(t.cell_com, t.cell_m, t.cell_q, sh.clist_off, sh.clist_idx)
            ctx.qg_run()
            a, phi = ctx.qg_get_forces()
            ctx.close()
            a_parts.append(a)
            p_parts.append(phi)
        assert np.array_equal(np.concatenate(a_parts), a0) and np.array_equal(np.concatenate(p_parts), p0)


@pytest.mark.parametrize("arith", [qgrav.QG_ARITH_SCALAR, qgrav.QG_ARITH_ENTRY_PAIRED])
@pytest.mark.parametrize("warps,tile", [(2, 256), (4, 128), (8, 1024)])
def test_sinks_per_thread_chosen_per_item(arith, warps, tile):
    """The kernels that choose 1 to 4 sinks per thread for every work item:
    on groups of 1 to 1500 sinks (several passes of the CTA's sink slots)
    with lists of 0 to ~3000 entries, every choice is taken; the results
    match the oracle, are bitwise repeatable, and agree with the fixed R = 4
    kernel to FP32 rounding."""
    rng = np.random.default_rng(61)
    ps = workloads.small_set("cube", 6000, 8, 2e-3)
    case = Case(ps, 0.5, leaf_max=8, n_crit=1500)
    small = Case(workloads.small_set("plummer", 5000, 9, 0.01), 0.5, leaf_max=8, n_crit=24)
    o = qgrav.Options(arith=arith, warps_per_group=warps, tile_j=tile, sinks_per_thread=4, sinks_adaptive=1)
    for c in (case, small):
        a1, p1, st = c.gpu(o)
        assert st["sinks_adaptive"] == 1 and st["sinks_per_thread"] == 4
        a2, p2, _ = c.gpu(o)
        assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
        a_ref, phi_ref = c.oracle()
        assert_parity(a1, p1, a_ref, phi_ref, label="adaptive R form %d, %d warps, tile %d" % (arith, warps, tile))
        a4, p4, _ = c.gpu(qgrav.Options(arith=arith, warps_per_group=warps, tile_j=tile, sinks_per_thread=4))
        assert np.max(rel_err(a1, a4)) < 1e-5 and np.max(rel_err(p1, p4)) < 1e-5


def test_sinks_per_thread_chosen_per_item_edges():
    """Empty and ragged lists, tiny softening with self pairs, zero softening
    (the guarded kernel) and the one-call path by both routes, bit for bit
    the separate calls."""
    for arith in (qgrav.QG_ARITH_SCALAR, qgrav.QG_ARITH_ENTRY_PAIRED):
        o = qgrav.Options(arith=arith, sinks_adaptive=1, tile_j=32)
        # zero softening: coincident self pairs skipped
        c0 = Case(workloads.small_set("sphere", 2000, 12, 0.0), 0.5)
        a, phi, _ = c0.gpu(o)
        a_ref, phi_ref = c0.oracle()
        assert_parity(a, phi, a_ref, phi_ref, label="adaptive eps=0 form %d" % arith)
        # one call from host arrays, copied and in place: the separate calls' results
        c1 = Case(workloads.batched_systems(nsys=6, seed=17, n_lo=800, n_hi=4000), 0.5)
        ctx = qgrav.Context(0, o)
        a_ref1, p_ref1, _ = c1.gpu(ctx=ctx)
        for pinned in (False, True):
            a2, p2 = _evaluate_host(c1, ctx, pinned=pinned)
            assert ctx.qg_get_stats()["eval_in_place"] == (1 if pinned else 0)
            assert np.array_equal(a2, a_ref1) and np.array_equal(p2, p_ref1)
        ctx.close()
    # the option is checked: up to 4 sinks per thread, not with the sink-paired form
    ctx = qgrav.Context(0)
    for bad in (qgrav.Options(sinks_adaptive=1, sinks_per_thread=2),
                qgrav.Options(sinks_adaptive=1, arith=qgrav.QG_ARITH_PAIRED),
                qgrav.Options(sinks_adaptive=1, precision=qgrav.QG_FP64),
                qgrav.Options(sinks_adaptive=2)):
        with pytest.raises(qgrav.QGError) as e:
            ctx.set_options(bad)
        assert e.value.status == qgrav.QG_ERR_ARG
    ctx.close()


def test_non_finite_or_out_of_range_inputs_are_rejected():
    """A position, mass, quadrupole component or softening that is not finite,
    or beyond 2^100 in magnitude, is refused (QG_ERR_ARG) by every entry point
    (host and device arrays, and the one-call evaluation), so that the FP32
    kernels' integer rounding of offsets only ever sees values inside its
    domain; the context then works again with good inputs."""
    import torch
    case = Case(workloads.small_set("sphere", 500, 2, 0.01), 0.5)
    t, L = case.tree, case.lists
    dv = lambda x: torch.as_tensor(np.ascontiguousarray(x)).cuda()
    ctx = qgrav.Context(0)
    for v in (np.nan, np.inf, 2.0 ** 101):
        x = t.x.copy()
        x[7, 1] = v
        for call in (lambda: ctx.qg_set_sinks(x, t.group_off, case.eps2_all),
                     lambda: ctx.qg_set_sinks_dev(dv(x), dv(t.group_off), case.eps2_all)):
            with pytest.raises(qgrav.QGError) as e:
                call()
            assert e.value.status == qgrav.QG_ERR_ARG, v
        ctx.qg_set_sinks(t.x, t.group_off, case.eps2_all)
        m = t.m.copy()
        m[3] = v
        with pytest.raises(qgrav.QGError) as e:
            ctx.qg_set_sources(t.x, m, L.plist_off, L.plist_idx)
        assert e.value.status == qgrav.QG_ERR_ARG
        with pytest.raises(qgrav.QGError) as e:
            ctx.qg_set_sources_dev(dv(x), dv(t.m), dv(L.plist_off), dv(L.plist_idx))
        assert e.value.status == qgrav.QG_ERR_ARG
        q = t.cell_q.copy()
        q[2, 4] = v
        com = t.cell_com.copy()
        com[1, 0] = v
        for cq, cc in ((q, t.cell_com), (t.cell_q, com)):
            with pytest.raises(qgrav.QGError) as e:
                ctx.qg_set_cells(cc, t.cell_m, cq, L.clist_off, L.clist_idx)
            assert e.value.status == qgrav.QG_ERR_ARG
            with pytest.raises(qgrav.QGError) as e:
                ctx.qg_set_cells_dev(dv(cc), dv(t.cell_m), dv(cq), dv(L.clist_off), dv(L.clist_idx))
            assert e.value.status == qgrav.QG_ERR_ARG
        with pytest.raises(qgrav.QGError) as e:
            ctx.qg_evaluate_host(x, t.group_off, case.eps2_all, None, x, t.m, L.plist_off, L.plist_idx,
                                 t.cell_com, t.cell_m, t.cell_q, L.clist_off, L.clist_idx)
        assert e.value.status == qgrav.QG_ERR_ARG
        with pytest.raises(qgrav.QGError) as e:
            ctx.qg_evaluate_host(t.x, t.group_off, case.eps2_all, None, t.x, t.m, L.plist_off, L.plist_idx,
                                 t.cell_com, t.cell_m, q, L.clist_off, L.clist_idx)
        assert e.value.status == qgrav.QG_ERR_ARG
    # softening: a global value beyond 2^100, a per-sink value that is negative or not finite
    with pytest.raises(qgrav.QGError) as e:
        ctx.qg_set_sinks(t.x, t.group_off, 2.0 ** 101)
    assert e.value.status == qgrav.QG_ERR_ARG
    for v in (-1.0, np.inf, np.nan):
        e2 = np.full(t.n, 1e-4, dtype=np.float32)
        e2[11] = v
        with pytest.raises(qgrav.QGError) as e:
            ctx.qg_set_sinks_dev(dv(t.x), dv(t.group_off), 0.0, dv(e2))
        assert e.value.status == qgrav.QG_ERR_ARG
    # good inputs afterwards: the same result as a fresh context
    a0, p0, _ = case.gpu()
    ctx.qg_set_sinks(t.x, t.group_off, case.eps2_all)
    ctx.qg_set_sources(t.x, t.m, L.plist_off, L.plist_idx)
    ctx.qg_set_cells(t.cell_com, t.cell_m, t.cell_q, L.clist_off, L.clist_idx)
    ctx.qg_run()
    a, phi = ctx.qg_get_forces()
    ctx.close()
    assert np.array_equal(a, a0) and np.array_equal(phi, p0)


def test_device_softening_array_chooses_the_kernel_like_the_host_array():
    """A per-sink softening given as a device array is checked on the GPU: all
    normal floats give bit for bit the result of the same host array; a zero
    among them selects the kernel that skips coincident pairs, and the
    result still matches the oracle."""
    import torch
    case = Case(workloads.small_set("plummer", 3000, 13, 0.02), 0.6)
    t, L = case.tree, case.lists
    dv = lambda x: torch.as_tensor(np.ascontiguousarray(x)).cuda()
    rng = np.random.default_rng(9)
    for zero in (False, True):
        e2 = rng.uniform(1e-4, 4e-3, t.n).astype(np.float32)
        if zero:
            e2[::7] = 0.0
        case.eps2, case.eps2_all = e2, 0.0
        a_h, p_h, _ = case.gpu()
        ctx = qgrav.Context(0)
        ctx.qg_set_sinks_dev(dv(t.x), dv(t.group_off), 0.0, dv(e2))
        ctx.qg_set_sources(t.x, t.m, L.plist_off, L.plist_idx)
        ctx.qg_set_cells(t.cell_com, t.cell_m, t.cell_q, L.clist_off, L.clist_idx)
        ctx.qg_run()
        a_d, p_d = ctx.qg_get_forces()
        ctx.close()
        assert np.array_equal(a_d, a_h) and np.array_equal(p_d, p_h), zero
        a_ref, phi_ref = case.oracle()
        assert_parity(a_d, p_d, a_ref, phi_ref, label="device eps2, zeros %s" % zero)


# ------------------------------------------------------------------ full sizes, sampled

@pytest.mark.parametrize("name,theta,k", [
    ("cube_1m", 0.5, 160), ("cube_1m", 0.3, 60), ("plummer_4m", 0.5, 120),
    ("batched_512", 0.5, 160), ("clumpy_16m", 0.5, 100)])
def test_full_size_sampled(name, theta, k):
    """Full workloads in the launch configuration the benchmark times; the
    oracle evaluates a seeded sample of groups (plus the largest group and
    the one with the longest list)."""
    case = Case.workload(name, theta)
    a, phi, st = case.gpu(autotune=True)
    groups = case.sample_groups(k, seed=zlib.crc32(name.encode()) % 1000)
    a_ref, phi_ref = case.oracle(groups=groups)
    s = case.sinks_of(groups)
    assert_parity(a[s], phi[s], a_ref[s], phi_ref[s], label="%s theta=%.2f" % (name, theta))
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(phi))


def test_batched_512_all_sinks_against_the_oracle():
    """The batched configuration (512 systems, 8.8 million sinks, n_crit 64,
    theta 0.5) at the autotuned launch shape, checked against the oracle on
    every sink (the oracle's groups split over the host cores)."""
    import os
    case = Case.workload("batched_512")
    a, phi, st = case.gpu(autotune=True)
    oracle.set_threads(os.cpu_count() or 1)
    try:
        a_ref, phi_ref = case.oracle()
    finally:
        oracle.set_threads(1)
    assert len(a_ref) == case.tree.n == 8826172
    assert_parity(a, phi, a_ref, phi_ref, label="batched_512, all %d sinks, launch %s" % (
        case.tree.n, {k: st[k] for k in ("sinks_per_thread", "warps_per_group", "tile_j", "paired")}))


def test_plummer_4m_theta_sweep_fp32_centred_vs_fp64_and_oracle():
    """The clustered configuration over theta 0.3 ... 0.8 (GPU-built tree and
    lists): the FP32 kernel with FP64 centring against the all-FP64 kernel on
    every sink, and both against the oracle on sampled groups (the largest
    group and the longest list included)."""
    import torch
    from paper_1812_07313_gb300 import gtree
    wl = workloads.WORKLOADS["plummer_4m"]
    ps = wl.particles()
    eps2 = float(ps.eps[0]) ** 2
    t = gtree.GpuTree(0)
    t.build(torch.as_tensor(ps.x).cuda(), torch.as_tensor(ps.m).cuda(), ps.sys_off, wl.leaf_max, wl.n_crit)
    xs, ms = t.host("xs"), t.host("ms")
    com, cm, cq = t.host("cell_com"), t.host("cell_m"), t.host("cell_q")
    goff = t.host("group_off")
    rng = np.random.default_rng(33)
    for theta in (0.3, 0.4, 0.5, 0.6, 0.7, 0.8):
        t.walk(theta)
        res = {}
        for name, opt in (("fp32", None), ("fp64", qgrav.Options(precision=qgrav.QG_FP64))):
            ctx = qgrav.Context(0, opt)
            t.attach(ctx, eps2)
            ctx.qg_run()
            res[name] = ctx.qg_get_forces()
            ctx.close()
        (a32, p32), (a64, p64) = res["fp32"], res["fp64"]
        sa, sp = assert_parity(a32, p32, a64, p64, label="theta %.1f fp32 vs fp64, every sink" % theta)
        # the oracle on sampled groups: their lists cut out of the device arrays
        po, co = t.host("plist_off"), t.host("clist_off")
        ni, nl = np.diff(goff), np.diff(po) + np.diff(co)
        groups = np.unique(np.concatenate([rng.choice(len(ni), 20, replace=False), [np.argmax(ni), np.argmax(nl)]]))
        s_goff, s_po, s_co, s_pi, s_ci, sinks = [0], [0], [0], [], [], []
        for g in groups:
            s_pi.append(t.host("plist_idx", po[g], po[g + 1]))
            s_ci.append(t.host("clist_idx", co[g], co[g + 1]))
            sinks.append(np.arange(goff[g], goff[g + 1]))
            s_goff.append(s_goff[-1] + len(sinks[-1]))
            s_po.append(s_po[-1] + len(s_pi[-1]))
            s_co.append(s_co[-1] + len(s_ci[-1]))
        sinks = np.concatenate(sinks)
        a_or, p_or = oracle.expansion_forces(np.array(s_goff), xs[sinks], xs, ms, np.array(s_po),
                                             np.concatenate(s_pi), com, cm, cq, np.array(s_co), np.concatenate(s_ci),
                                             eps2_all=eps2)
        assert_parity(a64[sinks], p64[sinks], a_or, p_or, med=TOL_FP64, p99=TOL_FP64,
                      label="theta %.1f fp64 vs oracle" % theta)
        assert_parity(a32[sinks], p32[sinks], a_or, p_or, label="theta %.1f fp32 vs oracle" % theta)
    t.close()


def test_plummer_4m_fp64_kernel_sampled():
    case = Case.workload("plummer_4m", 0.6)
    a, phi, _ = case.gpu(qgrav.Options(precision=qgrav.QG_FP64))
    groups = case.sample_groups(40, seed=5)
    a_ref, phi_ref = case.oracle(groups=groups)
    s = case.sinks_of(groups)
    assert_parity(a[s], phi[s], a_ref[s], phi_ref[s], med=TOL_FP64, p99=TOL_FP64, label="plummer fp64")


def test_cube_1m_monopole_cells_at_equal_error_theta_sampled():
    """Monopole cells (Eq. 4 alone) at the full cube size and theta 0.3, the
    opening angle whose error matches quadrupole cells at 0.65 (Fig. 1), in the
    autotuned launch shape."""
    case = Case.workload("cube_1m", 0.3)
    a, phi, _ = case.gpu(qgrav.Options(expansion=qgrav.QG_MONO), autotune=True)
    groups = case.sample_groups(60, seed=17)
    a_ref, phi_ref = case.oracle(use_quad=False, groups=groups)
    s = case.sinks_of(groups)
    assert_parity(a[s], phi[s], a_ref[s], phi_ref[s], label="cube_1m mono theta=0.30")


def test_cube_1m_pipelined_host_evaluation():
    """The one-call host entry point at the full cube size, in the autotuned
    launch shape, by both routes: bit for bit the separate calls, and the
    oracle on a sample."""
    case = Case.workload("cube_1m")
    ctx = qgrav.Context(0)
    a_ref, phi_ref, _ = case.gpu(ctx=ctx, autotune=True)
    for pinned in (False, True):
        a, phi = _evaluate_host(case, ctx, pinned=pinned)
        assert ctx.qg_get_stats()["eval_in_place"] == (1 if pinned else 0)
        assert np.array_equal(a, a_ref) and np.array_equal(phi, phi_ref)
    ctx.close()
    groups = case.sample_groups(80, seed=23)
    a_o, phi_o = case.oracle(groups=groups)
    s = case.sinks_of(groups)
    assert_parity(a[s], phi[s], a_o[s], phi_o[s], label="cube_1m pipelined")
