"""qg_forces_noalloc: the force evaluation for callers that cannot allocate
device memory (a host code whose memory pool owns every byte, or a step loop
that may not call cudaMalloc / cudaFree once running).  Its only scratch, the
step's work queue, is a fixed array inside the library.

Checked through the C-ABI against the context entry point (qg_set_* +
qg_run + qg_get_forces) on the same inputs, on two calls in a row (the second
call reuses the scratch the first one left behind), and against the FP64
oracle, on cases that reach each of its code paths: groups larger than one
pass of the CTA's sink slots, per-sink softening and zero softening (the
kernel that skips coincident pairs)."""
import numpy as np
import pytest

from paper_1812_07313_gb300 import qgrav, workloads
from tests.parity_util import Case, TOL_MEDIAN, TOL_P99, rel_err

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qgrav.lib()
    return torch


def _device_inputs(torch, case):
    t, L = case.tree, case.lists
    d = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)
    return dict(sink_x=d(t.x, torch.float64), group_off=d(t.group_off, torch.int64),
                src_x=d(t.x, torch.float64), src_m=d(t.m, torch.float64),
                plist_off=d(L.plist_off, torch.int64), plist_idx=d(L.plist_idx, torch.int32),
                cell_com=d(t.cell_com, torch.float64), cell_m=d(t.cell_m, torch.float64),
                cell_q=d(t.cell_q, torch.float64), clist_off=d(L.clist_off, torch.int64),
                clist_idx=d(L.clist_idx, torch.int32))


def _case(kind):
    """plummer: groups of at most 64 sinks; big: groups of up to 1500 sinks
    (several passes of the 512 sink slots of one CTA); per_sink: a softening
    per sink (device array); zero: no softening at all."""
    if kind == "big":
        return Case(workloads.small_set("cube", 6000, 8, 2e-3), 0.5, leaf_max=8, n_crit=1500)
    case = Case(workloads.small_set("plummer", 20000, 17, 0.0 if kind == "zero" else 0.01), 0.5, leaf_max=8,
                n_crit=64)
    if kind == "per_sink":
        case.eps2 = np.random.default_rng(5).uniform(1e-5, 4e-4, case.tree.n).astype(np.float32)
        case.eps2_all = 0.0
    return case


def _check(a_h, phi_h, a_ref, phi_ref, what):
    ea, ep = rel_err(a_h, a_ref), rel_err(phi_h, phi_ref)
    assert np.all(np.isfinite(a_h)) and np.all(np.isfinite(phi_h)), what
    assert np.median(ea) <= TOL_MEDIAN and np.percentile(ea, 99) <= TOL_P99, (what, np.median(ea))
    assert np.median(ep) <= TOL_MEDIAN and np.percentile(ep, 99) <= TOL_P99, (what, np.median(ep))


@pytest.mark.parametrize("kind", ["plummer", "big", "per_sink", "zero"])
@pytest.mark.parametrize("expansion", [qgrav.QG_QUAD, qgrav.QG_MONO])
def test_noalloc_matches_context_entry_point_twice(expansion, kind):
    torch = _need_gpu()
    case = _case(kind)
    if kind == "big":
        assert np.diff(case.tree.group_off).max() > 512
    a_ctx, phi_ctx, _ = case.gpu(qgrav.Options(expansion=expansion))
    a_or, phi_or = case.oracle(use_quad=expansion == qgrav.QG_QUAD)
    inp = _device_inputs(torch, case)
    eps2 = None if case.eps2 is None else torch.as_tensor(case.eps2).cuda()
    n = case.tree.n
    for call in range(2):
        a = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        phi = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        qgrav.qg_forces_noalloc(a=a, phi=phi, eps2_all=case.eps2_all, eps2=eps2, expansion=expansion, **inp)
        torch.cuda.synchronize()
        a_h, phi_h = a.cpu().numpy(), phi.cpu().numpy()
        _check(a_h, phi_h, a_ctx, phi_ctx, ("context", kind, call))
        _check(a_h, phi_h, a_or, phi_or, ("oracle", kind, call))


def test_noalloc_rejects_too_many_groups_and_bad_indices():
    torch = _need_gpu()
    case = Case(workloads.small_set("sphere", 600, 3, 0.01), 0.5)
    inp = _device_inputs(torch, case)
    n = case.tree.n
    a = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    # more groups than the fixed scratch holds: refused before any GPU work
    L = qgrav.lib()
    st = L.qg_forces_noalloc(0, 0, None, None, 1e-4, qgrav.QG_NOALLOC_MAX_GROUPS + 1, inp["group_off"].data_ptr(),
                             0, None, None, inp["plist_off"].data_ptr(), None, 0, 0, None, None, None,
                             inp["clist_off"].data_ptr(), None, 0, qgrav.QG_QUAD, None, None, None)
    assert st == qgrav.QG_ERR_SIZE
    # an out-of-range list index is caught by the device-side check
    bad = inp["plist_idx"].clone()
    bad[len(bad) // 3] = n + 7
    with pytest.raises(qgrav.QGError) as e:
        qgrav.qg_forces_noalloc(a=a, phi=phi, eps2_all=case.eps2_all, **dict(inp, plist_idx=bad))
    assert e.value.status == qgrav.QG_ERR_ARG
    # input values that are not finite, or beyond 2^100, are refused too
    for name, k in (("sink_x", 5), ("src_m", 3), ("cell_q", 7), ("cell_com", 1)):
        for v in (float("nan"), float("inf"), 2.0 ** 101):
            badv = inp[name].clone()
            badv.view(-1)[k] = v
            with pytest.raises(qgrav.QGError) as e:
                qgrav.qg_forces_noalloc(a=a, phi=phi, eps2_all=case.eps2_all, **dict(inp, **{name: badv}))
            assert e.value.status == qgrav.QG_ERR_ARG, (name, v)
    with pytest.raises(qgrav.QGError) as e:
        qgrav.qg_forces_noalloc(a=a, phi=phi, eps2_all=2.0 ** 101, **inp)
    assert e.value.status == qgrav.QG_ERR_ARG
    # and a good call afterwards still works
    qgrav.qg_forces_noalloc(a=a, phi=phi, eps2_all=case.eps2_all, **inp)
    torch.cuda.synchronize()
    assert torch.isfinite(a).all() and torch.isfinite(phi).all()
