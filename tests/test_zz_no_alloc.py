"""qg_forces_noalloc: the force evaluation for callers that cannot allocate
device memory (a host code whose memory pool owns every byte, or a step loop
that may not call cudaMalloc / cudaFree once running).  Its only scratch, the
step's work queue, is a fixed array inside the library.

Checked through the C-ABI against the context entry point (qg_set_* +
qg_run + qg_get_forces) on the same inputs, on two calls in a row (the second
call reuses the scratch the first one left behind)."""
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


@pytest.mark.parametrize("expansion", [qgrav.QG_QUAD, qgrav.QG_MONO])
def test_noalloc_matches_context_entry_point_twice(expansion):
    torch = _need_gpu()
    ps = workloads.small_set("plummer", 20000, 17, 0.01)
    case = Case(ps, 0.5, leaf_max=8, n_crit=64)
    a_ref, phi_ref, _ = case.gpu(qgrav.Options(expansion=expansion))
    inp = _device_inputs(torch, case)
    n = case.tree.n
    for call in range(2):
        a = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        phi = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        qgrav.qg_forces_noalloc(a=a, phi=phi, eps2_all=case.eps2_all, expansion=expansion, **inp)
        torch.cuda.synchronize()
        a_h, phi_h = a.cpu().numpy(), phi.cpu().numpy()
        ea, ep = rel_err(a_h, a_ref), rel_err(phi_h, phi_ref)
        assert np.all(np.isfinite(a_h)) and np.all(np.isfinite(phi_h)), call
        assert np.median(ea) <= TOL_MEDIAN and np.percentile(ea, 99) <= TOL_P99, (call, np.median(ea))
        assert np.median(ep) <= TOL_MEDIAN and np.percentile(ep, 99) <= TOL_P99, (call, np.median(ep))


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
    # and a good call afterwards still works
    qgrav.qg_forces_noalloc(a=a, phi=phi, eps2_all=case.eps2_all, **inp)
    torch.cuda.synchronize()
    assert torch.isfinite(a).all() and torch.isfinite(phi).all()
