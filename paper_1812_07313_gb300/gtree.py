"""Python binding of the GPU tree build and group walk (``include/qg_gtree.h``).

Argument marshalling only: the build, moments, groups and walk run in
``libqgrav.so``.  Inputs are torch CUDA tensors; ``GpuTree.host(...)`` copies
a result array to numpy (for tests and inspection).

    python -m paper_1812_07313_gb300.gtree --workload plummer_4m --repeat 3

builds and walks a named workload's tree and prints the device times.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import qgrav

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double

SIGNATURES = {
    "qg_gtree_create": ([ctypes.POINTER(_vp), _int], _int),
    "qg_gtree_destroy": ([_vp], None),
    "qg_gtree_build": ([_vp, _i64, _vp, _vp, _i64, _vp, _int, _int, _vp], _int),
    "qg_gtree_walk": ([_vp, _dbl, _vp], _int),
    "qg_gtree_sizes": ([_vp, _vp, _vp, _vp, _vp, _vp], _int),
    "qg_gtree_arrays": ([_vp] + [_vp] * 14, _int),
    "qg_gtree_attach": ([_vp, _vp, _dbl, _vp], _int),
    "qg_gtree_attach_move": ([_vp, _vp, _dbl, _vp], _int),
    "qg_gtree_unsort": ([_vp, _vp, _vp, _int, _vp], _int),
    "qg_gtree_timing": ([_vp, _vp, _vp], _int),
}

_bound = False


def _lib():
    global _bound
    L = qgrav.lib()
    if not _bound:
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        L.cudaMemcpy.argtypes = [_vp, _vp, ctypes.c_size_t, _int]
        L.cudaMemcpy.restype = _int
        _bound = True
    return L


ARRAYS = ("perm", "xs", "ms", "node_range", "node_level", "cell_com", "cell_m", "cell_q", "cell_side",
          "group_off", "plist_off", "plist_idx", "clist_off", "clist_idx")


class GpuTree:
    """Oct-tree, moments, groups and lists built on the GPU."""

    def __init__(self, device=0):
        self._L = _lib()
        self._h = _vp()
        st = self._L.qg_gtree_create(ctypes.byref(self._h), int(device))
        if st != qgrav.QG_OK:
            raise qgrav.QGError(st, "qg_gtree_create(device=%d) failed" % device)
        self.device = device

    def _ok(self, st, what):
        if st != qgrav.QG_OK:
            raise qgrav.QGError(st, what)

    def close(self):
        if self._h:
            self._L.qg_gtree_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, x, m, sys_off=None, leaf_max=8, n_crit=64, stream=None):
        """x: CUDA float64 [n,3], m: CUDA float64 [n]; sys_off: host int64 [nsys+1]."""
        qgrav._check_dev(x, "float64"), qgrav._check_dev(m, "float64")
        n = m.numel()
        so = np.array([0, n], dtype=np.int64) if sys_off is None else np.ascontiguousarray(sys_off, np.int64)
        self._ok(self._L.qg_gtree_build(self._h, n, x.data_ptr(), m.data_ptr(), len(so) - 1, so.ctypes.data,
                                        int(leaf_max), int(n_crit), stream), "qg_gtree_build")

    def walk(self, theta, stream=None):
        self._ok(self._L.qg_gtree_walk(self._h, float(theta), stream), "qg_gtree_walk")

    def sizes(self):
        v = [ctypes.c_int64() for _ in range(5)]
        self._ok(self._L.qg_gtree_sizes(self._h, *[ctypes.addressof(x) for x in v]), "qg_gtree_sizes")
        return dict(zip(("n", "nnodes", "ngroups", "n_plist", "n_clist"), [x.value for x in v]))

    def pointers(self):
        ptrs = [_vp() for _ in ARRAYS]
        self._ok(self._L.qg_gtree_arrays(self._h, *[ctypes.addressof(p) for p in ptrs]), "qg_gtree_arrays")
        return {k: p.value for k, p in zip(ARRAYS, ptrs)}

    def host(self, name, start=None, stop=None):
        """A device array of the last build / walk, copied to numpy (rows
        [start, stop) of it when given)."""
        sz = self.sizes()
        n, nn, G = sz["n"], sz["nnodes"], sz["ngroups"]
        shapes = {"perm": ((n,), np.int64), "xs": ((n, 3), np.float64), "ms": ((n,), np.float64),
                  "node_range": ((nn, 2), np.int64), "node_level": ((nn,), np.int32),
                  "cell_com": ((nn, 3), np.float64), "cell_m": ((nn,), np.float64),
                  "cell_q": ((nn, 6), np.float64), "cell_side": ((nn,), np.float64),
                  "group_off": ((G + 1,), np.int64), "plist_off": ((G + 1,), np.int64),
                  "clist_off": ((G + 1,), np.int64), "plist_idx": ((sz["n_plist"],), np.int32),
                  "clist_idx": ((sz["n_clist"],), np.int32)}
        shape, dt = shapes[name]
        rows = shape[0]
        lo = 0 if start is None else max(0, min(int(start), rows))
        hi = rows if stop is None else max(lo, min(int(stop), rows))
        out = np.empty((hi - lo,) + shape[1:], dtype=dt)
        row_bytes = int(np.prod(shape[1:], dtype=np.int64)) * np.dtype(dt).itemsize
        ptr = self.pointers()[name]
        if out.nbytes:
            if not ptr:
                raise qgrav.QGError(qgrav.QG_ERR_STATE, "%s is not available" % name)
            rc = self._L.cudaMemcpy(out.ctypes.data, ptr + lo * row_bytes, out.nbytes, 2)  # device -> host
            if rc != 0:
                raise qgrav.QGError(qgrav.QG_ERR_CUDA, "cudaMemcpy of %s failed (%d)" % (name, rc))
        return out

    def attach(self, ctx, eps2_all, stream=None):
        """Set a qgrav.Context's sinks, sources and cells from this tree (device to device)."""
        self._ok(self._L.qg_gtree_attach(self._h, ctx._h, float(eps2_all), stream), "qg_gtree_attach")
        sz = self.sizes()
        ctx.n, ctx.G = sz["n"], sz["ngroups"]

    def attach_move(self, ctx, eps2_all, stream=None):
        """As attach, with the lists moved into the context instead of copied:
        the tree holds no lists until its next walk."""
        self._ok(self._L.qg_gtree_attach_move(self._h, ctx._h, float(eps2_all), stream), "qg_gtree_attach_move")
        sz = self.sizes()
        ctx.n, ctx.G = sz["n"], sz["ngroups"]

    def unsort(self, inp, out, k, stream=None):
        """out[perm[i]] = inp[i] (k values per particle; CUDA float64 tensors)."""
        qgrav._check_dev(inp, "float64"), qgrav._check_dev(out, "float64")
        self._ok(self._L.qg_gtree_unsort(self._h, inp.data_ptr(), out.data_ptr(), int(k), stream),
                 "qg_gtree_unsort")

    def timing(self):
        b, w = ctypes.c_float(), ctypes.c_float()
        self._ok(self._L.qg_gtree_timing(self._h, ctypes.addressof(b), ctypes.addressof(w)), "qg_gtree_timing")
        return b.value, w.value


def main():
    import argparse
    import json

    import torch

    from . import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="plummer_4m")
    ap.add_argument("--theta", type=float, default=None)
    ap.add_argument("--repeat", type=int, default=3)
    args = ap.parse_args()
    wl = workloads.WORKLOADS[args.workload]
    ps = wl.particles()
    x, m = torch.as_tensor(ps.x).cuda(), torch.as_tensor(ps.m).cuda()
    t = GpuTree(0)
    theta = wl.theta if args.theta is None else args.theta
    for k in range(args.repeat):
        t.build(x, m, ps.sys_off, wl.leaf_max, wl.n_crit)
        t.walk(theta)
        b, w = t.timing()
        print(json.dumps({"workload": args.workload, "pass": k, "build_ms": b, "walk_ms": w, **t.sizes()}), flush=True)
    t.close()


if __name__ == "__main__":
    main()
