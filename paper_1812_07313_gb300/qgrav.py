"""Python binding of the ``qg_*`` C-ABI (``include/qgrav.h``).

Argument marshalling only: every step of the force evaluation runs in the
CUDA library ``_build/libqgrav.so``.  There is no Python or CPU fallback: if
the library cannot be built or loaded, importing a function raises.

Host inputs are numpy arrays; device inputs are torch CUDA tensors (their
storage is passed by pointer to the ``*_dev`` entry points).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native

QG_OK, QG_ERR_ARG, QG_ERR_CUDA, QG_ERR_NOMEM, QG_ERR_STATE, QG_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
QG_ERR_SIZE = -6
QG_NOALLOC_MAX_GROUPS = 1 << 20
QG_FP32_CENTRED, QG_FP32_RAW, QG_FP64 = 0, 1, 2
QG_QUAD, QG_MONO = 0, 1
QG_ARITH_DEFAULT, QG_ARITH_SCALAR, QG_ARITH_PAIRED, QG_ARITH_ENTRY_PAIRED = 0, 1, 2, 3

_STATUS = {0: "QG_OK", -1: "QG_ERR_ARG", -2: "QG_ERR_CUDA", -3: "QG_ERR_NOMEM", -4: "QG_ERR_STATE",
           -5: "QG_ERR_TIMEOUT", -6: "QG_ERR_SIZE"}

_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double

# every symbol include/qgrav.h declares, with its argument types
SIGNATURES = {
    "qg_create": ([_P(_vp), _int, _vp], _int),
    "qg_destroy": ([_vp], None),
    "qg_set_options": ([_vp, _vp], _int),
    "qg_set_sinks": ([_vp, _i64, _vp, _vp, _dbl, _i64, _vp], _int),
    "qg_set_sources": ([_vp, _i64, _vp, _vp, _vp, _vp], _int),
    "qg_set_cells": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp], _int),
    "qg_set_sinks_dev": ([_vp, _i64, _vp, _vp, _dbl, _i64, _vp, _vp], _int),
    "qg_set_sources_dev": ([_vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp], _int),
    "qg_set_cells_dev": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp], _int),
    "qg_run": ([_vp, _vp], _int),
    "qg_get_forces": ([_vp, _vp, _vp], _int),
    "qg_get_forces_dev": ([_vp, _vp, _vp, _vp], _int),
    "qg_get_stats": ([_vp, _vp], _int),
    "qg_evaluate_host": ([_vp, _i64, _vp, _vp, _dbl, _i64, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp,
                          _vp, _vp, _vp], _int),
    "qg_last_error": ([_vp], ctypes.c_char_p),
    "qg_last_timing": ([_vp, _vp, _vp], _int),
    "qg_autotune": ([_vp, _vp, _int, _vp, _vp], _int),
    "qg_direct_dev": ([_int, _i64, _vp, _dbl, _i64, _vp, _vp, _vp, _vp, _vp], _int),
    "qg_round_f32_host": ([_i64, _vp, _vp], _int),
    "qg_round_f32_dev": ([_i64, _vp, _vp, _vp, _vp], _int),
    "qg_forces_noalloc": ([_int, _i64, _vp, _vp, _dbl, _i64, _vp, _i64, _vp, _vp, _vp, _vp, _i64,
                           _i64, _vp, _vp, _vp, _vp, _vp, _i64, _int, _vp, _vp, _vp], _int),
}


class qg_options(ctypes.Structure):
    _fields_ = [("precision", _int), ("expansion", _int), ("tile_j", _int),
                ("warps_per_group", _int), ("sinks_per_thread", _int), ("flush_j", _int), ("arith", _int),
                ("split_j", _int), ("sinks_adaptive", _int)]


class qg_stats(ctypes.Structure):
    _fields_ = [("n_sinks", _i64), ("n_groups", _i64), ("n_sources", _i64), ("n_cells", _i64),
                ("n_plist", _i64), ("n_clist", _i64), ("i_pp", _i64), ("i_pc", _i64),
                ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("sinks_per_thread", ctypes.c_int32), ("tile_j", ctypes.c_int32),
                ("warps_per_group", ctypes.c_int32), ("flush_j", ctypes.c_int32),
                ("paired", ctypes.c_int32), ("eval_in_place", ctypes.c_int32), ("n_items", _i64),
                ("n_split", _i64), ("sinks_adaptive", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None


def lib(build: bool = True):
    """Load (building first if needed) the CUDA library and bind every symbol."""
    global _lib
    if _lib is None:
        path = _native.build_cuda() if build else _native.CUDA_LIB
        L = _native.load(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


class QGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


def _host(a, dtype, shape=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _hp(a):
    return None if a is None else a.ctypes.data


def _dp(t):
    return None if t is None else t.data_ptr()


def _check_dev(t, dtype_name):
    if t is None:
        return
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("device entry points take CUDA tensors")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError("expected torch.%s, got %s" % (dtype_name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")


@dataclass
class Options:
    precision: int = QG_FP32_CENTRED
    expansion: int = QG_QUAD
    tile_j: int = 0
    warps_per_group: int = 0
    sinks_per_thread: int = 0
    flush_j: int = 0
    arith: int = QG_ARITH_DEFAULT
    split_j: int = 0
    sinks_adaptive: int = 0

    def c(self):
        return qg_options(self.precision, self.expansion, self.tile_j, self.warps_per_group,
                          self.sinks_per_thread, self.flush_j, self.arith, self.split_j, self.sinks_adaptive)


class Context:
    """One ``qg_ctx``: inputs resident on one GPU, one force evaluation per run()."""

    def __init__(self, device: int = 0, options: Options | None = None):
        self._L = lib()
        self._h = _vp()
        o = (options or Options()).c()
        st = self._L.qg_create(ctypes.byref(self._h), int(device), ctypes.addressof(o))
        if st != QG_OK:
            raise QGError(st, "qg_create(device=%d) failed" % device)
        self.device = device
        self.n = 0
        self.G = -1

    def _ok(self, st, what):
        if st != QG_OK:
            raise QGError(st, "%s: %s" % (what, self._L.qg_last_error(self._h).decode()))

    def close(self):
        if self._h:
            self._L.qg_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, options: Options):
        o = options.c()
        self._ok(self._L.qg_set_options(self._h, ctypes.addressof(o)), "qg_set_options")

    # ---- host inputs ------------------------------------------------------
    def qg_set_sinks(self, x, group_off, eps2_all=0.0, eps2=None):
        x = _host(x, np.float64, (-1, 3))
        g = _host(group_off, np.int64)
        e = None if eps2 is None else _host(eps2, np.float32)
        if g.ndim != 1 or len(g) < 1 or (e is not None and len(e) != len(x)):
            raise ValueError("qg_set_sinks: group_off must have ngroups+1 entries, eps2 one per sink")
        self._ok(self._L.qg_set_sinks(self._h, len(x), _hp(x), _hp(e), float(eps2_all), len(g) - 1, _hp(g)),
                 "qg_set_sinks")
        self.n = len(x)
        self.G = len(g) - 1

    def _check_list(self, off, idx, what):
        if len(off) != self.G + 1:
            raise ValueError("%s: list_off has %d entries, the sinks have %d groups" % (what, len(off), self.G))
        if off[-1] != len(idx):
            raise ValueError("%s: list_off[-1] = %d but list_idx has %d entries" % (what, off[-1], len(idx)))

    def qg_set_sources(self, x, m, list_off, list_idx):
        x = _host(x, np.float64, (-1, 3))
        m = _host(m, np.float64)
        o = _host(list_off, np.int64)
        i = _host(list_idx, np.int32)
        self._check_list(o, i, "qg_set_sources")
        if len(x) != len(m):
            raise ValueError("qg_set_sources: x and m differ in length")
        self._ok(self._L.qg_set_sources(self._h, len(m), _hp(x), _hp(m), _hp(o), _hp(i)), "qg_set_sources")

    def qg_set_cells(self, com, m, q, list_off, list_idx):
        com = _host(com, np.float64, (-1, 3))
        m = _host(m, np.float64)
        q = _host(q, np.float64, (-1, 6))
        o = _host(list_off, np.int64)
        i = _host(list_idx, np.int32)
        self._check_list(o, i, "qg_set_cells")
        if not (len(com) == len(m) == len(q)):
            raise ValueError("qg_set_cells: com, m and q differ in length")
        self._ok(self._L.qg_set_cells(self._h, len(m), _hp(com), _hp(m), _hp(q), _hp(o), _hp(i)),
                 "qg_set_cells")

    # ---- device inputs (torch CUDA tensors) --------------------------------
    def qg_set_sinks_dev(self, x, group_off, eps2_all=0.0, eps2=None, stream=None):
        _check_dev(x, "float64"), _check_dev(group_off, "int64"), _check_dev(eps2, "float32")
        self._ok(self._L.qg_set_sinks_dev(self._h, x.numel() // 3, _dp(x), _dp(eps2), float(eps2_all),
                                          group_off.numel() - 1, _dp(group_off), stream),
                 "qg_set_sinks_dev")
        self.n = x.numel() // 3
        self.G = group_off.numel() - 1

    def qg_set_sources_dev(self, x, m, list_off, list_idx, stream=None):
        _check_dev(x, "float64"), _check_dev(m, "float64"), _check_dev(list_off, "int64")
        _check_dev(list_idx, "int32")
        if list_off.numel() != self.G + 1:
            raise ValueError("qg_set_sources_dev: list_off must have ngroups+1 entries")
        self._ok(self._L.qg_set_sources_dev(self._h, m.numel(), _dp(x), _dp(m), _dp(list_off), _dp(list_idx),
                                            list_idx.numel(), stream), "qg_set_sources_dev")

    def qg_set_cells_dev(self, com, m, q, list_off, list_idx, stream=None):
        for t, d in ((com, "float64"), (m, "float64"), (q, "float64"), (list_off, "int64"), (list_idx, "int32")):
            _check_dev(t, d)
        if list_off.numel() != self.G + 1:
            raise ValueError("qg_set_cells_dev: list_off must have ngroups+1 entries")
        self._ok(self._L.qg_set_cells_dev(self._h, m.numel(), _dp(com), _dp(m), _dp(q), _dp(list_off),
                                          _dp(list_idx), list_idx.numel(), stream), "qg_set_cells_dev")

    # ---- run and results ---------------------------------------------------
    def qg_run(self, stream=None):
        """stream: a raw cudaStream_t (int), e.g. torch.cuda.current_stream().cuda_stream."""
        self._ok(self._L.qg_run(self._h, stream), "qg_run")

    def qg_get_forces(self, a=None, phi=None):
        if a is None:
            a = np.empty((self.n, 3))
        if phi is None:
            phi = np.empty(self.n)
        assert a.flags.c_contiguous and a.dtype == np.float64 and a.size == 3 * self.n
        assert phi.flags.c_contiguous and phi.dtype == np.float64 and phi.size == self.n
        self._ok(self._L.qg_get_forces(self._h, _hp(a), _hp(phi)), "qg_get_forces")
        return a, phi

    def qg_evaluate_host(self, x, group_off, eps2_all, eps2, src_x, src_m, plist_off, plist_idx, cell_com, cell_m,
                         cell_q, clist_off, clist_idx, a=None, phi=None):
        """One evaluation from host arrays (the inputs of the three qg_set_*
        calls); returns (a, phi).  Pass the same array as x and src_x to have
        it copied once; a / phi may be preallocated outputs.  With the lists
        and a / phi in page-locked memory the kernel reads the lists and
        writes the results in place (qg_get_stats()["eval_in_place"])."""
        x = _host(x, np.float64, (-1, 3))
        g = _host(group_off, np.int64)
        e = None if eps2 is None else _host(eps2, np.float32)
        sx = _host(src_x, np.float64, (-1, 3))
        sm = _host(src_m, np.float64)
        po, pi = _host(plist_off, np.int64), _host(plist_idx, np.int32)
        com, cm, cq = _host(cell_com, np.float64, (-1, 3)), _host(cell_m, np.float64), _host(cell_q, np.float64, (-1, 6))
        co, ci = _host(clist_off, np.int64), _host(clist_idx, np.int32)
        G = len(g) - 1
        if g.ndim != 1 or G < 0 or (e is not None and len(e) != len(x)):
            raise ValueError("qg_evaluate_host: group_off must have ngroups+1 entries, eps2 one per sink")
        for off, idx, what in ((po, pi, "particle"), (co, ci, "cell")):
            if len(off) != G + 1 or off[-1] != len(idx):
                raise ValueError("qg_evaluate_host: %s list offsets do not match the groups or the list" % what)
        if len(sx) != len(sm) or not (len(com) == len(cm) == len(cq)):
            raise ValueError("qg_evaluate_host: source or cell arrays differ in length")
        n = len(x)
        a = np.empty((n, 3)) if a is None else a
        phi = np.empty(n) if phi is None else phi
        if a.shape != (n, 3) or phi.shape != (n,) or a.dtype != np.float64 or phi.dtype != np.float64 \
                or not (a.flags.c_contiguous and phi.flags.c_contiguous):
            raise ValueError("qg_evaluate_host: a must be float64 [n,3] and phi float64 [n], contiguous")
        self._ok(self._L.qg_evaluate_host(self._h, n, _hp(x), _hp(e), float(eps2_all), G, _hp(g), len(sm), _hp(sx),
                                          _hp(sm), _hp(po), _hp(pi), len(cm), _hp(com), _hp(cm), _hp(cq), _hp(co),
                                          _hp(ci), _hp(a), _hp(phi)), "qg_evaluate_host")
        self.n, self.G = n, G
        return a, phi

    def qg_get_forces_dev(self, a, phi, stream=None):
        _check_dev(a, "float64"), _check_dev(phi, "float64")
        self._ok(self._L.qg_get_forces_dev(self._h, _dp(a), _dp(phi), stream), "qg_get_forces_dev")

    def qg_autotune(self, stream=None, reps=3):
        """Time every launch shape on the current inputs, keep the fastest.
        Returns (Options chosen, mean force-kernel ms)."""
        o = qg_options()
        ms = ctypes.c_float()
        self._ok(self._L.qg_autotune(self._h, stream, int(reps), ctypes.addressof(o), ctypes.addressof(ms)),
                 "qg_autotune")
        return (Options(o.precision, o.expansion, o.tile_j, o.warps_per_group, o.sinks_per_thread, o.flush_j,
                        o.arith, o.split_j, o.sinks_adaptive), ms.value)

    def qg_last_timing(self):
        """(step_ms, force_ms) of the last run, from events inside its graph."""
        st, fo = ctypes.c_float(), ctypes.c_float()
        self._ok(self._L.qg_last_timing(self._h, ctypes.addressof(st), ctypes.addressof(fo)), "qg_last_timing")
        return st.value, fo.value

    def qg_get_stats(self) -> dict:
        s = qg_stats()
        self._ok(self._L.qg_get_stats(self._h, ctypes.addressof(s)), "qg_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}


def qg_direct_dev(sink_x, src_x, src_m, eps2, a, phi, device=0, stream=None):
    """FP64 direct summation on the GPU (torch CUDA tensors in and out)."""
    for t, d in ((sink_x, "float64"), (src_x, "float64"), (src_m, "float64"), (a, "float64"),
                 (phi, "float64")):
        _check_dev(t, d)
    st = lib().qg_direct_dev(int(device), sink_x.numel() // 3, _dp(sink_x), float(eps2), src_m.numel(),
                             _dp(src_x), _dp(src_m), _dp(a), _dp(phi), stream)
    if st != QG_OK:
        raise QGError(st, "qg_direct_dev failed")


def qg_round_f32_host(x):
    """The kernels' FP64 -> FP32 rounding routine, run on the CPU."""
    x = _host(x, np.float64)
    out = np.empty(x.shape, dtype=np.float32)
    st = lib().qg_round_f32_host(x.size, _hp(x), _hp(out))
    if st != QG_OK:
        raise QGError(st, "qg_round_f32_host failed")
    return out


def qg_round_f32_dev(x, out, out_hw, stream=None):
    """The same routine on the GPU next to the hardware conversion (CUDA tensors)."""
    _check_dev(x, "float64"), _check_dev(out, "float32"), _check_dev(out_hw, "float32")
    st = lib().qg_round_f32_dev(x.numel(), _dp(x), _dp(out), _dp(out_hw), stream)
    if st != QG_OK:
        raise QGError(st, "qg_round_f32_dev failed")


def qg_forces_noalloc(sink_x, group_off, src_x, src_m, plist_off, plist_idx, cell_com, cell_m, cell_q,
                      clist_off, clist_idx, a, phi, eps2_all=0.0, eps2=None, expansion=QG_QUAD, device=0,
                      stream=None):
    """One force evaluation that allocates nothing (torch CUDA tensors in the
    qg_set_*_dev layouts in, a and phi out); its work-queue scratch is a fixed
    array inside the library, for at most QG_NOALLOC_MAX_GROUPS groups."""
    for t, d in ((sink_x, "float64"), (group_off, "int64"), (src_x, "float64"), (src_m, "float64"),
                 (plist_off, "int64"), (plist_idx, "int32"), (cell_com, "float64"), (cell_m, "float64"),
                 (cell_q, "float64"), (clist_off, "int64"), (clist_idx, "int32"), (a, "float64"),
                 (phi, "float64"), (eps2, "float32")):
        _check_dev(t, d)
    G = group_off.numel() - 1
    if plist_off.numel() != G + 1 or clist_off.numel() != G + 1:
        raise ValueError("qg_forces_noalloc: list offsets must have ngroups+1 entries")
    n = sink_x.numel() // 3
    if a.numel() != 3 * n or phi.numel() != n:
        raise ValueError("qg_forces_noalloc: a must be [n,3] and phi [n]")
    st = lib().qg_forces_noalloc(int(device), n, _dp(sink_x), _dp(eps2), float(eps2_all), G, _dp(group_off),
                                 src_m.numel(), _dp(src_x), _dp(src_m), _dp(plist_off), _dp(plist_idx),
                                 plist_idx.numel(), cell_m.numel(), _dp(cell_com), _dp(cell_m), _dp(cell_q),
                                 _dp(clist_off), _dp(clist_idx), clist_idx.numel(), int(expansion), _dp(a),
                                 _dp(phi), stream)
    if st != QG_OK:
        raise QGError(st, "qg_forces_noalloc failed")
