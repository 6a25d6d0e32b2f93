"""Python binding of the host oct-tree / group walk (``include/qg_tree.h``).

The tree and its lists are the *input* of the force hot path: ``Tree`` sorts
the particles along a Morton curve per system, builds the oct-tree with cell
moments (Eq. 2), forms the sink groups of the modified tree algorithm
(Sec. 3.4) and ``Tree.walk(theta)`` emits the shared interaction lists.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native

_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_i64 = _P(ctypes.c_int64)
_i32 = _P(ctypes.c_int32)
_lib = None


def _bind(lib):
    """Attach the qgt_* signatures to a loaded tree library."""
    lib.qgt_build.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_int64, _i64, ctypes.c_int,
                              ctypes.c_int, _P(ctypes.c_void_p)]
    lib.qgt_build.restype = ctypes.c_int
    lib.qgt_free.argtypes = [ctypes.c_void_p]
    lib.qgt_free.restype = None
    lib.qgt_sizes.argtypes = [ctypes.c_void_p, _i64, _i64, _i64]
    lib.qgt_sizes.restype = ctypes.c_int
    lib.qgt_perm.argtypes = [ctypes.c_void_p]
    lib.qgt_perm.restype = _i64
    lib.qgt_group_off.argtypes = [ctypes.c_void_p]
    lib.qgt_group_off.restype = _i64
    lib.qgt_nodes.argtypes = [ctypes.c_void_p, _P(_d), _P(_d), _P(_d), _P(_d), _P(_d),
                              _P(_i64), _P(_i32)]
    lib.qgt_nodes.restype = ctypes.c_int
    lib.qgt_walk.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
    lib.qgt_walk.restype = ctypes.c_int
    lib.qgt_lists.argtypes = [ctypes.c_void_p, _P(_i64), _P(_i32), _i64, _P(_i64), _P(_i32), _i64]
    lib.qgt_lists.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(_native.load(_native.build_tree()))
    return _lib


def _copy(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


@dataclass
class Lists:
    """Shared interaction lists of one walk (CSR over groups)."""
    theta: float
    plist_off: np.ndarray   # [G+1] int64
    plist_idx: np.ndarray   # int32, index into the sorted particles
    clist_off: np.ndarray   # [G+1] int64
    clist_idx: np.ndarray   # int32, index into the cells

    def interactions(self, group_off):
        ni = np.diff(group_off)
        ipp = int(np.sum(ni * np.diff(self.plist_off)))
        ipc = int(np.sum(ni * np.diff(self.clist_off)))
        return ipp, ipc


class Tree:
    """Oct-tree(s) of a particle set; particles are stored in sorted order.

    Attributes (numpy, owned copies):
      perm       sorted index -> input index
      x, m       sorted positions [n,3] and masses [n]
      group_off  [G+1] sink groups (contiguous sorted ranges)
      sink_sys   [n] system of each sorted particle
      cell_com, cell_m, cell_q, cell_side, cell_centre, cell_range, cell_sys
    """

    def __init__(self, x, m, sys_off=None, leaf_max=8, n_crit=64):
        lib = _load()
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        m = np.ascontiguousarray(m, dtype=np.float64).reshape(-1)
        n = len(x)
        if sys_off is None:
            sys_off = np.array([0, n], dtype=np.int64)
        sys_off = np.ascontiguousarray(sys_off, dtype=np.int64)
        h = ctypes.c_void_p()
        rc = lib.qgt_build(n, x.ctypes.data_as(_d), m.ctypes.data_as(_d), len(sys_off) - 1,
                           sys_off.ctypes.data_as(_i64), int(leaf_max), int(n_crit), ctypes.byref(h))
        if rc != 0:
            raise ValueError("qgt_build failed (%d)" % rc)
        self._h = h
        self._L = lib  # the library that owns the handle: walks and frees go through it
        self.leaf_max, self.n_crit = leaf_max, n_crit
        nn, nnodes, ng = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib.qgt_sizes(h, ctypes.byref(nn), ctypes.byref(nnodes), ctypes.byref(ng))
        self.n, self.nnodes, self.ngroups = nn.value, nnodes.value, ng.value
        self.perm = _copy(lib.qgt_perm(h), n, np.int64)
        self.group_off = _copy(lib.qgt_group_off(h), self.ngroups + 1, np.int64)
        self.x = x[self.perm]
        self.m = m[self.perm]
        self.sys_off = sys_off
        sink_sys = np.zeros(n, dtype=np.int64)
        for s in range(len(sys_off) - 1):
            sink_sys[sys_off[s]:sys_off[s + 1]] = s
        self.sink_sys = sink_sys  # systems are contiguous and sorting stays inside them
        p = [_d() for _ in range(5)]
        pr, ps = _i64(), _i32()
        lib.qgt_nodes(h, *[ctypes.byref(v) for v in p], ctypes.byref(pr), ctypes.byref(ps))
        k = self.nnodes
        self.cell_com = _copy(p[0], 3 * k, np.float64).reshape(k, 3)
        self.cell_m = _copy(p[1], k, np.float64)
        self.cell_q = _copy(p[2], 6 * k, np.float64).reshape(k, 6)
        self.cell_centre = _copy(p[3], 3 * k, np.float64).reshape(k, 3)
        self.cell_side = _copy(p[4], k, np.float64)
        self.cell_range = _copy(pr, 2 * k, np.int64).reshape(k, 2)
        self.cell_sys = _copy(ps, k, np.int32)

    def walk(self, theta, nthreads=0) -> Lists:
        lib = self._L
        rc = lib.qgt_walk(self._h, float(theta), int(nthreads))
        if rc != 0:
            raise ValueError("qgt_walk failed (%d)" % rc)
        po, pi, co, ci = _i64(), _i32(), _i64(), _i32()
        npt, nct = ctypes.c_int64(), ctypes.c_int64()
        lib.qgt_lists(self._h, ctypes.byref(po), ctypes.byref(pi), ctypes.byref(npt),
                      ctypes.byref(co), ctypes.byref(ci), ctypes.byref(nct))
        G = self.ngroups
        return Lists(theta=float(theta),
                     plist_off=_copy(po, G + 1, np.int64), plist_idx=_copy(pi, npt.value, np.int32),
                     clist_off=_copy(co, G + 1, np.int64), clist_idx=_copy(ci, nct.value, np.int32))

    def __del__(self):
        h = getattr(self, "_h", None)
        lib = getattr(self, "_L", None)
        if h is not None and lib is not None:
            lib.qgt_free(h)
            self._h = None
