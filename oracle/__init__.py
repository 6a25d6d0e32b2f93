"""FP64 CPU oracle for the monopole + quadrupole group-list force evaluation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_1812_07313_gb300``) never imports it and
shares no code with it.

The arithmetic lives in ``qg_oracle.c`` (plain C, double precision, one sink
and one list entry at a time).  This module only compiles it with gcc and
marshals numpy arrays through ctypes.

Functions and the passages of the paper they follow:
  * ``cell_moments``      -- Eq. 2 (quadrupole tensor about the centre of mass)
  * ``expansion_forces``  -- Eq. 1, Eqs. 4-5 and Eq. 7 (sign as -grad of Eq. 1),
                             over the shared interaction lists of the modified
                             tree algorithm (Sec. 3.4)
  * ``direct_forces``     -- direct summation, the reference of Eq. 8
  * ``relative_error``    -- Eq. 8
  * ``set_threads``       -- optional split of expansion_forces' groups over
                             host threads (for the multi-core CPU baseline)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libqg_oracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)
_i32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.qgo_cell_moments.argtypes = [ctypes.c_int64, _d, _d, _d, _d, _d]
            lib.qgo_cell_moments.restype = ctypes.c_int
            lib.qgo_set_threads.argtypes = [ctypes.c_int]
            lib.qgo_set_threads.restype = None
            lib.qgo_expansion_forces.argtypes = [
                ctypes.c_int64, _i64, _d, _d, ctypes.c_double,
                _d, _d, _i64, _i32,
                _d, _d, _d, _i64, _i32,
                ctypes.c_int, _i64, ctypes.c_int64, _d, _d]
            lib.qgo_expansion_forces.restype = ctypes.c_int
            lib.qgo_direct_forces.argtypes = [
                ctypes.c_int64, _d, _d, ctypes.c_double,
                ctypes.c_int64, _d, _d, _d, _d]
            lib.qgo_direct_forces.restype = ctypes.c_int
            _lib = lib
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of the
    oracle source (the mutation tests plant mistakes in copies of it)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in ("qgo_cell_moments", "qgo_expansion_forces", "qgo_direct_forces"):
            getattr(lib, name).argtypes = getattr(self._saved, name).argtypes
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def compile_variant(src_text, out_path):
    """Compile a (possibly modified) copy of the oracle source to out_path."""
    c = out_path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", c, "-o", out_path, "-lm"])
    return out_path


def source_text():
    with open(_SRC) as f:
        return f.read()


def _ptr(a, typ):
    if a is None:
        return ctypes.cast(None, typ)
    return a.ctypes.data_as(typ)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def cell_moments(x, m):
    """Eq. 2: (mass, com[3], q[6] = q00 q01 q02 q11 q12 q22) of point masses."""
    x = _f64(x, (-1, 3))
    m = _f64(m, (-1,))
    assert len(x) == len(m)
    mass = np.zeros(1)
    com = np.zeros(3)
    q = np.zeros(6)
    rc = _load().qgo_cell_moments(len(m), _ptr(x, _d), _ptr(m, _d), _ptr(mass, _d),
                                  _ptr(com, _d), _ptr(q, _d))
    if rc != 0:
        raise ValueError("qgo_cell_moments: bad arguments")
    return float(mass[0]), com, q


def expansion_forces(group_off, sink_x, src_x, src_m, plist_off, plist_idx,
                     cell_com, cell_m, cell_q, clist_off, clist_idx,
                     eps2_all=0.0, sink_eps2=None, use_quad=True, groups=None):
    """Eq. 1 / Eq. 7 over grouped interaction lists, all in double.

    Returns (a [n,3], phi [n]).  With ``groups`` given, only those groups are
    evaluated and the other sinks' rows are NaN.
    """
    group_off = np.ascontiguousarray(group_off, dtype=np.int64)
    ngroups = len(group_off) - 1
    sink_x = _f64(sink_x, (-1, 3))
    n = len(sink_x)
    src_x = _f64(src_x, (-1, 3))
    src_m = _f64(src_m, (-1,))
    cell_com = _f64(cell_com, (-1, 3))
    cell_m = _f64(cell_m, (-1,))
    cell_q = _f64(cell_q, (-1, 6))
    plist_off = np.ascontiguousarray(plist_off, dtype=np.int64)
    clist_off = np.ascontiguousarray(clist_off, dtype=np.int64)
    plist_idx = np.ascontiguousarray(plist_idx, dtype=np.int32)
    clist_idx = np.ascontiguousarray(clist_idx, dtype=np.int32)
    assert len(plist_off) == ngroups + 1 and len(clist_off) == ngroups + 1
    eps = None if sink_eps2 is None else _f64(sink_eps2, (-1,))
    if eps is not None:
        assert len(eps) == n
    gsel = None if groups is None else np.ascontiguousarray(groups, dtype=np.int64)
    a = np.full((n, 3), np.nan)
    phi = np.full(n, np.nan)
    rc = _load().qgo_expansion_forces(
        ngroups, _ptr(group_off, _i64), _ptr(sink_x, _d), _ptr(eps, _d), float(eps2_all),
        _ptr(src_x, _d), _ptr(src_m, _d), _ptr(plist_off, _i64), _ptr(plist_idx, _i32),
        _ptr(cell_com, _d), _ptr(cell_m, _d), _ptr(cell_q, _d),
        _ptr(clist_off, _i64), _ptr(clist_idx, _i32),
        1 if use_quad else 0, _ptr(gsel, _i64), 0 if gsel is None else len(gsel),
        _ptr(a, _d), _ptr(phi, _d))
    if rc != 0:
        raise ValueError("qgo_expansion_forces: bad arguments")
    return a, phi


def direct_forces(sink_x, src_x, src_m, eps2_all=0.0, sink_eps2=None):
    """Direct summation over every source (Plummer point masses), in double."""
    sink_x = _f64(sink_x, (-1, 3))
    src_x = _f64(src_x, (-1, 3))
    src_m = _f64(src_m, (-1,))
    eps = None if sink_eps2 is None else _f64(sink_eps2, (-1,))
    a = np.zeros((len(sink_x), 3))
    phi = np.zeros(len(sink_x))
    rc = _load().qgo_direct_forces(len(sink_x), _ptr(sink_x, _d), _ptr(eps, _d), float(eps2_all),
                                   len(src_x), _ptr(src_x, _d), _ptr(src_m, _d),
                                   _ptr(a, _d), _ptr(phi, _d))
    if rc != 0:
        raise ValueError("qgo_direct_forces: bad arguments")
    return a, phi


def set_threads(n):
    """Host threads over which expansion_forces splits its groups (1: the
    plain serial oracle).  Each group is still one thread's serial loop, so
    the results are the same for any n."""
    _load().qgo_set_threads(int(n))


def relative_error(a_test, a_ref):
    """Eq. 8: |a_test - a_ref| / |a_ref| per sink."""
    a_test = np.asarray(a_test, dtype=np.float64)
    a_ref = np.asarray(a_ref, dtype=np.float64)
    return np.linalg.norm(a_test - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
