"""Python binding of the GPU leapfrog integrator (``include/qg_sim.h``).

Argument marshalling only: the kicks, drift, tree build, walk, force kernel
and energy sums run in ``libqgrav.so``.  State arrays are copied in from
numpy and out to numpy; ``state_dev()`` gives the device pointers.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import qgrav

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


class qg_sim_params(ctypes.Structure):
    _fields_ = [("theta", _dbl), ("eps2", _dbl), ("n_crit", _int), ("leaf_max", _int), ("expansion", _int),
                ("autotune", _int)]


class qg_sim_times(ctypes.Structure):
    _fields_ = [("build_ms", ctypes.c_float), ("walk_ms", ctypes.c_float), ("force_ms", ctypes.c_float),
                ("integrate_ms", ctypes.c_float), ("wall_ms", _dbl), ("groups", _i64), ("n_plist", _i64),
                ("n_clist", _i64), ("i_pp", _i64), ("i_pc", _i64), ("retunes", _i64),
                ("sinks_per_thread", ctypes.c_int32), ("sinks_adaptive", ctypes.c_int32),
                ("warps_per_group", ctypes.c_int32), ("tile_j", ctypes.c_int32), ("form", ctypes.c_int32),
                ("trial_left", ctypes.c_int32)]


SIGNATURES = {
    "qg_sim_create": ([ctypes.POINTER(_vp), _int, _vp, _vp], _int),
    "qg_sim_destroy": ([_vp], None),
    "qg_sim_set_state": ([_vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp], _int),
    "qg_sim_step": ([_vp, _dbl, _i64, _vp], _int),
    "qg_sim_get_state": ([_vp, _vp, _vp, _vp, _vp], _int),
    "qg_sim_state_dev": ([_vp, _vp, _vp, _vp, _vp, _vp], _int),
    "qg_sim_energy": ([_vp, _vp, _vp, _vp, _vp], _int),
    "qg_sim_last_times": ([_vp, _vp], _int),
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
        _bound = True
    return L


@dataclass
class Params:
    theta: float = 0.5
    eps2: float = 0.0
    n_crit: int = 256
    leaf_max: int = 8
    expansion: int = qgrav.QG_QUAD
    autotune: bool = True

    def c(self):
        return qg_sim_params(float(self.theta), float(self.eps2), int(self.n_crit), int(self.leaf_max),
                             int(self.expansion), 1 if self.autotune else 0)


class Simulation:
    """Kick-drift-kick leapfrog with GPU tree forces; state resident on one GPU."""

    def __init__(self, params: Params, device: int = 0, options: qgrav.Options | None = None):
        self._L = _lib()
        self._h = _vp()
        p = params.c()
        o = None if options is None else options.c()
        st = self._L.qg_sim_create(ctypes.byref(self._h), int(device), ctypes.addressof(p),
                                   None if o is None else ctypes.addressof(o))
        if st != qgrav.QG_OK:
            raise qgrav.QGError(st, "qg_sim_create failed")
        self.params = params
        self.device = device
        self.n = 0

    def _ok(self, st, what):
        if st != qgrav.QG_OK:
            raise qgrav.QGError(st, what)

    def close(self):
        if self._h:
            self._L.qg_sim_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, x, v, m, sys_off=None, stream=None, eps2=None):
        """eps2: optional per-particle squared softening (else params.eps2 for all)."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        n = len(x)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(n, 3)
        m = np.ascontiguousarray(m, dtype=np.float64).reshape(n)
        e = None if eps2 is None else np.ascontiguousarray(eps2, dtype=np.float32).reshape(n)
        so = np.array([0, n], dtype=np.int64) if sys_off is None else np.ascontiguousarray(sys_off, np.int64)
        if so.ndim != 1 or len(so) < 2 or so[0] != 0 or so[-1] != n:
            raise ValueError("sys_off must run from 0 to n")
        self._ok(self._L.qg_sim_set_state(self._h, n, x.ctypes.data, v.ctypes.data, m.ctypes.data,
                                          None if e is None else e.ctypes.data, len(so) - 1, so.ctypes.data, stream),
                 "qg_sim_set_state")
        self.n = n

    def step(self, dt, nsteps=1, stream=None):
        self._ok(self._L.qg_sim_step(self._h, float(dt), int(nsteps), stream), "qg_sim_step")

    def state(self):
        """(x, v, a, phi) copied to numpy, in the caller's particle order."""
        n = self.n
        x, v, a = (np.empty((n, 3)) for _ in range(3))
        phi = np.empty(n)
        self._ok(self._L.qg_sim_get_state(self._h, x.ctypes.data, v.ctypes.data, a.ctypes.data, phi.ctypes.data),
                 "qg_sim_get_state")
        return x, v, a, phi

    def state_dev(self):
        ptrs = [_vp() for _ in range(5)]
        self._ok(self._L.qg_sim_state_dev(self._h, *[ctypes.addressof(p) for p in ptrs]), "qg_sim_state_dev")
        return dict(zip(("x", "v", "a", "phi", "m"), [p.value for p in ptrs]))

    def energy(self, stream=None):
        """(K, W, p[3]) of the current state."""
        k, w = _dbl(), _dbl()
        p = np.zeros(3)
        self._ok(self._L.qg_sim_energy(self._h, ctypes.addressof(k), ctypes.addressof(w), p.ctypes.data, stream),
                 "qg_sim_energy")
        return k.value, w.value, p

    def last_times(self):
        t = qg_sim_times()
        self._ok(self._L.qg_sim_last_times(self._h, ctypes.addressof(t)), "qg_sim_last_times")
        return {f: getattr(t, f) for f, _ in qg_sim_times._fields_}
