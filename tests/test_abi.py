"""The C-ABI library builds, loads and exports every symbol its header declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1812_07313_gb300 import _native, qgrav

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qgt?_[a-z0-9_]+)\s*\(", text)))


def test_cuda_library_exports_every_declared_symbol():
    L = qgrav.lib()
    names = _declared("qgrav.h")
    assert "qg_run" in names and len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(qgrav.SIGNATURES), set(names) ^ set(qgrav.SIGNATURES)


def test_gpu_tree_symbols_are_exported_and_bound():
    from paper_1812_07313_gb300 import gtree
    L = qgrav.lib()
    names = _declared("qg_gtree.h")
    assert "qg_gtree_build" in names and "qg_gtree_walk" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(gtree.SIGNATURES)


def test_integrator_symbols_are_exported_and_bound():
    from paper_1812_07313_gb300 import sim
    L = qgrav.lib()
    names = _declared("qg_sim.h")
    assert "qg_sim_step" in names and "qg_sim_energy" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(sim.SIGNATURES)


def test_tree_library_exports_every_declared_symbol():
    L = ctypes.CDLL(_native.build_tree())
    for n in _declared("qg_tree.h"):
        assert hasattr(L, n), n


def test_library_is_built_for_sm_103a_only():
    assert _native.CUDA_ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(qgrav.lib()._name)


def test_invalid_device_is_an_error_not_a_crash():
    h = ctypes.c_void_p()
    st = qgrav.lib().qg_create(ctypes.byref(h), 4096, None)
    assert st == qgrav.QG_ERR_ARG and not h.value


def test_null_arguments_are_errors():
    L = qgrav.lib()
    assert L.qg_create(None, 0, None) == qgrav.QG_ERR_ARG
    assert L.qg_run(None, None) == qgrav.QG_ERR_ARG
    assert L.qg_get_forces(None, None, None) == qgrav.QG_ERR_ARG
    assert L.qg_direct_dev(0, -1, None, 0.0, 0, None, None, None, None, None) == qgrav.QG_ERR_ARG
