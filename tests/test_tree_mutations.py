"""Plant plausible mistakes in copies of the host tree builder's source
(csrc/qg_tree.cpp) and check that the pins in test_tree.py reject every one
of them (on the CPU).  The builder makes the lists that the FP64 oracle and
the CUDA path both consume, so a mistake in it would never show as a parity
failure: these pins are what hold it to the method (Sec. 3.4)."""
import ctypes
import os
import subprocess

import pytest

from paper_1812_07313_gb300 import _native, workloads
from paper_1812_07313_gb300 import tree as qtree
from tests import test_tree as pins

SRC = os.path.join(_native.CSRC, "qg_tree.cpp")

# (description, text in the builder's source, replacement)
MUTANTS = [
    ("opens more cells than theta asks", "if (t->side[k] * t->side[k] < theta2 * d2) open = false;",
     "if (t->side[k] * t->side[k] < 0.5 * theta2 * d2) open = false;"),
    ("accepts cells theta rejects", "if (t->side[k] * t->side[k] < theta2 * d2) open = false;",
     "if (t->side[k] * t->side[k] < 2.0 * theta2 * d2) open = false;"),
    ("distance from the cube centre, not the centre of mass", "const double c = t->com[3 * k + d];",
     "const double c = t->centre[3 * k + d];"),
    ("groups one particle short of n_crit", "if (nd.end - nd.begin <= n_crit || nd.first_child < 0) {",
     "if (nd.end - nd.begin < n_crit || nd.first_child < 0) {"),
    ("leaves split at leaf_max particles", "if (cnt <= leaf_max || nd.level >= kMaxLevel) continue;",
     "if (cnt < leaf_max || nd.level >= kMaxLevel) continue;"),
    ("an opened leaf loses its last particle", "for (int64_t i = nd.begin; i < nd.end; i++) pb.push_back((int32_t)i);",
     "for (int64_t i = nd.begin; i + 1 < nd.end; i++) pb.push_back((int32_t)i);"),
]


def _variant(source, tmp_path):
    src = tmp_path / "qg_tree_mutant.cpp"
    src.write_text(source)
    lib = tmp_path / "libqg_tree_mutant.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-I" + _native.INCLUDE, str(src), "-o", str(lib)])
    return qtree._bind(ctypes.CDLL(str(lib)))


def _sphere():
    ps = workloads.small_set("sphere", 4096, 1, 1e-2)
    return ps, qtree.Tree(ps.x, ps.m, ps.sys_off, 8, 64)


PINS = [
    pins.test_groups_partition_and_respect_n_crit,
    pins.test_leaves_split_at_leaf_max_and_groups_are_maximal,
    pins.test_leaves_and_ranges,
    pins.test_moments_match_eq2_direct_sum,
    lambda s: pins.test_lists_cover_all_mass_exactly_once(s, 0.5),
    pins.test_accepted_cells_satisfy_opening_test,
    pins.test_cells_are_opened_only_when_the_test_requires_it,
    lambda s: pins.test_lattice_groups_and_leaves_in_closed_form(),
]


def _caught(monkeypatch, lib):
    monkeypatch.setattr(qtree, "_lib", lib)
    sphere = _sphere()
    caught = 0
    for pin in PINS:
        try:
            pin(sphere)
        except AssertionError:
            caught += 1
    return caught


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(desc, old, new, tmp_path, monkeypatch):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, desc
    assert _caught(monkeypatch, _variant(text.replace(old, new), tmp_path)) > 0, "no pin rejects: " + desc


def test_the_unmutated_source_passes_every_pin(tmp_path, monkeypatch):
    with open(SRC) as f:
        text = f.read()
    assert _caught(monkeypatch, _variant(text, tmp_path)) == 0
