"""Plant plausible mistakes in copies of the oracle leapfrog's source
(oracle/integrate.py) and check that the pins in test_integrate_pins.py reject
every one of them (on the CPU)."""
import importlib.util
import inspect
import sys

import pytest

from oracle import integrate
from tests import test_integrate_pins as pins

PINS = [
    pins.test_circular_orbit_closes_at_second_order,
    pins.test_orbit_follows_the_closed_form_at_quarter_period,
    pins.test_energies_of_the_two_body_state_and_their_conservation,
    pins.test_energies_with_per_particle_softening,
    pins.test_energies_and_momentum_with_unequal_masses,
    pins.test_leapfrog_is_time_reversible,
]

# (description, text in the oracle source, replacement)
MUTANTS = [
    ("first half kick a full kick", "        v = v + a * (0.5 * dt)\n        x = x + v * dt",
     "        v = v + a * dt\n        x = x + v * dt"),
    ("drift by half a step", "x = x + v * dt", "x = x + v * (0.5 * dt)"),
    ("second kick with the old acceleration", "        a, phi = accel(x)\n        v = v + a * (0.5 * dt)",
     "        v = v + a * (0.5 * dt)\n        a, phi = accel(x)"),
    ("drift before the first kick", "        v = v + a * (0.5 * dt)\n        x = x + v * dt",
     "        x = x + v * dt\n        v = v + a * (0.5 * dt)"),
    ("kinetic energy without 1/2", "K = 0.5 * float(", "K = 1.0 * float("),
    ("potential energy without 1/2", "W = 0.5 * float(", "W = 1.0 * float("),
    ("self pair kept in W", "W = 0.5 * float(np.sum(m * (phi + self_term)))", "W = 0.5 * float(np.sum(m * phi))"),
    ("self term m / eps^2", "m[pos] / np.sqrt(e2[pos])", "m[pos] / e2[pos]"),
    ("momentum without the masses", "p = (m[:, None] * v).sum(axis=0)", "p = v.sum(axis=0)"),
]


def _variant(source, tmp_path):
    path = tmp_path / "integrate_mutant.py"
    path.write_text(source)
    spec = importlib.util.spec_from_file_location("integrate_mutant", str(path))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["integrate_mutant"] = mod
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(desc, old, new, tmp_path, monkeypatch):
    src = inspect.getsource(integrate)
    assert src.count(old) == 1, desc
    monkeypatch.setattr(pins, "integrate", _variant(src.replace(old, new), tmp_path))
    caught = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught > 0, "no pin rejects the mutant: " + desc


def test_the_unmutated_source_passes_every_pin(tmp_path, monkeypatch):
    monkeypatch.setattr(pins, "integrate", _variant(inspect.getsource(integrate), tmp_path))
    for pin in PINS:
        pin()
