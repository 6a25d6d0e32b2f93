"""Plant plausible mistakes in copies of the oracle source and check that the
pins in test_oracle_pins.py reject every one of them (on the CPU)."""
import pytest

import oracle
from tests import test_oracle_pins as pins

PINS = [
    pins.test_two_mass_golden_closed_form,
    pins.test_quadrupole_traceless_symmetric_and_rotation,
    pins.test_one_particle_cell_is_point_mass,
    lambda: pins.test_expansion_error_order(True, 3.0),
    lambda: pins.test_expansion_error_order(False, 2.0),
    pins.test_force_is_minus_gradient_of_potential,
    pins.test_softening_and_self_pair,
    pins.test_direct_sum_momentum_conservation,
    pins.test_per_sink_softening_matches_global,
    pins.test_theta_zero_is_direct_summation,
]

# (description, text in the oracle source, replacement)
MUTANTS = [
    ("5 of Eq. 7 -> 4", "(phi_mono + 5.0 * phi_quad)", "(phi_mono + 4.0 * phi_quad)"),
    ("1/2 of Eq. 5 dropped", "dQd / (2.0 * rhat5)", "dQd / (1.0 * rhat5)"),
    ("sign of the Q r term", "- Qd[a] / rhat5", "+ Qd[a] / rhat5"),
    ("Q transposed index", "{ q[1], q[3], q[4] },", "{ q[2], q[3], q[4] },"),
    ("quadrupole potential sign", "*pot -= phi_mono + phi_quad;", "*pot -= phi_mono - phi_quad;"),
    ("trace term of Eq. 2 dropped on q00", "q00 += m[k] * (3.0 * xk * xk - r2);",
     "q00 += m[k] * (3.0 * xk * xk);"),
    ("Eq. 2 without the factor 3", "q01 += m[k] * (3.0 * xk * yk);", "q01 += m[k] * (xk * yk);"),
    ("softening missing in rhat", "double rhat2 = d0 * d0 + d1 * d1 + d2 * d2 + eps2;",
     "double rhat2 = d0 * d0 + d1 * d1 + d2 * d2;"),
    ("rhat^5 as rhat^4", "double rhat5 = rhat2 * rhat2 * rhat;", "double rhat5 = rhat2 * rhat2;"),
    ("wrong d direction", "double d0 = xj[0] - xi[0];", "double d0 = xi[0] - xj[0];"),
    ("centre of mass not mass-weighted", "cx += m[k] * x[3 * k + 0];", "cx += x[3 * k + 0];"),
    ("cell mass not summed", "mass += m[k];", "mass += 0.0 * m[k];"),
    ("trace term of Eq. 2 dropped on q22", "q22 += m[k] * (3.0 * zk * zk - r2);", "q22 += m[k] * (3.0 * zk * zk);"),
    ("Q off-diagonal q12 and q22 swapped", "{ q[2], q[4], q[5] },", "{ q[2], q[5], q[4] },"),
    ("particle potential sign", "*pot -= phi_mono;  ", "*pot += phi_mono;  "),
    ("particle force as m / rhat^2", "double c = phi_mono / rhat2;", "double c = phi_mono / rhat;"),
    ("per-sink softening ignored", "return eps2 ? eps2[i] : eps2_all;", "return eps2_all;"),
    ("cell softening missing", "double rhat2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;",
     "double rhat2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];"),
    ("rhat == 0 pair not skipped",
     "    if (rhat2 == 0.0) return;\n    double rhat = sqrt(rhat2);\n    double phi_mono = mj / rhat;                 /* Eq. 4 */\n    *pot",
     "    double rhat = sqrt(rhat2);\n    double phi_mono = mj / rhat;                 /* Eq. 4 */\n    *pot"),
    ("quadrupole terms in monopole-only mode", "    if (use_quad) {\n        for (int a = 0; a < 3; a++)\n            for (int b",
     "    if (1) {\n        for (int a = 0; a < 3; a++)\n            for (int b"),
    ("particle list loses its last entry", "for (int64_t k = plist_off[g]; k < plist_off[g + 1]; k++) {",
     "for (int64_t k = plist_off[g]; k + 1 < plist_off[g + 1]; k++) {"),
    ("direct sum misses the last source", "for (int64_t j = 0; j < nsrc; j++)", "for (int64_t j = 0; j + 1 < nsrc; j++)"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(desc, old, new, tmp_path):
    src = oracle.source_text()
    assert src.count(old) == 1, desc
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "libmutant.so"))
    caught = 0
    with oracle.use_library(lib):
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                caught += 1
    assert caught > 0, "no pin rejects the mutant: " + desc
