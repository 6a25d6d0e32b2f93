"""Pins of the oracle leapfrog (oracle/integrate.py) against what mechanics
fixes: a circular two-body orbit (closed form), second-order convergence,
bounded energy error, time reversibility, and the energies and momentum of
known configurations."""
import math

import numpy as np

import oracle
from oracle import integrate


def _two_body(eps2=0.0):
    # equal masses 1/2 at +-1/2 on x, separation 1, G M = 1: circular orbit
    # with relative speed 1 (each body 1/2), angular frequency 1, period 2 pi
    x = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    v = np.array([[0.0, 0.5, 0.0], [0.0, -0.5, 0.0]])
    m = np.array([0.5, 0.5])
    return x, v, m, (lambda y: oracle.direct_forces(y, y, m, eps2_all=eps2))


def _orbit_error(nsteps):
    x0, v0, m, acc = _two_body()
    x, v, _, _ = integrate.leapfrog_kdk(x0, v0, m, 2 * math.pi / nsteps, nsteps, acc)
    return float(np.abs(x - x0).max()), x, v, m, acc


def test_circular_orbit_closes_at_second_order():
    e1, *_ = _orbit_error(200)
    e2, *_ = _orbit_error(400)
    assert e2 < 5e-4
    assert 3.9 < e1 / e2 < 4.1  # O(dt^2)


def test_orbit_follows_the_closed_form_at_quarter_period():
    x0, v0, m, acc = _two_body()
    n = 800
    x, v, _, _ = integrate.leapfrog_kdk(x0, v0, m, (math.pi / 2) / n, n, acc)
    # after a quarter turn (counter-clockwise): body 0 at (0, 1/2), moving (-1/2, 0)
    assert np.allclose(x[0], [0.0, 0.5, 0.0], atol=1e-5)
    assert np.allclose(v[0], [-0.5, 0.0, 0.0], atol=1e-5)
    assert np.allclose(x[0], -x[1], atol=1e-14)  # centre of mass stays at the origin


def test_energies_of_the_two_body_state_and_their_conservation():
    for eps2 in (0.0, 0.01):
        x0, v0, m, acc = _two_body(eps2)
        a, phi = acc(x0)
        K, W, p = integrate.energies(v0, m, phi, eps2)
        assert abs(K - 0.125) < 1e-15  # 2 x 1/2 x 1/2 x (1/2)^2; virial: 2K = |W| on a circle
        assert abs(W + 0.25 / math.sqrt(1.0 + eps2)) < 1e-15
        assert np.abs(p).max() < 1e-16
    # an eccentric orbit (speeds 0.35 instead of 0.5): the leapfrog's energy
    # error is O(dt^2) and bounded
    x0, _, m, acc = _two_body()
    v0 = np.array([[0.0, 0.35, 0.0], [0.0, -0.35, 0.0]])
    E0 = 2 * 0.5 * 0.5 * 0.35 ** 2 - 0.25
    errs = []
    for n in (200, 400):
        x, v, a, phi = integrate.leapfrog_kdk(x0, v0, m, 2.0 / n, n, acc)
        K, W, _ = integrate.energies(v, m, phi, 0.0)
        errs.append(abs((K + W - E0) / E0))
    assert errs[1] < 1e-5 and 3.5 < errs[0] / errs[1] < 4.5


def test_energies_with_per_particle_softening():
    # each sink feels its own softening: W = -1/2 (m1 m2 / sqrt(d^2 + e1^2) + m2 m1 / sqrt(d^2 + e2^2))
    x = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    m = np.array([0.5, 0.5])
    e2 = np.array([0.01, 0.04])
    _, phi = oracle.direct_forces(x, x, m, sink_eps2=e2)
    _, W, _ = integrate.energies(np.zeros((2, 3)), m, phi, e2)
    assert abs(W + 0.5 * (0.25 / math.sqrt(1.01) + 0.25 / math.sqrt(1.04))) < 1e-15


def test_energies_and_momentum_with_unequal_masses():
    # masses 1 and 2 at distance 2, velocities (1, 0, 0) and (0, 1, 0):
    # p = (1, 2, 0), K = (1 + 2) / 2, W = -m1 m2 / d = -1 (no softening)
    x = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]])
    m = np.array([1.0, 2.0])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    _, phi = oracle.direct_forces(x, x, m)
    K, W, p = integrate.energies(v, m, phi, 0.0)
    assert np.allclose(p, [1.0, 2.0, 0.0], rtol=0, atol=1e-15)
    assert abs(K - 1.5) < 1e-15 and abs(W + 1.0) < 1e-15


def test_leapfrog_is_time_reversible():
    rng = np.random.default_rng(12)
    n = 32
    x0 = rng.standard_normal((n, 3))
    v0 = 0.3 * rng.standard_normal((n, 3))
    m = np.full(n, 1.0 / n)
    acc = lambda y: oracle.direct_forces(y, y, m, eps2_all=0.01)  # noqa: E731
    x, v, _, _ = integrate.leapfrog_kdk(x0, v0, m, 0.01, 20, acc)
    assert np.abs(x - x0).max() > 1e-3
    xb, vb, _, _ = integrate.leapfrog_kdk(x, -v, m, 0.01, 20, acc)
    assert np.abs(xb - x0).max() < 1e-12
    assert np.abs(-vb - v0).max() < 1e-12


def test_a_planted_first_order_drift_is_caught():
    # drifting with the old velocity (a plausible slip) makes the scheme first
    # order: the convergence check above would see a ratio near 2, not 4
    x0, v0, m, acc = _two_body()

    def euler_like(n):
        x, v = x0.copy(), v0.copy()
        a, _ = acc(x)
        dt = 2 * math.pi / n
        for _ in range(n):
            x_new = x + v * dt
            v = v + a * (0.5 * dt)
            a, _ = acc(x_new)
            v = v + a * (0.5 * dt)
            x = x_new
        return float(np.abs(x - x0).max())

    r = euler_like(200) / euler_like(400)
    assert not (3.6 < r < 4.4)
