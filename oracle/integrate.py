"""FP64 CPU oracle of the time integration: the leapfrog integrator the paper
uses for its cold-collapse runs (Sec. 5: G = M = 1, a fixed step Delta t).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only ``tests/`` and
``bench.py``'s CPU legs may use it.

The leapfrog is taken in its kick-drift-kick form, one step of length dt:
    v_half = v + a(x) dt/2
    x'     = x + v_half dt
    v'     = v_half + a(x') dt/2
``accel`` is any callable x -> (a, phi); the tests pass the oracle's own
direct summation or its expansion forces on lists built for x.

Energies: K = 1/2 sum m |v|^2 and W = 1/2 sum m (phi + m / eps) -- the force
evaluation includes each particle's own pair in phi (-m/eps for eps > 0),
which is no part of the potential energy and is taken out again.
"""
from __future__ import annotations

import numpy as np


def leapfrog_kdk(x, v, m, dt, nsteps, accel, a=None):
    """nsteps kick-drift-kick steps; returns (x, v, a, phi) after the last one.

    ``a``: the acceleration at the initial x if already known.
    """
    x = np.array(x, dtype=np.float64, copy=True)
    v = np.array(v, dtype=np.float64, copy=True)
    phi = None
    if a is None:
        a, phi = accel(x)
    for _ in range(int(nsteps)):
        v = v + a * (0.5 * dt)
        x = x + v * dt
        a, phi = accel(x)
        v = v + a * (0.5 * dt)
    if phi is None:
        _, phi = accel(x)
    return x, v, a, phi


def energies(v, m, phi, eps2):
    """(K, W, p) in double, the self pair removed from W where eps2 > 0.

    eps2: one squared softening for all particles, or one per particle."""
    v = np.asarray(v, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    K = 0.5 * float(np.sum(m * np.sum(v * v, axis=1)))
    e2 = np.broadcast_to(np.asarray(eps2, dtype=np.float64), m.shape)
    self_term = np.zeros_like(m)
    pos = e2 > 0
    self_term[pos] = m[pos] / np.sqrt(e2[pos])
    W = 0.5 * float(np.sum(m * (phi + self_term)))
    p = (m[:, None] * v).sum(axis=0)
    return K, W, p
