"""Seeded synthetic particle sets for the tree-force hot path.

This module holds no force or moment arithmetic: it only draws particle
positions and masses.  Both the CUDA path and the FP64 oracle consume what it
produces, so it is the one piece of code they share.

The distributions follow the paper's test problems (Sec. 4-5: a homogeneous
sphere, a Plummer model; equal-mass particles, G = M = 1) and the synthetic
workloads this library is measured on:

  ``sphere_4k``     4096 particles uniform in the unit sphere, eps = 1e-2,
                    leaf <= 8, n_crit = 64, theta = 0.5
  ``cube_1m``       2^20 particles uniform in the unit cube,
                    eps = 1/(20 N^(1/3)), n_crit = 256, theta in {0.3,0.5,0.7}
  ``plummer_4m``    2^22-particle Plummer sphere (a = 1, r <= 100), eps = 1e-3,
                    n_crit = 256, theta 0.3-0.8
  ``batched_512``   512 independent Plummer / Hernquist systems with N
                    log-uniform in [1024, 65536], eps = 1e-2, n_crit = 64,
                    theta = 0.5, each system placed far from the origin
  ``batched_64``    the first 64 systems' distribution of batched_512 (a
                    smaller case of the same kernel shape, for profiling)
  ``clumpy_16m``    2^24 particles in the unit cube: 70 % in 2000 Plummer clumps
                    (clump masses dN/dM ~ M^-1.9 on [1, 1000], scale radii
                    log-uniform in [1e-3, 1e-2], truncated at 10 scale radii,
                    centres uniform in [0.05, 0.95]^3) + 30 % uniform
                    background, eps = 5e-5, theta = 0.5

Random numbers come from numpy's PCG64 with the stated seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ParticleSet:
    """Positions [n,3] (float64), masses [n] (float64), and system offsets.

    ``sys_off`` has nsys+1 entries; system s owns particles
    [sys_off[s], sys_off[s+1]) and is treated as an independent problem with
    its own tree and softening ``eps[s]``.
    """
    x: np.ndarray
    m: np.ndarray
    sys_off: np.ndarray
    eps: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def nsys(self) -> int:
        return int(len(self.sys_off) - 1)


def _isotropic(rng, n):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def uniform_sphere(n, seed, radius=1.0):
    """Uniform density inside a sphere: isotropic direction, r = R U^(1/3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return _isotropic(rng, n) * r[:, None]


def uniform_cube(n, seed, lo=0.0, hi=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return lo + (hi - lo) * rng.random((n, 3))


def _plummer_radii(rng, n, a, rmax):
    """Plummer cumulative mass M(<r)/M = r^3/(r^2+a^2)^(3/2) inverted, resampled above rmax."""
    r = np.empty(n)
    todo = np.arange(n)
    while len(todo):
        u = rng.random(len(todo))
        u = np.clip(u, 1e-300, None)
        rr = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        ok = rr <= rmax
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    return r


def _hernquist_radii(rng, n, a, rmax):
    """Hernquist cumulative mass M(<r)/M = r^2/(r+a)^2 inverted, resampled above rmax."""
    r = np.empty(n)
    todo = np.arange(n)
    while len(todo):
        s = np.sqrt(rng.random(len(todo)))
        with np.errstate(divide="ignore"):
            rr = a * s / (1.0 - s)
        ok = np.isfinite(rr) & (rr <= rmax)
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    return r


def plummer(n, seed, a=1.0, rmax=100.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    r = _plummer_radii(rng, n, a, rmax)
    return _isotropic(rng, n) * r[:, None]


def hernquist(n, seed, a=1.0, rmax=100.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    r = _hernquist_radii(rng, n, a, rmax)
    return _isotropic(rng, n) * r[:, None]


def exponential_disk(n, seed, r_d=1.0, z0=0.1, rmax=10.0):
    """Exponential disk: surface density proportional to exp(-R / r_d) --
    the cylindrical radius then follows a Gamma(2, r_d) distribution --
    truncated at R <= rmax r_d (resampled), uniform azimuth, and a
    sech^2(z / z0) vertical profile (z = z0 atanh(2U - 1)).  The paper gives
    no disk parameters; r_d = 1, z0 = 0.1 r_d and the truncation at 10 r_d
    are this generator's choice."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = rng.gamma(2.0, r_d, n)
    bad = R > rmax * r_d
    while bad.any():
        R[bad] = rng.gamma(2.0, r_d, int(bad.sum()))
        bad = R > rmax * r_d
    phi = 2.0 * np.pi * rng.random(n)
    u = rng.random(n)
    u = np.clip(u, 1e-15, 1.0 - 1e-15)
    z = z0 * np.arctanh(2.0 * u - 1.0)
    return np.stack([R * np.cos(phi), R * np.sin(phi), z], axis=1)


def clumpy_field(n, seed, nclumps=2000, clump_frac=0.7, slope=-1.9, mass_range=1000.0,
                 rs_lo=1e-3, rs_hi=1e-2, trunc=10.0):
    """Unit cube: clump_frac of the particles in Plummer clumps, the rest uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    # clump masses from dN/dM ~ M^slope on [1, mass_range] by inverse transform
    u = rng.random(nclumps)
    k = slope + 1.0
    mc = (1.0 + u * (mass_range ** k - 1.0)) ** (1.0 / k)
    n_clumped = int(round(clump_frac * n))
    counts = np.floor(n_clumped * mc / mc.sum()).astype(np.int64)
    short = n_clumped - int(counts.sum())
    order = np.argsort(-(n_clumped * mc / mc.sum() - counts))
    counts[order[:short]] += 1
    rs = np.exp(rng.uniform(np.log(rs_lo), np.log(rs_hi), nclumps))
    centres = rng.uniform(0.05, 0.95, (nclumps, 3))
    parts = []
    for c in range(nclumps):
        nc = int(counts[c])
        if nc == 0:
            continue
        r = _plummer_radii(rng, nc, rs[c], trunc * rs[c])
        parts.append(centres[c] + _isotropic(rng, nc) * r[:, None])
    parts.append(rng.random((n - n_clumped, 3)))
    x = np.concatenate(parts, axis=0)
    return x[rng.permutation(n)]


def single_system(name, x, eps, meta=None):
    n = len(x)
    return ParticleSet(x=np.ascontiguousarray(x, dtype=np.float64),
                       m=np.full(n, 1.0 / n), sys_off=np.array([0, n], dtype=np.int64),
                       eps=np.array([eps], dtype=np.float64), name=name, meta=meta or {})


def batched_systems(nsys=512, seed=4, n_lo=1024, n_hi=65536, eps=1e-2, spacing=1000.0,
                    rmax=100.0):
    """Independent Plummer or Hernquist systems (p = 1/2 each), N log-uniform.

    System s is centred at spacing * (i, j, k) for its index on a cubic grid,
    so coordinates reach several thousand: far enough from the origin that
    casting absolute positions to FP32 would lose most of the bits that the
    pairwise separations need.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), nsys))).astype(np.int64)
    kinds = rng.random(nsys) < 0.5
    side = int(np.ceil(nsys ** (1.0 / 3.0)))
    xs, ms = [], []
    for s in range(nsys):
        sub = int(rng.integers(0, 2 ** 62))
        if kinds[s]:
            xs_s = plummer(int(ns[s]), sub, 1.0, rmax)
        else:
            xs_s = hernquist(int(ns[s]), sub, 1.0, rmax)
        i, j, k = s % side, (s // side) % side, s // (side * side)
        xs.append(xs_s + spacing * np.array([i + 1, j + 1, k + 1], dtype=np.float64))
        ms.append(np.full(int(ns[s]), 1.0 / ns[s]))
    sys_off = np.zeros(nsys + 1, dtype=np.int64)
    sys_off[1:] = np.cumsum(ns)
    return ParticleSet(x=np.concatenate(xs), m=np.concatenate(ms), sys_off=sys_off,
                       eps=np.full(nsys, eps), name="batched_%d" % nsys,
                       meta={"kinds": ["plummer" if k else "hernquist" for k in kinds]})


def cold_collapse(n, seed, virial=0.1, radius=1.0):
    """Initial state of the cold-collapse runs (Sec. 5): a homogeneous sphere
    of radius 1 and total mass 1 (G = 1), at rest except for isotropic
    Gaussian velocities scaled so that the virial ratio 2K/|W| equals
    ``virial``, with W = -3/5 G M^2 / R of the uniform sphere.  The velocity
    distribution is not given in the paper; Gaussian is this generator's
    choice.  Returns (x [n,3], v [n,3], m [n])."""
    x = uniform_sphere(n, seed, radius)
    rng = np.random.Generator(np.random.PCG64(seed + 1000003))
    v = rng.standard_normal((n, 3))
    v -= v.mean(axis=0)
    m = np.full(n, 1.0 / n)
    K_target = 0.5 * virial * 0.6 / radius
    K = 0.5 * float(np.sum(m * np.sum(v * v, axis=1)))
    v *= np.sqrt(K_target / K)
    return x, v, m


@dataclass(frozen=True)
class Workload:
    name: str
    leaf_max: int
    n_crit: int
    thetas: tuple
    theta: float           # the theta a single benchmark step uses

    def particles(self) -> ParticleSet:
        return _GENERATORS[self.name]()


def _cube_1m():
    n = 1 << 20
    return single_system("cube_1m", uniform_cube(n, 2), 1.0 / (20.0 * n ** (1.0 / 3.0)))


_GENERATORS = {
    "sphere_4k": lambda: single_system("sphere_4k", uniform_sphere(4096, 1), 1e-2),
    "cube_1m": _cube_1m,
    "plummer_4m": lambda: single_system("plummer_4m", plummer(1 << 22, 3), 1e-3),
    "batched_512": lambda: batched_systems(512, 4),
    "batched_64": lambda: batched_systems(64, 4),
    "clumpy_16m": lambda: single_system("clumpy_16m", clumpy_field(1 << 24, 5), 5e-5),
}

WORKLOADS = {
    "sphere_4k": Workload("sphere_4k", 8, 64, (0.5,), 0.5),
    "cube_1m": Workload("cube_1m", 8, 256, (0.3, 0.5, 0.7), 0.5),
    "plummer_4m": Workload("plummer_4m", 8, 256, (0.3, 0.4, 0.5, 0.6, 0.7, 0.8), 0.5),
    "batched_512": Workload("batched_512", 8, 64, (0.5,), 0.5),
    "batched_64": Workload("batched_64", 8, 64, (0.5,), 0.5),
    "clumpy_16m": Workload("clumpy_16m", 8, 256, (0.5,), 0.5),
}


def small_set(kind, n, seed, eps):
    """Small sets for tests: 'sphere', 'cube', 'plummer', 'hernquist', 'clumpy', 'disk'."""
    if kind == "sphere":
        x = uniform_sphere(n, seed)
    elif kind == "cube":
        x = uniform_cube(n, seed)
    elif kind == "plummer":
        x = plummer(n, seed)
    elif kind == "hernquist":
        x = hernquist(n, seed)
    elif kind == "clumpy":
        x = clumpy_field(n, seed, nclumps=max(1, n // 200))
    elif kind == "disk":
        x = exponential_disk(n, seed)
    else:
        raise ValueError(kind)
    return single_system("%s_%d" % (kind, n), x, eps)
