"""The seeded input generators follow the recipes they state: distribution
functions with closed-form quantiles and moments, sizes, masses and system
layout (no force arithmetic involved)."""
import numpy as np

from paper_1812_07313_gb300 import workloads


def test_uniform_sphere_and_cube():
    x = workloads.uniform_sphere(200000, 3)
    r = np.linalg.norm(x, axis=1)
    assert r.max() <= 1.0
    assert abs(r.mean() - 0.75) < 3e-3           # E[U^(1/3)] = 3/4
    assert abs(np.mean(r < 0.5) - 0.125) < 3e-3   # (1/2)^3
    assert np.abs(x.mean(axis=0)).max() < 5e-3   # isotropic
    c = workloads.uniform_cube(200000, 4)
    assert c.min() >= 0.0 and c.max() < 1.0 and np.abs(c.mean(axis=0) - 0.5).max() < 3e-3


def test_plummer_and_hernquist_radii():
    r = np.linalg.norm(workloads.plummer(200000, 5), axis=1)
    assert r.max() <= 100.0
    # M(<r) = r^3 / (r^2 + 1)^(3/2): median 1 / sqrt(2^(2/3) - 1), M(<1) = 2^(-3/2)
    assert abs(np.median(r) - 1.0 / np.sqrt(2 ** (2 / 3) - 1)) < 0.02
    assert abs(np.mean(r < 1.0) - 2 ** -1.5) < 4e-3
    r = np.linalg.norm(workloads.hernquist(200000, 6), axis=1)
    assert r.max() <= 100.0
    # M(<r) = r^2 / (r + 1)^2 conditioned on r <= 100: median where r^2/(r+1)^2 = 0.5 (100/101)^2
    s = np.sqrt(0.5) * 100.0 / 101.0
    assert abs(np.median(r) - s / (1 - s)) < 0.03


def test_clumpy_field_layout():
    n = 100000
    x = workloads.clumpy_field(n, 7, nclumps=300)
    assert x.shape == (n, 3)
    # clump centres in [0.05, 0.95], truncated at 10 scale radii <= 0.1; the background fills [0, 1)
    assert x.min() >= -0.05 and x.max() <= 1.05
    # 70 % in clumps: far more particles in the densest 1 % of the cells of a 20^3 grid than uniform
    h, _ = np.histogramdd(np.clip(x, 0, 1 - 1e-12), bins=20, range=[(0, 1)] * 3)
    top = np.sort(h.ravel())[::-1][:80].sum() / n
    assert top > 0.3


def test_batched_systems_layout():
    ps = workloads.batched_systems(nsys=64, seed=4, n_lo=1024, n_hi=4096)
    ns = np.diff(ps.sys_off)
    assert ns.min() >= 1024 and ns.max() <= 4096 and len(ns) == 64
    for s in range(64):
        b, e = ps.sys_off[s], ps.sys_off[s + 1]
        assert abs(ps.m[b:e].sum() - 1.0) < 1e-12
        c = np.median(ps.x[b:e], axis=0)
        side = 4  # ceil(64^(1/3))
        want = 1000.0 * np.array([s % side + 1, (s // side) % side + 1, s // (side * side) + 1])
        assert np.abs(c - want).max() < 5.0   # centred on its grid point, far from the origin
    kinds = ps.meta["kinds"]
    assert 16 < sum(k == "plummer" for k in kinds) < 48


def test_cold_collapse_initial_state():
    x, v, m = workloads.cold_collapse(50000, 8)
    K = 0.5 * float(np.sum(m * np.sum(v * v, axis=1)))
    assert abs(K - 0.5 * 0.1 * 0.6) < 1e-12       # 2K/|W| = 0.1 with W = -3/5
    assert np.abs((m[:, None] * v).sum(axis=0)).max() < 1e-12
    assert abs(m.sum() - 1.0) < 1e-12 and np.linalg.norm(x, axis=1).max() <= 1.0


def test_named_workloads_sizes():
    ps = workloads.WORKLOADS["sphere_4k"].particles()
    assert ps.n == 4096 and abs(ps.m.sum() - 1.0) < 1e-12 and ps.eps[0] == 1e-2
    assert workloads.WORKLOADS["cube_1m"].n_crit == 256 and workloads.WORKLOADS["batched_512"].n_crit == 64
