"""Pins of the FP64 oracle against things other than itself.

Each test fixes the oracle to a closed form, a brute-force sum, an invariant or
a limit that the paper and the mathematics determine, so that a plausible slip
in the oracle (a dropped term, a wrong sign, the 1/2 of Eq. 5 or the 5 of
Eq. 7 misplaced, a transposed Q index) fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1812_07313_gb300 import tree as qtree
from paper_1812_07313_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _one_group(sinks, src_x=None, src_m=None, cells=None, eps2=0.0, use_quad=True):
    """Evaluate the oracle for one group holding `sinks` with explicit lists."""
    sinks = np.atleast_2d(np.asarray(sinks, dtype=np.float64))
    n = len(sinks)
    if src_x is None:
        src_x, src_m = np.zeros((0, 3)), np.zeros(0)
    src_x = np.atleast_2d(np.asarray(src_x, dtype=np.float64)).reshape(-1, 3)
    src_m = np.asarray(src_m, dtype=np.float64).reshape(-1)
    if cells is None:
        com, cm, cq = np.zeros((0, 3)), np.zeros(0), np.zeros((0, 6))
    else:
        com, cm, cq = cells
        com = np.atleast_2d(com).reshape(-1, 3)
        cm = np.asarray(cm, dtype=np.float64).reshape(-1)
        cq = np.atleast_2d(cq).reshape(-1, 6)
    return oracle.expansion_forces(
        [0, n], sinks, src_x, src_m,
        [0, len(src_m)], np.arange(len(src_m), dtype=np.int32),
        com, cm, cq, [0, len(cm)], np.arange(len(cm), dtype=np.int32),
        eps2_all=eps2, use_quad=use_quad)


def _random_cluster(rng, k, size):
    x = rng.uniform(-size, size, (k, 3))
    m = rng.uniform(0.5, 1.5, k)
    return x, m


# ---------------------------------------------------------------- Eq. 2

def test_two_mass_golden_closed_form():
    """Hand-derived values for two masses (tests/golden/two_mass_expansion.txt)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "two_mass_expansion.txt"))
    for r in rows:
        m, s, R = r[0], r[1], r[2]
        sink = r[3:6]
        q_ref, phi_ref, a_ref = r[6:12], r[12], r[13:16]
        x = np.array([[s, 0, 0], [-s, 0, 0]])
        mass, com, q = oracle.cell_moments(x, [m, m])
        assert mass == 2 * m
        np.testing.assert_allclose(com, 0.0, atol=1e-15)
        np.testing.assert_allclose(q, q_ref, rtol=1e-15, atol=1e-15)
        a, phi = _one_group(sink, cells=(com, [mass], q))
        np.testing.assert_allclose(phi[0], phi_ref, rtol=1e-14)
        np.testing.assert_allclose(a[0], a_ref, rtol=1e-14, atol=1e-16)
        # and the exact two-body values differ by O((s/R)^4) relative
        ad, phid = oracle.direct_forces(sink, x, [m, m])
        rel = abs(phi[0] - phid[0]) / abs(phid[0])
        assert rel < 3 * (s / R) ** 4


def test_quadrupole_traceless_symmetric_and_rotation():
    rng = np.random.default_rng(11)
    x, m = _random_cluster(rng, 37, 0.7)
    mass, com, q = oracle.cell_moments(x, m)
    r2 = np.sum(m * np.sum((x - com) ** 2, axis=1))
    assert abs(q[0] + q[3] + q[5]) <= 1e-14 * r2
    Q = np.array([[q[0], q[1], q[2]], [q[1], q[3], q[4]], [q[2], q[4], q[5]]])
    # brute force of the definition with numpy outer products
    Qb = sum(mk * (3 * np.outer(d, d) - d @ d * np.eye(3)) for mk, d in zip(m, x - com))
    np.testing.assert_allclose(Q, Qb, rtol=1e-12, atol=1e-14)
    # rotation covariance Q' = R Q R^T
    A = rng.standard_normal((3, 3))
    Rm, _ = np.linalg.qr(A)
    _, com2, q2 = oracle.cell_moments(x @ Rm.T, m)
    Q2 = np.array([[q2[0], q2[1], q2[2]], [q2[1], q2[3], q2[4]], [q2[2], q2[4], q2[5]]])
    np.testing.assert_allclose(Q2, Rm @ Q @ Rm.T, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(com2, Rm @ com, atol=1e-14)
    # the expansion force transforms as a vector
    sink = np.array([3.0, -4.0, 2.5])
    a1, p1 = _one_group(sink, cells=(com, [mass], q), eps2=1e-3)
    a2, p2 = _one_group(Rm @ sink, cells=(com2, [mass], q2), eps2=1e-3)
    np.testing.assert_allclose(a2[0], Rm @ a1[0], rtol=1e-12)
    np.testing.assert_allclose(p2[0], p1[0], rtol=1e-13)


def test_one_particle_cell_is_point_mass():
    x = np.array([[0.3, -0.2, 0.9]])
    mass, com, q = oracle.cell_moments(x, [0.25])
    assert np.max(np.abs(q)) <= 1e-30
    sinks = np.array([[1.0, 2.0, 3.0], [-0.5, 0.1, 0.2]])
    a, phi = _one_group(sinks, cells=(com, [mass], q), eps2=1e-2)
    ad, phid = oracle.direct_forces(sinks, x, [0.25], eps2_all=1e-2)
    np.testing.assert_allclose(a, ad, rtol=1e-14)
    np.testing.assert_allclose(phi, phid, rtol=1e-14)


# ---------------------------------------------------------------- Eq. 1 / Eq. 7

@pytest.mark.parametrize("use_quad,slope", [(False, 2.0), (True, 3.0)])
def test_expansion_error_order(use_quad, slope):
    """About the centre of mass the dipole vanishes: the monopole-only residual
    falls as (s/R)^2 and the monopole+quadrupole residual as (s/R)^3 (the
    octupole).  A wrong quadrupole coefficient or sign leaves an (s/R)^2 term."""
    rng = np.random.default_rng(5)
    x, m = _random_cluster(rng, 25, 0.5)
    mass, com, q = oracle.cell_moments(x, m)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    Rs = np.array([8.0, 16.0, 32.0, 64.0])
    ea, ep = [], []
    for R in Rs:
        sink = com + R * u
        a, phi = _one_group(sink, cells=(com, [mass], q), use_quad=use_quad)
        ad, phid = oracle.direct_forces(sink, x, m)
        ea.append(np.linalg.norm(a[0] - ad[0]) / np.linalg.norm(ad[0]))
        ep.append(abs(phi[0] - phid[0]) / abs(phid[0]))
    for e in (ea, ep):
        k = -np.polyfit(np.log(Rs), np.log(e), 1)[0]
        assert abs(k - slope) < 0.15, (k, e)


def test_force_is_minus_gradient_of_potential():
    """Central differences of the oracle's phi reproduce its a (Eq. 6): this
    fixes the sign and every coefficient of Eq. 7 against Eq. 1."""
    rng = np.random.default_rng(7)
    src = rng.uniform(-1, 1, (9, 3)) + np.array([2.0, 0, 0])
    srcm = rng.uniform(0.1, 1.0, 9)
    cells_com, cells_m, cells_q = [], [], []
    for c in range(6):
        xc, mc = _random_cluster(rng, 12, 0.3)
        xc += rng.uniform(-3, 3, 3) + np.array([0, 3.0, 0])
        M, com, q = oracle.cell_moments(xc, mc)
        cells_com.append(com), cells_m.append(M), cells_q.append(q)
    cells = (np.array(cells_com), np.array(cells_m), np.array(cells_q))
    x0 = np.array([0.1, -0.2, 0.05])
    h = 1e-5
    pts = [x0]
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        pts += [x0 + e, x0 - e]
    a, phi = _one_group(np.array(pts), src, srcm, cells, eps2=0.04)
    fd = np.array([-(phi[1 + 2 * k] - phi[2 + 2 * k]) / (2 * h) for k in range(3)])
    np.testing.assert_allclose(a[0], fd, rtol=2e-8, atol=2e-8 * np.linalg.norm(a[0]))


def test_softening_and_self_pair():
    """Plummer softening: a self pair with eps > 0 adds -m/eps to phi and no
    force; with eps = 0 the coincident pair is skipped."""
    x = np.array([[0.2, 0.3, 0.4]])
    a, phi = _one_group(x, x, [0.5], eps2=0.01)
    assert phi[0] == pytest.approx(-0.5 / 0.1, rel=1e-15)
    assert np.all(a[0] == 0.0)
    a, phi = _one_group(x, x, [0.5], eps2=0.0)
    assert phi[0] == 0.0 and np.all(a[0] == 0.0)
    # one softened pair in closed form
    a, phi = _one_group([0, 0, 0], [[3.0, 4.0, 0.0]], [2.0], eps2=11.0)  # rhat = 6
    np.testing.assert_allclose(phi[0], -2.0 / 6.0, rtol=1e-15)
    np.testing.assert_allclose(a[0], 2.0 / 216.0 * np.array([3.0, 4.0, 0.0]), rtol=1e-15)


def test_direct_sum_momentum_conservation():
    """Direct summation with one softening: sum_i m_i a_i = 0 (Newton's third law)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((200, 3))
    m = rng.uniform(0.1, 1, 200)
    a, phi = oracle.direct_forces(x, x, m, eps2_all=1e-4)
    tot = np.sum(m[:, None] * a, axis=0)
    scale = np.sum(m[:, None] * np.abs(a))
    assert np.all(np.abs(tot) < 1e-13 * scale)
    # potential energy is symmetric: sum m_i phi_i equals the pair sum twice
    d = x[:, None, :] - x[None, :, :]
    r = np.sqrt(np.sum(d * d, axis=2) + 1e-4)
    W = -np.sum(np.outer(m, m) / r)  # includes i == j terms, as phi does
    np.testing.assert_allclose(np.sum(m * phi), W, rtol=1e-12)


def test_per_sink_softening_matches_global():
    rng = np.random.default_rng(9)
    x = rng.standard_normal((30, 3))
    m = rng.uniform(0.1, 1, 30)
    a1, p1 = oracle.direct_forces(x[:5], x, m, eps2_all=0.02)
    a2, p2 = oracle.direct_forces(x[:5], x, m, sink_eps2=np.full(5, 0.02))
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)


# ---------------------------------------------------------------- with the tree

def _tree(kind, n, seed, eps, n_crit=64, leaf=8):
    ps = workloads.small_set(kind, n, seed, eps)
    return ps, qtree.Tree(ps.x, ps.m, ps.sys_off, leaf, n_crit)


def test_theta_zero_is_direct_summation():
    ps, tr = _tree("plummer", 512, 21, 0.05, n_crit=32)
    L = tr.walk(0.0)
    assert len(L.clist_idx) == 0
    a, phi = oracle.expansion_forces(tr.group_off, tr.x, tr.x, tr.m, L.plist_off, L.plist_idx,
                                     tr.cell_com, tr.cell_m, tr.cell_q, L.clist_off, L.clist_idx,
                                     eps2_all=0.05 ** 2)
    ad, phid = oracle.direct_forces(tr.x, tr.x, tr.m, eps2_all=0.05 ** 2)
    np.testing.assert_allclose(a, ad, rtol=1e-11, atol=1e-13 * np.abs(ad).max())
    np.testing.assert_allclose(phi, phid, rtol=1e-12)


def test_error_falls_with_theta_and_quad_beats_mono():
    """p90 of Eq. 8 falls as theta shrinks; with quadrupoles it is lower than
    monopole-only at the same theta and falls more steeply (Sec. 4: roughly
    theta^(5/2) and theta^(7/2))."""
    ps, tr = _tree("sphere", 8192, 31, 1e-2, n_crit=64)
    eps2 = 1e-4
    ad, _ = oracle.direct_forces(tr.x, tr.x, tr.m, eps2_all=eps2)
    thetas = np.array([0.3, 0.4, 0.5, 0.6, 0.7])
    p90 = {True: [], False: []}
    for th in thetas:
        L = tr.walk(th)
        for uq in (True, False):
            a, _ = oracle.expansion_forces(tr.group_off, tr.x, tr.x, tr.m, L.plist_off, L.plist_idx,
                                           tr.cell_com, tr.cell_m, tr.cell_q, L.clist_off,
                                           L.clist_idx, eps2_all=eps2, use_quad=uq)
            p90[uq].append(np.percentile(oracle.relative_error(a, ad), 90))
    for uq in (True, False):
        assert np.all(np.diff(p90[uq]) > 0), p90[uq]
    assert np.all(np.array(p90[True]) < np.array(p90[False]))
    s_mono = np.polyfit(np.log(thetas), np.log(p90[False]), 1)[0]
    s_quad = np.polyfit(np.log(thetas), np.log(p90[True]), 1)[0]
    assert 1.5 < s_mono < 3.5, s_mono
    assert 2.5 < s_quad < 5.0, s_quad
    assert s_quad > s_mono


def test_threaded_oracle_gives_identical_results():
    """Splitting the groups over host threads changes no bit of the result."""
    from paper_1812_07313_gb300 import tree as qtree
    from paper_1812_07313_gb300 import workloads
    ps = workloads.small_set("plummer", 8000, 21, 1e-2)
    t = qtree.Tree(ps.x, ps.m, ps.sys_off, 8, 64)
    L = t.walk(0.5)
    args = (t.group_off, t.x, t.x, t.m, L.plist_off, L.plist_idx, t.cell_com, t.cell_m, t.cell_q, L.clist_off,
            L.clist_idx)
    a1, p1 = oracle.expansion_forces(*args, eps2_all=1e-4)
    try:
        oracle.set_threads(4)
        a2, p2 = oracle.expansion_forces(*args, eps2_all=1e-4)
    finally:
        oracle.set_threads(1)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
