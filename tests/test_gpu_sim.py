"""GPU leapfrog integration (include/qg_sim.h) against the oracle leapfrog
(oracle/integrate.py) with oracle forces on lists the host builder makes from
the same positions: state after a few steps, energies and momentum."""
import numpy as np
import pytest

import oracle
from oracle import integrate
from paper_1812_07313_gb300 import qgrav, sim, workloads
from paper_1812_07313_gb300 import tree as qtree
from tests.parity_util import TOL_MEDIAN, TOL_P99, assert_parity, rel_err, summary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qgrav.lib()


def _oracle_accel(m, sys_off, leaf, n_crit, theta, eps2, use_quad):
    def accel(x):
        t = qtree.Tree(x, m, sys_off, leaf, n_crit)
        L = t.walk(theta)
        a_s, phi_s = oracle.expansion_forces(t.group_off, t.x, t.x, t.m, L.plist_off, L.plist_idx, t.cell_com,
                                             t.cell_m, t.cell_q, L.clist_off, L.clist_idx, eps2_all=eps2,
                                             use_quad=use_quad)
        a = np.empty_like(a_s)
        phi = np.empty_like(phi_s)
        a[t.perm] = a_s
        phi[t.perm] = phi_s
        return a, phi
    return accel


@pytest.mark.parametrize("expansion,theta", [(qgrav.QG_QUAD, 0.5), (qgrav.QG_MONO, 0.4)], ids=["quad", "mono"])
def test_steps_match_the_oracle_leapfrog(expansion, theta):
    n, eps2, dt, steps = 6000, 2.0 ** -16, 2.0 ** -8, 3
    x0, v0, m = workloads.cold_collapse(n, 21)
    s = sim.Simulation(sim.Params(theta=theta, eps2=eps2, n_crit=64, leaf_max=8, expansion=expansion))
    s.set_state(x0, v0, m)
    x1, v1, a1, phi1 = s.state()
    acc = _oracle_accel(m, np.array([0, n]), 8, 64, theta, eps2, expansion == qgrav.QG_QUAD)
    a0_ref, phi0_ref = acc(x0)
    assert_parity(a1, phi1, a0_ref, phi0_ref, label="initial forces")
    assert np.array_equal(x1, x0) and np.array_equal(v1, v0)
    s.step(dt, steps)
    x, v, a, phi = s.state()
    xr, vr, ar, phir = integrate.leapfrog_kdk(x0, v0, m, dt, steps, acc, a=a0_ref)
    assert_parity(a, phi, ar, phir, label="forces after %d steps" % steps)
    # the velocity change is a sum of FP32-accurate kicks; positions follow it
    dv = summary(rel_err(v - v0, vr - v0))
    print("dv", dv)
    assert dv["median"] <= TOL_MEDIAN and dv["p99"] <= TOL_P99
    dx = summary(rel_err(x - x0, xr - x0))
    print("dx", dx)
    assert dx["median"] <= TOL_MEDIAN and dx["p99"] <= TOL_P99
    t = s.last_times()
    assert t["wall_ms"] > 0 and t["force_ms"] > 0 and t["groups"] > 0 and t["i_pc"] > 0
    s.close()


def test_energy_and_momentum_reductions():
    n, eps2 = 5000, 1e-4
    x0, v0, m = workloads.cold_collapse(n, 5)
    m = m * (1.0 + 0.5 * np.random.default_rng(3).random(n))  # unequal masses
    s = sim.Simulation(sim.Params(theta=0.5, eps2=eps2, n_crit=64))
    s.set_state(x0, v0, m)
    K, W, p = s.energy()
    _, _, a, phi = s.state()
    Kr, Wr, pr = integrate.energies(v0, m, phi, eps2)
    assert abs(K - Kr) <= 1e-13 * abs(Kr) and abs(W - Wr) <= 1e-13 * abs(Wr)
    assert np.abs(p - pr).max() <= 1e-15
    # W of the tree forces against W of the exact direct sum (method error only)
    _, phid = oracle.direct_forces(x0, x0, m, eps2_all=eps2)
    _, Wd, _ = integrate.energies(v0, m, phid, eps2)
    assert abs(W - Wd) <= 1e-3 * abs(Wd)
    s.close()


def test_cold_collapse_conserves_energy_before_collapse():
    n, eps2, dt = 1 << 15, 2.0 ** -16, 2.0 ** -8
    x0, v0, m = workloads.cold_collapse(n, 8)
    s = sim.Simulation(sim.Params(theta=0.5, eps2=eps2, n_crit=128))
    s.set_state(x0, v0, m)
    K0, W0, _ = s.energy()
    assert abs(2 * K0 / abs(W0) - 0.1) < 0.01  # initial virial ratio, W of the sampled sphere
    s.step(dt, 64)  # t = 0.25: contraction well under way, no collapse yet
    K, W, p = s.energy()
    E0, E = K0 + W0, K + W
    print("E0 %.8f E %.8f rel %.2e K %.4f W %.4f" % (E0, E, (E - E0) / abs(E0), K, W))
    assert K > 1.3 * K0 and W < W0  # it falls in (free fall of this sphere takes t ~ 1.1)
    assert abs(E - E0) < 1e-4 * abs(E0)
    assert np.abs(p).max() < 1e-5
    s.close()


def test_per_particle_softening_matches_the_oracle_leapfrog():
    # independent systems, each with its own softening (one value per system)
    ps = workloads.batched_systems(nsys=3, seed=11, n_lo=800, n_hi=3000)
    n = len(ps.m)
    sys_of = np.repeat(np.arange(3), np.diff(ps.sys_off))
    e2 = (np.array([1e-2, 3e-2, 2e-3])[sys_of] ** 2).astype(np.float32)
    rng = np.random.default_rng(5)
    v0 = 0.05 * rng.standard_normal((n, 3))
    dt, steps = 2e-3, 2
    s = sim.Simulation(sim.Params(theta=0.5, eps2=0.0, n_crit=64))
    s.set_state(ps.x, v0, ps.m, ps.sys_off, eps2=e2)

    def accel(x):
        t = qtree.Tree(x, ps.m, ps.sys_off, 8, 64)
        L = t.walk(0.5)
        a_s, phi_s = oracle.expansion_forces(t.group_off, t.x, t.x, t.m, L.plist_off, L.plist_idx, t.cell_com,
                                             t.cell_m, t.cell_q, L.clist_off, L.clist_idx,
                                             sink_eps2=e2[t.perm].astype(np.float64))
        a = np.empty_like(a_s)
        phi = np.empty_like(phi_s)
        a[t.perm] = a_s
        phi[t.perm] = phi_s
        return a, phi

    _, _, a1, phi1 = s.state()
    a0, phi0 = accel(ps.x)
    assert_parity(a1, phi1, a0, phi0, label="per-particle softening, initial")
    K, W, _ = s.energy()
    Kr, Wr, _ = integrate.energies(v0, ps.m, phi1, e2)
    assert abs(K - Kr) <= 1e-13 * Kr and abs(W - Wr) <= 1e-12 * abs(Wr)
    s.step(dt, steps)
    x, v, a, phi = s.state()
    xr, vr, ar, phir = integrate.leapfrog_kdk(ps.x, v0, ps.m, dt, steps, accel, a=a0)
    assert_parity(a, phi, ar, phir, label="per-particle softening, after %d steps" % steps)
    dv = summary(rel_err(v - v0, vr - v0))
    assert dv["median"] <= TOL_MEDIAN and dv["p99"] <= TOL_P99
    s.close()
    with pytest.raises(qgrav.QGError):
        s2 = sim.Simulation(sim.Params(theta=0.5))
        bad = e2.copy()
        bad[3] = -1.0
        s2.set_state(ps.x, v0, ps.m, ps.sys_off, eps2=bad)


def test_single_particle_moves_freely():
    s = sim.Simulation(sim.Params(theta=0.5, eps2=1e-4, n_crit=8, autotune=False))
    s.set_state(np.array([[0.25, -0.5, 1.0]]), np.array([[0.1, 0.0, -0.2]]), np.array([2.0]))
    s.step(0.5, 4)
    x, v, a, phi = s.state()
    assert np.allclose(x, [[0.45, -0.5, 0.6]], rtol=0, atol=1e-15) and np.array_equal(v, [[0.1, 0.0, -0.2]])
    assert np.array_equal(a, np.zeros((1, 3))) and abs(phi[0] + 2.0 / 1e-2) < 1e-9  # only its own pair, -m/eps
    K, W, p = s.energy()
    assert abs(K - 0.05) < 1e-15 and abs(W) < 1e-9 and np.allclose(p, [0.2, 0.0, -0.4])
    s.close()


def test_batched_systems_step_like_each_system_alone():
    # every system has its own root, so its tree, groups and lists -- and, at
    # one launch shape, its forces -- are the same in the batch and alone
    ps = workloads.batched_systems(nsys=4, seed=3, n_lo=500, n_hi=3000)
    n = len(ps.m)
    v = np.zeros((n, 3))
    prm = sim.Params(theta=0.5, eps2=1e-4, n_crit=64, autotune=False)
    s = sim.Simulation(prm)
    with pytest.raises(qgrav.QGError):
        s.step(0.01, 1)  # no state yet
    s.set_state(ps.x, v, ps.m, ps.sys_off)
    s.step(1e-3, 2)
    x, v1, a, phi = s.state()
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(a))
    for q in range(4):
        b, e = ps.sys_off[q], ps.sys_off[q + 1]
        one = sim.Simulation(prm)
        one.set_state(ps.x[b:e], v[b:e], ps.m[b:e])
        one.step(1e-3, 2)
        xq, vq, aq, phiq = one.state()
        assert np.array_equal(xq, x[b:e]) and np.array_equal(vq, v1[b:e]), q
        assert np.array_equal(aq, a[b:e]) and np.array_equal(phiq, phi[b:e]), q
        one.close()
    with pytest.raises(qgrav.QGError):
        s.step(float("nan"), 1)
    s.close()
    with pytest.raises(qgrav.QGError):
        sim.Simulation(sim.Params(theta=0.0))


def test_autotuning_follows_the_lists():
    """With autotune on, the force launch is tuned at the first force
    evaluation and again only when the step's list entries have changed by
    more than a quarter since the last tuning: steps that hardly move the
    particles keep the tuning; a new state with much longer lists (a
    centrally concentrated sphere after a uniform one) starts an online
    trial, whose evaluations each run one neighbouring launch shape, after
    which the fastest shape stays."""
    n = 20000
    ps = workloads.small_set("sphere", n, 7, 0.01)
    s = sim.Simulation(sim.Params(theta=0.5, eps2=1e-4, n_crit=64, autotune=True))
    s.set_state(ps.x, np.zeros((n, 3)), ps.m)
    t0 = s.last_times()
    assert t0["retunes"] == 1 and t0["trial_left"] == 0
    s.step(1e-3, 3)   # hardly moves: the same lists, no tuning
    t1 = s.last_times()
    assert t1["retunes"] == 1 and t1["trial_left"] == 0
    assert abs((t1["n_plist"] + t1["n_clist"]) / (t0["n_plist"] + t0["n_clist"]) - 1) < 0.25
    pl = workloads.small_set("plummer", n, 8, 0.01)
    s.set_state(pl.x, np.zeros((n, 3)), pl.m)
    t2 = s.last_times()
    ratio = (t2["n_plist"] + t2["n_clist"]) / (t1["n_plist"] + t1["n_clist"])
    print("list entries, Plummer over uniform: %.2fx; %d tunings" % (ratio, t2["retunes"]))
    assert abs(ratio - 1) > 0.25 and t2["retunes"] == 2
    shape = lambda t: (t["sinks_per_thread"], t["sinks_adaptive"], t["warps_per_group"], t["tile_j"], t["form"])
    tried, left = [shape(t2)], t2["trial_left"]
    assert 1 <= left <= 5
    while left:
        s.step(1e-4, 1)
        t = s.last_times()
        assert t["trial_left"] == left - 1 and t["retunes"] == 2
        left = t["trial_left"]
        tried.append(shape(t))
    assert len(set(tried)) == len(tried) >= 2
    s.step(1e-4, 1)   # the trial is over: one of its shapes stays
    kept = shape(s.last_times())
    assert kept in tried
    s.step(1e-4, 3)
    assert shape(s.last_times()) == kept and s.last_times()["retunes"] == 2
    x, v, a, phi = s.state()
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(phi))
    s.close()
