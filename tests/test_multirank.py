"""The N > 1 path on the CPU with gloo, world size 2: the group split that
shards a step across ranks (each rank evaluates its range of groups; the
gathered result equals the unsharded one) and the benchmark's aggregation of
the ranks' timings (max over ranks; replicas' units times the ranks, shards'
units added up)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1812_07313_gb300 import shard
from paper_1812_07313_gb300 import tree as qtree
from paper_1812_07313_gb300 import workloads

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    ps = workloads.small_set("plummer", 3000, 41, 0.02)
    tr = qtree.Tree(ps.x, ps.m, ps.sys_off, 8, 32)
    return ps, tr, tr.walk(0.6)


def _worker_shard(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ps, tr, L = _case()
        sh = shard.shards(tr.group_off, L.plist_off, L.plist_idx, L.clist_off, L.clist_idx, world)[rank]
        a, phi = oracle.expansion_forces(sh.group_off, tr.x[sh.s0:sh.s1], tr.x, tr.m, sh.plist_off, sh.plist_idx,
                                         tr.cell_com, tr.cell_m, tr.cell_q, sh.clist_off, sh.clist_idx,
                                         eps2_all=0.02 ** 2)
        part = torch.as_tensor(np.concatenate([a, phi[:, None]], axis=1))
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([part.shape[0]]))
        n_max = int(max(int(v) for v in sizes))
        padded = torch.zeros((n_max, 4), dtype=torch.float64)
        padded[:part.shape[0]] = part
        bufs = [torch.zeros((n_max, 4), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(bufs, padded)
        if rank == 0:
            full = np.concatenate([b[:int(n)].numpy() for b, n in zip(bufs, sizes)])
            q.put(full)
    finally:
        dist.destroy_process_group()


def test_sharded_step_equals_unsharded():
    ps, tr, L = _case()
    costs = shard.group_costs(tr.group_off, L.plist_off, L.clist_off)
    ranges = shard.split_ranges(costs, 2)
    assert ranges[0][0] == 0 and ranges[-1][1] == tr.ngroups and ranges[0][1] == ranges[1][0]
    c0, c1 = costs[:ranges[0][1]].sum(), costs[ranges[0][1]:].sum()
    assert abs(c0 - c1) <= costs.max() + 1e-9 * costs.sum()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_shard, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a, phi = oracle.expansion_forces(tr.group_off, tr.x, tr.x, tr.m, L.plist_off, L.plist_idx, tr.cell_com,
                                     tr.cell_m, tr.cell_q, L.clist_off, L.clist_idx, eps2_all=0.02 ** 2)
    assert full.shape == (tr.n, 4)
    assert np.array_equal(full[:, :3], a) and np.array_equal(full[:, 3], phi)


def _worker_aggregate(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        total_ms, value = bench.aggregate_ranks(100.0 + 50.0 * rank, 10, 1e9, world, dist, "cpu")
        # shards: each rank's own units, added up, over the slowest rank's time
        _, value_s = bench.aggregate_ranks(100.0 + 50.0 * rank, 10, 1e9 * (1 + rank), world, dist, "cpu",
                                           summed=True)
        q.put((rank, total_ms, value, value_s))
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_aggregate, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, total_ms, value, value_s in got:
        assert total_ms == 150.0
        assert value == pytest.approx(2 * 10 * 1e9 / 0.150)
        assert value_s == pytest.approx(10 * 3e9 / 0.150)


def test_split_ranges_edge_cases():
    assert shard.split_ranges(np.ones(5), 1) == [(0, 5)]
    r = shard.split_ranges(np.ones(3), 4)
    assert r[0][0] == 0 and r[-1][1] == 3
    assert all(g0 <= g1 for g0, g1 in r)
    assert sum(g1 - g0 for g0, g1 in r) == 3
    assert shard.split_ranges(np.zeros(0), 2) == [(0, 0), (0, 0)]
