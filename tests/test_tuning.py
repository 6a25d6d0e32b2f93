"""Host logic of the group-size tuner on GPU-built trees (tuning.tune_group_size_gpu),
with the tree and the force context replaced by fakes that report given
device times: the candidate with the shortest whole step (tree build + walk +
force step) wins, a tie on the force step alone is broken by the tree's time,
every candidate is built and walked twice before its timing is read, and the
winner's tree is left built."""
import pytest

from paper_1812_07313_gb300 import tuning

# n_crit -> (build ms, walk ms, force step ms, groups)
TIMES = {64: (7.3, 14.8, 24.00, 517), 128: (7.3, 8.4, 24.01, 280), 256: (7.1, 5.2, 25.20, 158)}


class FakeTree:
    def __init__(self):
        self.calls = []
        self.n_crit = None

    def build(self, x, m, sys_off, leaf_max, n_crit, stream=None):
        self.calls.append(("build", n_crit))
        self.n_crit = n_crit

    def walk(self, theta, stream=None):
        self.calls.append(("walk", self.n_crit))

    def timing(self):
        b, w, _, _ = TIMES[self.n_crit]
        return b, w

    def sizes(self):
        return {"ngroups": TIMES[self.n_crit][3]}

    def attach(self, ctx, eps2_all, stream=None):
        ctx.n_crit = self.n_crit


class FakeContext:
    closed = 0

    def __init__(self, device, options=None):
        self.n_crit = None

    def qg_autotune(self, stream=None, reps=2):
        pass

    def qg_run(self, stream=None):
        pass

    def qg_last_timing(self):
        f = TIMES[self.n_crit][2]
        return f + 0.05, f

    def qg_get_stats(self):
        return {"i_pp": 1, "i_pc": 2, "sinks_per_thread": 4, "sinks_adaptive": 0, "warps_per_group": 2,
                "tile_j": 256, "paired": 2}

    def close(self):
        FakeContext.closed += 1


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(tuning.qgrav, "Context", FakeContext)
    FakeContext.closed = 0
    return FakeTree()


def test_whole_step_decides(fakes):
    best, table = tuning.tune_group_size_gpu(fakes, None, None, None, 8, 0.5, [64, 128, 256])
    whole = {r.n_crit: r.step_ms + r.tree_ms for r in table}
    assert whole[256] < whole[128] < whole[64]
    assert best.n_crit == 256
    # by the force step alone 64 would have won
    assert min(table, key=lambda r: r.step_ms).n_crit == 64
    assert [r.tree_ms for r in table] == [pytest.approx(TIMES[c][0] + TIMES[c][1]) for c in (64, 128, 256)]
    assert FakeContext.closed == 3


def test_each_candidate_built_twice_and_winner_left_built(fakes):
    best, _ = tuning.tune_group_size_gpu(fakes, None, None, None, 8, 0.5, [256, 64, 128])
    assert best.n_crit == 256
    for c in (64, 128, 256):
        assert fakes.calls.count(("build", c)) >= 2 and fakes.calls.count(("walk", c)) >= 2
    # the last candidate was 128, so the winner's tree is built and walked again at the end
    assert fakes.calls[-2:] == [("build", 256), ("walk", 256)]
    assert fakes.n_crit == 256


def test_force_step_tie_broken_by_tree_time(fakes, monkeypatch):
    monkeypatch.setitem(TIMES, 256, (7.1, 9.0, 24.00, 158))
    best, _ = tuning.tune_group_size_gpu(fakes, None, None, None, 8, 0.5, [64, 128, 256])
    assert best.n_crit == 128  # 24.01 + 15.7 beats 24.00 + 22.1 and 24.00 + 16.1
