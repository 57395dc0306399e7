"""The schedule autotuner's search, on a stand-in handle (no GPU): it times
every candidate of each knob group through the handle's own setters, keeps
the fastest, leaves the handle with it, and caches the pick per graph
signature."""
import numpy as np

from paper_2507_11094_gb300 import autotune


class FakeStats:
    def __init__(self, ms):
        self.ms_total = ms


class FakeGraph:
    """Times a 'solve' from the current knobs with a cost model that has one
    best point: delta 4x the mean weight, pool 64, small 32, local 1024."""

    def __init__(self, n=1000, m=16000):
        self.n, self.m = n, m
        self.delta = self.pool = self.local = 0
        self.small = 8
        self.solves = 0

    def set_delta(self, d):
        self.delta = d

    def set_schedule(self, small, pool):
        self.small, self.pool = small, pool

    def set_local_rounds(self, e):
        self.local = e

    def solve(self, stats=False):
        self.solves += 1
        cost = (10.0 + abs(self.delta - 200) / 50 + (0 if self.pool == 64 else 3)
                + (0 if self.small == 32 else 1) + (0 if self.local == 1024 else 0.5))
        return FakeStats(cost) if stats else None


def test_tuner_finds_the_best_point_and_caches_it():
    autotune._cache.clear()
    w = np.full(16000, 50, dtype=np.int32)          # mean weight 50 -> 4x = 200
    g = FakeGraph()
    res = autotune.tune_schedule(g, lambda h, stats=False: h.solve(stats), w, reps=1)
    assert res["schedule"] == {"delta": 200, "pool_rounds": 64, "small_deg": 32,
                               "local_edges": 1024}
    assert (g.delta, g.pool, g.small, g.local) == (200, 64, 32, 1024)
    # every timed candidate is reported, the best one among them
    best = min(res["ms"], key=res["ms"].get)
    assert best == "delta=200,pool=64,small=32,local=1024"
    # a second handle of the same graph takes the cached pick after one solve
    g2 = FakeGraph()
    res2 = autotune.tune_schedule(g2, lambda h, stats=False: h.solve(stats), w, reps=1)
    assert res2["schedule"] == res["schedule"] and g2.solves == 1
    assert (g2.delta, g2.pool, g2.small, g2.local) == (200, 64, 32, 1024)


def test_candidates_scale_with_the_mean_weight():
    assert autotune.candidates(np.array([], dtype=np.int32)) == [0]
    c = autotune.candidates(np.full(10, 500, dtype=np.int32))
    assert c == [0, 500, 1000, 2000, 8000, 32000]
