"""Host logic of the tuners in autotune.py on the CPU, with stand-ins for the
graph handle and the batch: each keeps the fastest setting, refuses one that
changes a result, and caches its choice by workload shape; the width tuner
also leaves the handle at the winning width."""
import numpy as np
import pytest

from paper_1710_01144_gb300 import autotune


class FakeGraph:
    """Answers gains(S, cand, stats=...) like gc.Graph, with a kernel time per
    width from `ms` and the same gains at every width unless `bad` names one."""

    def __init__(self, ms, bad=None, n=1000, nnz=8000):
        self.ms, self.bad, self.n, self.nnz = ms, bad, n, nnz
        self.lanes, self.calls, self.log = 64, 0, []

    def set_gain_lanes(self, lanes):
        assert lanes in (64, 128, 256)
        self.lanes = lanes
        self.log.append(lanes)

    def gains(self, S, cand, stats=False):
        self.calls += 1
        g = np.arange(np.size(cand), dtype=np.int64) + int(np.size(S))
        if self.bad == self.lanes:
            g = g + 1
        return (g, {"ms_gain_kernel": self.ms[self.lanes]}) if stats else g


def test_picks_fastest_and_caches(tmp_path):
    cache = str(tmp_path / "t.json")
    G = FakeGraph({64: 3.0, 128: 2.0, 256: 5.0})
    best, entry = autotune.tune_gain_lanes(G, [1, 2], np.arange(500), reps=2, cache=cache)
    assert best == {"gain_lanes": 128} and G.lanes == 128
    assert [t["gain_lanes"] for t in entry["trials"]] == [64, 128, 256]
    assert [t["ms"] for t in entry["trials"]] == [3.0, 2.0, 5.0]
    calls = G.calls
    # a new handle of the same shape: answered from the cache, no gains run
    H = FakeGraph({64: 1.0, 128: 9.0, 256: 9.0})
    again, _ = autotune.tune_gain_lanes(H, [7, 8], np.arange(500), cache=cache)
    assert again == best and H.calls == 0 and H.lanes == 128
    # another shape (candidate count) is tuned afresh
    again2, _ = autotune.tune_gain_lanes(H, [7, 8], np.arange(600), cache=cache)
    assert again2 == {"gain_lanes": 64} and H.lanes == 64
    assert G.calls == calls


def test_refuses_a_width_that_changes_a_gain(tmp_path):
    G = FakeGraph({64: 3.0, 128: 2.0, 256: 1.0}, bad=256)
    with pytest.raises(RuntimeError, match="changed a gain"):
        autotune.tune_gain_lanes(G, [1], np.arange(10), reps=1, cache=str(tmp_path / "t.json"))


def test_no_cache_file(tmp_path):
    G = FakeGraph({64: 1.0, 128: 2.0, 256: 3.0})
    best, _ = autotune.tune_gain_lanes(G, [1], np.arange(10), reps=1, cache=None, space=(256, 64))
    assert best == {"gain_lanes": 64} and G.lanes == 64 and G.log[:2] == [256, 64]


class FakeSolver:
    """greedy(...) of a graph handle or a batch: the same answer for every
    setting unless `bad` names one, and a time per setting in `ms`."""

    def __init__(self, ms, bad=None, n=100, nnz=800):
        self.ms, self.bad, self.n, self.nnz, self.last = ms, bad, n, nnz, None

    def greedy(self, k, **kw):
        self.last = tuple(sorted(kw.items()))
        wrong = self.bad is not None and all(kw.get(a) == b for a, b in self.bad.items())
        if isinstance(k, list):  # a batch: one group per graph
            groups = [np.arange(x) + (1 if wrong else 0) for x in k]
            return groups, np.array(k, dtype=np.int64), {}
        return np.arange(k) + (1 if wrong else 0), 10 * k, {}


def _fake_time(monkeypatch, solver):
    def timed(fn, reps):
        out = fn()
        return solver.ms[solver.last], out
    monkeypatch.setattr(autotune, "_time", timed)


def test_tune_single_picks_fastest_and_caches(monkeypatch, tmp_path):
    space = [{"active_target": a, "round1_heavy": h} for a in (512, 2048) for h in (256, 1024)]
    ms = {tuple(sorted(c.items())): 5.0 for c in space}
    ms[(("active_target", 2048), ("round1_heavy", 256))] = 1.0
    G = FakeSolver(ms)
    _fake_time(monkeypatch, G)
    cache = str(tmp_path / "t.json")
    best, entry = autotune.tune_single(G, 7, cache=cache, space=space)
    assert best == {"active_target": 2048, "round1_heavy": 256} and len(entry["trials"]) == 4
    G.ms = {}  # from the cache: nothing is timed again
    assert autotune.tune_single(G, 7, cache=cache, space=space)[0] == best


def test_tune_single_refuses_a_setting_that_changes_the_group(monkeypatch, tmp_path):
    space = [{"active_target": 512, "round1_heavy": 256}, {"active_target": 2048, "round1_heavy": 256}]
    G = FakeSolver({tuple(sorted(c.items())): 1.0 for c in space}, bad={"active_target": 2048})
    _fake_time(monkeypatch, G)
    with pytest.raises(RuntimeError, match="changed the group"):
        autotune.tune_single(G, 5, cache=str(tmp_path / "t.json"), space=space)


def test_tune_batch_picks_fastest(monkeypatch, tmp_path):
    space = [{"lanes": l, "A": a} for l in (32, 64) for a in (256, 4096)]
    ms = {(("active_target", c["A"]), ("lanes", c["lanes"])): 3.0 for c in space}
    ms[(("active_target", 4096), ("lanes", 32))] = 0.5
    B = FakeSolver(ms)
    _fake_time(monkeypatch, B)
    best, entry = autotune.tune_batch(B, [3, 4], [100, 200], cache=str(tmp_path / "t.json"), space=space)
    assert best == {"lanes": 32, "A": 4096} and len(entry["trials"]) == 4
    B2 = FakeSolver(ms, bad={"lanes": 64})
    _fake_time(monkeypatch, B2)
    with pytest.raises(RuntimeError, match="changed a group"):
        autotune.tune_batch(B2, [3, 4], [100, 201], cache=str(tmp_path / "t.json"), space=space)
