"""Host logic of the width tuner (autotune.tune_gain_lanes) on the CPU, with a
stand-in for the graph handle: it keeps the fastest width by the gain
kernel's device time, refuses a width whose gains differ, caches the choice
by workload shape, and leaves the handle at the winning width."""
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
