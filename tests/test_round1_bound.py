"""The round-1 upper bound used to start the lazy rounds at round 1.

With S = {s0} and d = d(s0, .), every candidate v satisfies
    gain(v|S) <= d[v] + sum_{w in N(v)} ((d[w] - 1)^+ + c3[w]) + sum_u (d[u] - 3)^+,
c3[w] = #{u in N(w): d[u] >= 3} (distance 1 gains at most d - 1; distance 2
at most [d >= 3] + (d - 3)^+ with each such u next to some w in N(v);
farther at most (d - 3)^+).  These tests check the inequality against the
oracle's exact gains, and that neighbours with d <= 1 contribute nothing (the
kernel sums over the pruned rows only)."""
import numpy as np
import pytest

import oracle
from paper_1710_01144_gb300 import graphgen
from tests import smallgraphs as sg


def bound(rp, ci, d, only_pruned_rows=False):
    n = rp.size - 1
    deg = np.diff(rp)
    src = np.repeat(np.arange(n), deg)
    c3 = np.bincount(src, weights=(d[ci] >= 3), minlength=n)
    term = np.maximum(d - 1, 0) + c3
    w = term[ci] * ((d[ci] >= 2) if only_pruned_rows else 1)
    ub = d + np.bincount(src, weights=w, minlength=n) + np.maximum(d - 3, 0).sum()
    ub[d == 0] = -1
    return ub.astype(np.int64)


def cases():
    return [("path40", sg.path(40)), ("cycle31", sg.cycle(31)), ("star30", sg.star(30)), ("grid9x13", sg.grid(9, 13)),
            ("cater", sg.caterpillar(12, 3)), ("k9", sg.complete(9)), ("tree", sg.tree_random(400, 3)),
            ("gnp", sg.gnp_connected(150, 0.03, 5)), ("ba", graphgen.barabasi_albert(600, 3, 7)),
            ("rmat10", graphgen.rmat(10, 8.0, seed=3)), ("road", graphgen.grid_road(30, 27, 0.2, 0.01, 5))]


@pytest.mark.parametrize("name,g", cases())
def test_round1_bound_holds(name, g):
    rp, ci = g
    n = rp.size - 1
    s0 = int(np.asarray(oracle.top1_closeness(rp, ci)).ravel()[0])
    d = oracle.bfs(rp, ci, [s0]).astype(np.int64)
    ub = bound(rp, ci, d)
    cand = np.arange(n)
    gain = np.asarray(oracle.gains(rp, ci, [s0], cand), dtype=np.int64)
    assert gain[s0] == 0 and ub[s0] == -1
    others = cand != s0
    assert (gain[others] <= ub[others]).all()
    # the pruned rows (neighbours with d >= 2) give the same bound
    np.testing.assert_array_equal(bound(rp, ci, d, only_pruned_rows=True), ub)


def test_round1_bound_prunes_rmat():
    """On an R-MAT graph the bound leaves few candidates at or above the best
    exact round-1 gain (the reason round 1 can skip most evaluations)."""
    rp, ci = graphgen.rmat(12, 16.0, seed=1)
    s0 = int(np.asarray(oracle.top1_closeness(rp, ci)).ravel()[0])
    d = oracle.bfs(rp, ci, [s0]).astype(np.int64)
    ub = bound(rp, ci, d)
    top = np.argsort(-ub)[:64]
    gstar = int(np.asarray(oracle.gains(rp, ci, [s0], top)).max())
    assert (ub >= gstar).sum() < 64


@pytest.mark.parametrize("name,g", cases())
def test_two_hop_bound_holds_for_larger_groups(name, g):
    """The same inequality with d, c3 and the (d - 3)^+ sum taken for a group
    of 2 to 5 vertices (the refresh of later rounds)."""
    rp, ci = g
    n = rp.size - 1
    rng = np.random.default_rng(11)
    for size in (2, 3, 5):
        if size >= n:
            continue
        S = rng.choice(n, size=size, replace=False)
        d = oracle.bfs(rp, ci, S).astype(np.int64)
        ub = bound(rp, ci, d)
        gain = np.asarray(oracle.gains(rp, ci, S, np.arange(n)), dtype=np.int64)
        off = d > 0
        assert (gain[off] <= ub[off]).all()
        assert (ub[~off] == -1).all()
        np.testing.assert_array_equal(bound(rp, ci, d, only_pruned_rows=True), ub)
