"""Pins of the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
closed form, the paper's worked example (tests/golden), an independent
all-pairs computation (Floyd-Warshall in numpy, no BFS), brute force, or an
invariant the paper proves (supermodularity of farness, Sec. 3.2; Theorem 1,
Sec. 4.3; pruning and laziness leave the greedy result unchanged, Sec. 4.1-4.2).
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1710_01144_gb300 import graphgen
from tests import smallgraphs as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------- independent ---
def apsp_fw(rp, ci):
    """All-pairs distances by Floyd-Warshall on the adjacency matrix."""
    n = rp.size - 1
    D = np.full((n, n), 10**9, dtype=np.int64)
    np.fill_diagonal(D, 0)
    for u in range(n):
        for k in range(rp[u], rp[u + 1]):
            D[u, ci[k]] = 1
    for m in range(n):
        D = np.minimum(D, D[:, m:m + 1] + D[m:m + 1, :])
    return D


def greedy_by_definition(D, k):
    """Greedy on farness from the distance matrix; ties to the smallest id."""
    n = D.shape[0]
    f1 = D.sum(axis=1)
    s0 = int(np.argmin(f1))  # argmin returns the first (smallest id) minimiser
    group, dS = [s0], D[s0].copy()
    trace = [int(dS.sum())]
    for _ in range(1, k):
        best, best_f = -1, None
        for v in range(n):
            if v in group:
                continue
            f = int(np.minimum(dS, D[v]).sum())
            if best_f is None or f < best_f:
                best, best_f = v, f
        group.append(best)
        dS = np.minimum(dS, D[best])
        trace.append(best_f)
    return group, trace


def path_group_farness(n, group):
    s = sorted(group)
    f = s[0] * (s[0] + 1) // 2 + (n - 1 - s[-1]) * (n - s[-1]) // 2
    for a, b in zip(s, s[1:]):
        g = b - a - 1
        f += (g + 1) ** 2 // 4
    return f


# ---------------------------------------------------------- closed forms ---
@pytest.mark.parametrize("n", [2, 3, 7, 10, 33])
def test_path_single_vertex_farness_and_s0(n):
    rp, ci = sg.path(n)
    for v in range(n):
        assert oracle.farness(rp, ci, [v]) == v * (v + 1) // 2 + (n - 1 - v) * (n - v) // 2
    g, ft, _ = oracle.greedy_plain(rp, ci, 1)
    assert g[0] == (n - 1) // 2


@pytest.mark.parametrize("n,k", [(10, 3), (17, 4), (40, 6)])
def test_path_group_farness_closed_form(n, k):
    rp, ci = sg.path(n)
    rng = np.random.default_rng(n * 31 + k)
    for _ in range(20):
        S = sorted(rng.choice(n, size=k, replace=False).tolist())
        assert oracle.farness(rp, ci, S) == path_group_farness(n, S)
    g, ft, _ = oracle.greedy_plain(rp, ci, k)
    for i in range(k):
        assert ft[i] == path_group_farness(n, g[: i + 1].tolist())


@pytest.mark.parametrize("n", [3, 4, 9, 16])
def test_cycle(n):
    rp, ci = sg.cycle(n)
    for v in range(n):
        assert oracle.farness(rp, ci, [v]) == n * n // 4
    g, _, _ = oracle.greedy_plain(rp, ci, 1)
    assert g[0] == 0


@pytest.mark.parametrize("n", [3, 6, 12])
def test_star(n):
    rp, ci = sg.star(n)
    assert oracle.farness(rp, ci, [0]) == n - 1
    for v in range(1, n):
        assert oracle.farness(rp, ci, [v]) == 2 * n - 3
    k = n - 1
    g, ft, gt = oracle.greedy_plain(rp, ci, k)
    assert g.tolist() == list(range(k))
    assert gt[1:].tolist() == [1] * (k - 1)
    assert ft.tolist() == [n - 1 - i for i in range(k)]


@pytest.mark.parametrize("a,b", [(3, 4), (5, 5), (2, 9)])
def test_grid_single_vertex(a, b):
    rp, ci = sg.grid(a, b)

    def T(m, i):
        return i * (i + 1) // 2 + (m - 1 - i) * (m - i) // 2

    for i in range(a):
        for j in range(b):
            assert oracle.farness(rp, ci, [i * b + j]) == b * T(a, i) + a * T(b, j)


@pytest.mark.parametrize("n", [2, 5, 8])
def test_complete(n):
    rp, ci = sg.complete(n)
    g, ft, gt = oracle.greedy_plain(rp, ci, n)
    assert g.tolist() == list(range(n))
    assert ft.tolist() == [n - 1 - i for i in range(n)]
    assert gt[1:].tolist() == [1] * (n - 1)


def test_k5_worked_example_golden():
    """Sec. 3.2: K5 closeness values printed by the paper."""
    rp, ci = sg.complete(5)
    rows = [l for l in open(os.path.join(GOLDEN, "k5_worked_example.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 4
    for row in rows:
        grp, num, den = row.strip().split("|")
        S = [int(x) for x in grp.split(",")]
        # c(S) = n / sum_{w not in S} d(S,w); members contribute 0 to f(S)
        assert Fraction(5, oracle.farness(rp, ci, S)) == Fraction(int(num), int(den))
    # the paper's inequality: c(S+v)-c(S) = 5/6 < c(T+v)-c(T) = 5/2
    c = lambda S: Fraction(5, oracle.farness(rp, ci, S))
    assert c([0, 1, 3]) - c([0, 1]) == Fraction(5, 6)
    assert c([0, 1, 2, 3]) - c([0, 1, 2]) == Fraction(5, 2)


# ------------------------------------------------ brute force / FW checks ---
def tiny_graphs():
    out = [("path9", sg.path(9)), ("cycle8", sg.cycle(8)), ("star7", sg.star(7)),
           ("grid3x4", sg.grid(3, 4)), ("cater", sg.caterpillar(4, 2)), ("k6", sg.complete(6))]
    for s in range(8):
        out.append(("gnp%d" % s, sg.gnp_connected(12 + s, 0.15, s)))
        out.append(("tree%d" % s, sg.tree_random(14 + s, 100 + s)))
    out.append(("ba20", graphgen.barabasi_albert(20, 2, 3)))
    return out


@pytest.mark.parametrize("name,g", tiny_graphs())
def test_bfs_matches_floyd_warshall(name, g):
    rp, ci = g
    D = apsp_fw(rp, ci)
    for s in range(rp.size - 1):
        assert (oracle.bfs(rp, ci, [s]) == D[s]).all()


@pytest.mark.parametrize("name,g", tiny_graphs())
def test_greedy_plain_matches_definition(name, g):
    rp, ci = g
    n = rp.size - 1
    k = min(6, n)
    D = apsp_fw(rp, ci)
    grp, trace = greedy_by_definition(D, k)
    g1, ft, gt = oracle.greedy_plain(rp, ci, k)
    assert g1.tolist() == grp
    assert ft.tolist() == trace
    assert gt[0] == trace[0]
    assert gt[1:].tolist() == [trace[i - 1] - trace[i] for i in range(1, k)]


@pytest.mark.parametrize("name,g", tiny_graphs()[:10])
def test_opt_bruteforce(name, g):
    rp, ci = g
    n = rp.size - 1
    D = apsp_fw(rp, ci)
    for k in (1, 2, 3):
        best = min(int(D[list(S)].min(axis=0).sum()) for S in itertools.combinations(range(n), k))
        f, grp = oracle.opt_bruteforce(rp, ci, k)
        assert f == best
        assert int(D[grp].min(axis=0).sum()) == f
        _, ft, _ = oracle.greedy_plain(rp, ci, k)
        assert ft[-1] >= f  # greedy can never beat the optimum


@pytest.mark.parametrize("name,g", tiny_graphs())
def test_gain_identities(name, g):
    """Delta(v|S) = f(S) - f(S+v) (two independent farness BFSs), = Theorem 1's
    popcount sum, = the distance-matrix form; >= 1 off S and 0 on S."""
    rp, ci = g
    n = rp.size - 1
    D = apsp_fw(rp, ci)
    rng = np.random.default_rng(n)
    for trial in range(3):
        S = sorted(rng.choice(n, size=1 + trial, replace=False).tolist())
        gains = oracle.gains(rp, ci, S, np.arange(n))
        bits = oracle.gains_bitparallel(rp, ci, S)
        dS = D[S].min(axis=0)
        fS = oracle.farness(rp, ci, S)
        for v in range(n):
            expect = int(np.maximum(0, dS - D[v]).sum())
            assert gains[v] == expect == bits[v]
            if v in S:
                assert gains[v] == 0
            else:
                assert gains[v] >= 1
                assert gains[v] == fS - oracle.farness(rp, ci, S + [v])


def test_supermodularity_invariant():
    """Sec. 3.2 lemma: S subset of T, v not in T => Delta(v|T) <= Delta(v|S)."""
    rng = np.random.default_rng(7)
    graphs = [graphgen.barabasi_albert(300, 3, 5), graphgen.rmat(9, 8.0, seed=4),
              graphgen.grid_road(15, 15, 0.2, 0.01, 2), sg.gnp_connected(40, 0.08, 9)]
    checks = 0
    for rp, ci in graphs:
        n = rp.size - 1
        for _ in range(40):
            T = rng.choice(n, size=int(rng.integers(2, 8)), replace=False)
            S = T[: int(rng.integers(1, T.size))]
            cand = np.setdiff1d(np.arange(n), T)
            gS = oracle.gains(rp, ci, S, cand)
            gT = oracle.gains(rp, ci, T, cand)
            assert (gT <= gS).all()
            checks += cand.size
    assert checks > 10000


# ------------------------------------ Greedy++ (O2) equals plain greedy ---
def o2_cases():
    out = [("path50", sg.path(50)), ("cycle31", sg.cycle(31)), ("star40", sg.star(40)),
           ("grid7x9", sg.grid(7, 9)), ("cater", sg.caterpillar(9, 3)), ("k12", sg.complete(12))]
    for s in range(4):
        out.append(("ba%d" % s, graphgen.barabasi_albert(400 + 50 * s, 1 + s, s + 11)))
        out.append(("rmat%d" % s, graphgen.rmat(9 + s % 3, 6.0, seed=s + 21)))
        out.append(("road%d" % s, graphgen.grid_road(20 + 3 * s, 17, 0.2, 0.01, s + 31)))
        out.append(("tree%d" % s, sg.tree_random(300, 41 + s)))
    return out


@pytest.mark.parametrize("name,g", o2_cases())
def test_greedypp_equals_plain(name, g):
    rp, ci = g
    n = rp.size - 1
    k = min(12, n)
    a = oracle.greedy_plain(rp, ci, k)
    b = oracle.greedypp(rp, ci, k)
    for x, y in zip(a, b[:3]):
        assert (x == y).all(), name


def test_greedypp_config1_equals_plain():
    """The small evaluation workload (BA n=2000, m=5, k=10) in full."""
    rp, ci = graphgen.ba_n2000_m5()
    a = oracle.greedy_plain(rp, ci, 10)
    b = oracle.greedypp(rp, ci, 10)
    for x, y in zip(a, b[:3]):
        assert (x == y).all()


@pytest.mark.parametrize("name,g", o2_cases())
def test_top1_closeness(name, g):
    rp, ci = g
    n = rp.size - 1
    f = [oracle.farness(rp, ci, [v]) for v in range(n)]
    s0, f0, _ = oracle.top1_closeness(rp, ci)
    assert s0 == int(np.argmin(f)) and f0 == min(f)


# --------------------------- top-k closeness (Sec. 3.1, Algorithm 3, k > 1) ---
def topk_by_definition(f, k):
    """The k smallest (farness, id) pairs of a list of single-vertex farness values."""
    order = sorted(range(len(f)), key=lambda v: (f[v], v))[:k]
    return np.array(order, dtype=np.int32), np.array([f[v] for v in order], dtype=np.int64)


@pytest.mark.parametrize("name,g", o2_cases())
def test_topk_closeness_equals_sorted_farness(name, g):
    rp, ci = g
    n = rp.size - 1
    if n <= 500:  # farness from Floyd-Warshall row sums: no BFS code involved
        f = [int(x) for x in apsp_fw(rp, ci).sum(axis=1)]
    else:         # the plain BFS farness, itself pinned to Floyd-Warshall above
        f = [oracle.farness(rp, ci, [v]) for v in range(n)]
    for k in sorted({1, 2, 5, 17, n // 3 or 1, n}):
        if k > n:
            continue
        ids, fk, _ = oracle.topk_closeness(rp, ci, k)
        want_ids, want_f = topk_by_definition(f, k)
        np.testing.assert_array_equal(ids, want_ids, err_msg="%s k=%d" % (name, k))
        np.testing.assert_array_equal(fk, want_f, err_msg="%s k=%d" % (name, k))


@pytest.mark.parametrize("n", [9, 20, 33])
def test_topk_closeness_closed_forms(n):
    # path: f(v) = v(v+1)/2 + (n-1-v)(n-v)/2, smallest around the middle
    rp, ci = sg.path(n)
    f = [v * (v + 1) // 2 + (n - 1 - v) * (n - v) // 2 for v in range(n)]
    ids, fk, _ = oracle.topk_closeness(rp, ci, 5)
    np.testing.assert_array_equal(ids, topk_by_definition(f, 5)[0])
    np.testing.assert_array_equal(fk, topk_by_definition(f, 5)[1])
    # cycle: every vertex has floor(n^2/4), so the k smallest ids
    rp, ci = sg.cycle(n)
    ids, fk, _ = oracle.topk_closeness(rp, ci, 4)
    assert ids.tolist() == [0, 1, 2, 3] and (fk == n * n // 4).all()
    # star with centre 0: n-1, then leaves at 2n-3 in id order
    rp, ci = sg.star(n)
    ids, fk, _ = oracle.topk_closeness(rp, ci, 3)
    assert ids.tolist() == [0, 1, 2] and fk.tolist() == [n - 1, 2 * n - 3, 2 * n - 3]


def test_topk_closeness_k1_and_threads():
    rp, ci = graphgen.rmat(12, 8.0, seed=5)
    s0, f0, _ = oracle.top1_closeness(rp, ci)
    ids, fk, _ = oracle.topk_closeness(rp, ci, 1)
    assert ids.tolist() == [s0] and fk.tolist() == [f0]
    a = oracle.topk_closeness(rp, ci, 40, threads=1)
    b = oracle.topk_closeness(rp, ci, 40, threads=4)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    with pytest.raises(ValueError):
        oracle.topk_closeness(rp, ci, 0)
    with pytest.raises(ValueError):
        oracle.topk_closeness(rp, ci, rp.size)


# ------------------------------------- weighted graphs (Sec. 3.2, Dijkstra) ---
def apsp_fw_weighted(rp, ci, w):
    """All-pairs weighted distances by Floyd-Warshall on the weight matrix."""
    n = rp.size - 1
    D = np.full((n, n), 10**15, dtype=np.int64)
    np.fill_diagonal(D, 0)
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            D[u, ci[e]] = min(D[u, ci[e]], int(w[e]))
    for m in range(n):
        D = np.minimum(D, D[:, m:m + 1] + D[m:m + 1, :])
    return D


@pytest.mark.parametrize("name,g", o2_cases())
def test_weighted_with_unit_weights_is_unweighted(name, g):
    rp, ci = g
    n = rp.size - 1
    w = np.ones(ci.size, np.int32)
    k = min(8, n)
    a = oracle.greedy_plain(rp, ci, k)
    b = oracle.wgreedy_plain(rp, ci, w, k)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y, err_msg=name)
    S = [0, n - 1] if n > 1 else [0]
    cand = list(range(0, n, max(1, n // 40)))
    np.testing.assert_array_equal(oracle.wgains(rp, ci, w, S, cand), oracle.gains(rp, ci, S, cand))


@pytest.mark.parametrize("name,g", tiny_graphs())
def test_weighted_matches_floyd_warshall(name, g):
    rp, ci = g
    n = rp.size - 1
    for seed in (1, 2):
        w = graphgen.edge_weights(rp, ci, 9, seed)
        D = apsp_fw_weighted(rp, ci, w)
        for v in range(n):
            np.testing.assert_array_equal(oracle.dijkstra(rp, ci, w, v), D[v], err_msg=name)
        S = [v for v in range(0, n, 3)][:3]
        dS = D[S].min(axis=0)
        assert oracle.wfarness(rp, ci, w, S) == int(dS.sum())
        want = [int(np.maximum(0, dS - D[v]).sum()) for v in range(n)]
        np.testing.assert_array_equal(oracle.wgains(rp, ci, w, S, list(range(n))), want)
        k = min(5, n)
        grp, tr = greedy_by_definition(D, k)
        g2, ft, _ = oracle.wgreedy_plain(rp, ci, w, k)
        assert g2.tolist() == grp and ft.tolist() == tr, name


@pytest.mark.parametrize("n", [5, 12, 30])
def test_weighted_path_closed_form(n):
    rp, ci = sg.path(n)
    w = graphgen.edge_weights(rp, ci, 7, n)
    P = np.zeros(n, np.int64)  # P[i] = distance from vertex 0 along the path
    for i in range(1, n):
        e = next(e for e in range(rp[i], rp[i + 1]) if ci[e] == i - 1)
        P[i] = P[i - 1] + int(w[e])
    for v in (0, n // 2, n - 1):
        assert oracle.wfarness(rp, ci, w, [v]) == int(np.abs(P - P[v]).sum())
    f = [int(np.abs(P - P[v]).sum()) for v in range(n)]
    g, ft, _ = oracle.wgreedy_plain(rp, ci, w, 1)
    assert g[0] == int(np.argmin(f)) and ft[0] == min(f)


def test_weighted_scaling_and_supermodularity():
    rp, ci = graphgen.rmat(9, 6.0, seed=3)
    n = rp.size - 1
    w = graphgen.edge_weights(rp, ci, 12, 5)
    g1, f1, t1 = oracle.wgreedy_plain(rp, ci, w, 6)
    g3, f3, t3 = oracle.wgreedy_plain(rp, ci, 3 * w, 6)
    np.testing.assert_array_equal(g1, g3)
    np.testing.assert_array_equal(3 * f1, f3)
    rng = np.random.default_rng(7)
    checks = 0
    for _ in range(60):
        T = rng.choice(n, size=6, replace=False)
        S = T[:3]
        v = rng.integers(0, n, size=20)
        a = oracle.wgains(rp, ci, w, S, v)
        b = oracle.wgains(rp, ci, w, T, v)
        assert (b <= a).all()
        checks += v.size
    assert checks >= 1000


def test_errors():
    rp, ci = sg.disjoint_union(sg.path(3), sg.path(4))
    with pytest.raises(ValueError):
        oracle.farness(rp, ci, [0])
    with pytest.raises(ValueError):
        oracle.greedy_plain(rp, ci, 2)
    rp, ci = sg.path(5)
    with pytest.raises(ValueError):
        oracle.farness(rp, ci, [])
    with pytest.raises(ValueError):
        oracle.gains(rp, ci, [9], [0])
