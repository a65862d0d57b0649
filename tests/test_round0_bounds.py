"""The round-0 lower bounds on f({v}) that decide which BFScut searches are
cut (Sec. 3.1, Algorithm 3), checked on the CPU against the oracle's exact
distances.

After the levels up to d of a search from v are known (cnt vertices within
distance d, their distance sum s), every other vertex is at distance >= d + 1,
so f({v}) >= s + (d + 1)(n - cnt).  The bottom-up kernel also learns, for some
of the others, that they are at distance >= d + 2 (their whole row holds no
vertex at distance d): with `far` of them,
    f({v}) >= s + (d + 1)(n - cnt - far) + (d + 2) far,
for any such subset.  The degree bound of the survivor filter is the d = 1
form with the two-hop count in place of the vertices at distance 2:
    LB(v) = deg + 2 c2 + 3 (n - 1 - deg - c2),
    c2 = min(sum_{w in N(v)} (deg(w) - 1), n - 1 - deg).
The tests take the distances from the oracle's BFS, restate the bounds, and
check that none exceeds the exact farness, that the far form equals the
exact farness when every vertex beyond d + 1 is exactly at d + 2 and every
one of them is counted, and that the cut (bound > best) never removes the
top-1 vertex."""
import numpy as np
import pytest

import oracle
from paper_1710_01144_gb300 import graphgen
from tests import smallgraphs as sg


def cases():
    return [("path40", sg.path(40)), ("cycle31", sg.cycle(31)), ("star30", sg.star(30)), ("grid9x13", sg.grid(9, 13)),
            ("cater", sg.caterpillar(12, 3)), ("k9", sg.complete(9)), ("tree", sg.tree_random(400, 3)),
            ("gnp", sg.gnp_connected(150, 0.03, 5)), ("ba", graphgen.barabasi_albert(600, 3, 7)),
            ("rmat10", graphgen.rmat(10, 8.0, seed=3)), ("rmat12", graphgen.rmat(12, 16.0, seed=1)),
            ("road", graphgen.grid_road(30, 27, 0.2, 0.01, 5))]


def far_bound(dist, d, far):
    """s + (d + 1)(n - cnt - far) + (d + 2) far for the levels up to d."""
    n = dist.size
    near = dist <= d
    s, cnt = int(dist[near].sum()), int(near.sum())
    return s + (d + 1) * (n - cnt - far) + (d + 2) * far


@pytest.mark.parametrize("name,g", cases())
def test_far_vertex_bound_is_a_lower_bound(name, g):
    rp, ci = g
    n = rp.size - 1
    rng = np.random.default_rng(11)
    for v in rng.choice(n, size=min(n, 25), replace=False):
        dist = oracle.bfs(rp, ci, [int(v)]).astype(np.int64)
        f = int(dist.sum())
        assert f == oracle.farness(rp, ci, [int(v)])
        ecc = int(dist.max())
        for d in range(1, ecc + 1):
            beyond = int((dist >= d + 2).sum())
            prev = None
            # any number of the vertices at distance >= d + 2 may have been proven so far
            for far in sorted({0, beyond // 3, beyond // 2, beyond}):
                b = far_bound(dist, d, far)
                assert b <= f
                if prev is not None:
                    assert b >= prev  # each proven vertex raises the bound by one
                prev = b
            # every vertex at distance >= d + 2 proven, none beyond d + 2: the bound is exact
            if int((dist >= d + 3).sum()) == 0:
                assert far_bound(dist, d, beyond) == f
            # without far vertices: the plain BFScut bound after level d
            assert far_bound(dist, d, 0) == int(dist[dist <= d].sum()) + (d + 1) * int((dist > d).sum())


@pytest.mark.parametrize("name,g", cases())
def test_degree_bound_and_cuts_keep_the_top1_vertex(name, g):
    rp, ci = g
    n = rp.size - 1
    deg = np.diff(rp).astype(np.int64)
    two_hop = np.add.reduceat(deg[ci] - 1, rp[:-1].astype(np.int64)) if ci.size else np.zeros(n, np.int64)
    two_hop[deg == 0] = 0
    rest = n - 1 - deg
    c2 = np.minimum(two_hop, rest)
    lb = deg + 2 * c2 + 3 * (rest - c2)
    s0, f0, _ = oracle.top1_closeness(rp, ci)
    far_all = np.array([int(oracle.bfs(rp, ci, [v]).astype(np.int64).sum()) for v in range(n)])
    assert far_all.min() == f0 and int(np.argmin(far_all)) == s0
    assert np.all(lb <= far_all)
    # the cut rule (bound > best, ties kept) at any level with any proven subset
    # never drops s0 while the best farness found is at least f0
    dist = oracle.bfs(rp, ci, [s0]).astype(np.int64)
    for d in range(1, int(dist.max()) + 1):
        beyond = int((dist >= d + 2).sum())
        for far in (0, beyond):
            assert not (far_bound(dist, d, far) > f0)
