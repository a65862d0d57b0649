"""Weighted graphs (the paper's weighted case: every SSSP a shortest-path
search): gc_greedy_weighted against the oracle's plain weighted greedy
(Dijkstra for every SSSP, pinned to weighted Floyd-Warshall in
test_oracle_pins.py), group and farness bit for bit; unit weights reproduce
gc_greedy; and the weight checks."""
import numpy as np
import pytest

import oracle
from paper_1710_01144_gb300 import graphgen
from tests import smallgraphs as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gcm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1710_01144_gb300 import build, gc

    build.build()
    return gc


def cases():
    out = [("path40", sg.path(40)), ("cycle31", sg.cycle(31)), ("star40", sg.star(40)),
           ("grid7x9", sg.grid(7, 9)), ("cater", sg.caterpillar(9, 3)), ("k12", sg.complete(12))]
    for s in range(3):
        out.append(("ba%d" % s, graphgen.barabasi_albert(500 + 200 * s, 1 + s, s + 11)))
        out.append(("rmat%d" % s, graphgen.rmat(9 + s, 8.0, seed=s + 21)))
        out.append(("road%d" % s, graphgen.grid_road(20 + 6 * s, 25, 0.2, 0.01, s + 31)))
        out.append(("tree%d" % s, sg.tree_random(600, 41 + s)))
    return out


@pytest.mark.parametrize("w_max", [1, 9, 1000])
@pytest.mark.parametrize("name,g", cases())
def test_greedy_weighted_matches_oracle(gcm, name, g, w_max):
    rp, ci = g
    n = rp.size - 1
    k = min(n, 12)
    w = graphgen.edge_weights(rp, ci, w_max, seed=7)
    with gcm.Graph(rp, ci) as G:
        G.set_weights(w, validate=True)
        grp, f, st = G.greedy_weighted(k)
        if w_max == 1:  # unit weights: the unweighted path's group
            g2, f2, _ = G.greedy(k)
            np.testing.assert_array_equal(grp, g2)
            assert f == f2
    want, ft, _ = oracle.wgreedy_plain(rp, ci, w, k)
    np.testing.assert_array_equal(grp, want, err_msg="%s w_max %d" % (name, w_max))
    assert f == ft[-1]
    assert st["rounds"] == k and st["round0_evals"] == n


def test_weighted_config1_size(gcm):
    rp, ci = graphgen.ba_n2000_m5()
    w = graphgen.edge_weights(rp, ci, 16, seed=1)
    with gcm.Graph(rp, ci) as G:
        G.set_weights(w)
        grp, f, st = G.greedy_weighted(10)
    want, ft, _ = oracle.wgreedy_plain(rp, ci, w, 10)
    np.testing.assert_array_equal(grp, want)
    assert f == ft[-1]


def test_weight_checks(gcm):
    rp, ci = sg.grid(6, 7)
    n = rp.size - 1
    with gcm.Graph(rp, ci) as G:
        with pytest.raises(gcm.GcError) as e:
            G.greedy_weighted(3)  # no weights yet
        assert e.value.code == gcm.GC_EINVAL
        w = graphgen.edge_weights(rp, ci, 5, seed=2)
        bad = w.copy()
        bad[3] = 0
        with pytest.raises(gcm.GcError) as e:
            G.set_weights(bad)
        assert e.value.code == gcm.GC_EINVAL
        asym = w.copy()
        asym[0] += 1  # one row of an edge only
        with pytest.raises(gcm.GcError) as e:
            G.set_weights(asym, validate=True)
        assert e.value.code == gcm.GC_EINVAL
        big = np.full(ci.size, (1 << 30) // (n - 1) + 1, np.int32)
        with pytest.raises(gcm.GcError) as e:
            G.set_weights(big)
        assert e.value.code == gcm.GC_ERANGE
        G.set_weights(w)  # usable again
        grp, f, _ = G.greedy_weighted(3)
    want, ft, _ = oracle.wgreedy_plain(rp, ci, w, 3)
    np.testing.assert_array_equal(grp, want)
    assert f == ft[-1]
