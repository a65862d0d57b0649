"""bitGreedy++ (Sec. 4.3, Theorem 1) on the GPU: gc_greedy_bits scores every
vertex every round by bit vectors and must return exactly the oracle's group
and farness (smallest-id ties), across chunk boundaries of the target bit
vectors (64 W targets per chunk, W <= 32 words) and for k up to n."""
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
    out = [("path50", sg.path(50)), ("cycle31", sg.cycle(31)), ("star40", sg.star(40)),
           ("grid7x9", sg.grid(7, 9)), ("cater", sg.caterpillar(9, 3)), ("k12", sg.complete(12)),
           ("path64", sg.path(64)), ("path65", sg.path(65)), ("tree2047", sg.tree_random(2047, 3)),
           ("tree2049", sg.tree_random(2049, 4))]
    for s in range(3):
        out.append(("ba%d" % s, graphgen.barabasi_albert(700 + 300 * s, 1 + s, s + 11)))
        out.append(("rmat%d" % s, graphgen.rmat(11 + s, 8.0, seed=s + 21)))
        out.append(("road%d" % s, graphgen.grid_road(40 + 9 * s, 50, 0.2, 0.01, s + 31)))
    return out


@pytest.mark.parametrize("name,g", cases())
def test_greedy_bits_matches_oracle(gcm, name, g):
    rp, ci = g
    n = rp.size - 1
    k = min(n, 24)
    grp, f, st = None, None, None
    with gcm.Graph(rp, ci) as G:
        grp, f, st = G.greedy_bits(k)
        g2, f2, _ = G.greedy(k)
    want, ft, _, _ = oracle.greedypp(rp, ci, k)
    np.testing.assert_array_equal(grp, want, err_msg=name)
    assert f == ft[-1]
    np.testing.assert_array_equal(g2, grp)  # the same group as the pruned-SSSP path
    assert st["rounds"] == k


def test_greedy_bits_config1(gcm):
    """The BA n = 2000, m = 5, k = 10 workload in full."""
    rp, ci = graphgen.ba_n2000_m5()
    with gcm.Graph(rp, ci) as G:
        grp, f, st = G.greedy_bits(10)
    want, ft, _ = oracle.greedy_plain(rp, ci, 10)
    np.testing.assert_array_equal(grp, want)
    assert f == ft[-1]


def test_greedy_bits_all_vertices_and_limits(gcm):
    rp, ci = sg.grid(9, 11)
    n = rp.size - 1
    with gcm.Graph(rp, ci) as G:
        grp, f, _ = G.greedy_bits(n)  # every vertex: the farness reaches 0
        assert f == 0 and sorted(grp.tolist()) == list(range(n))
        np.testing.assert_array_equal(grp, oracle.greedy_plain(rp, ci, n)[0])
        with pytest.raises(gcm.GcError) as e:
            G.greedy_bits(0)
        assert e.value.code == gcm.GC_EINVAL
    big = sg.path(65537)
    with gcm.Graph(*big) as G:
        with pytest.raises(gcm.GcError) as e:
            G.greedy_bits(2)
        assert e.value.code == gcm.GC_ERANGE
