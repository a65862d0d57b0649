"""Top-k closeness (Sec. 3.1, Algorithm 3 with general k) on the GPU:
gc_top_closeness against the CPU oracle's Algorithm 3 (itself pinned to sorted
Floyd-Warshall farness in test_oracle_pins.py), ids and farness values bit for
bit, for every search path (wide bottom-up batches, 64-lane CTA batches,
grid-wide batches) and k from 1 to n.  Also the overlap of the greedy group
with the top-k closeness and top-k degree sets (Sec. 6.5's comparison)."""
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
           ("grid7x9", sg.grid(7, 9)), ("cater", sg.caterpillar(9, 3)), ("k12", sg.complete(12))]
    for s in range(3):
        out.append(("ba%d" % s, graphgen.barabasi_albert(600 + 150 * s, 1 + s, s + 11)))
        out.append(("rmat%d" % s, graphgen.rmat(10 + s, 8.0, seed=s + 21)))
        out.append(("road%d" % s, graphgen.grid_road(30 + 5 * s, 23, 0.2, 0.01, s + 31)))
        out.append(("tree%d" % s, sg.tree_random(700, 41 + s)))
    return out


@pytest.mark.parametrize("name,g", cases())
def test_top_closeness_matches_oracle(gcm, name, g):
    rp, ci = g
    n = rp.size - 1
    with gcm.Graph(rp, ci) as G:
        for k in sorted({1, 2, 5, 17, 64, 65, max(1, n // 3), n}):
            if k > n:
                continue
            ids, f, st = G.top_closeness(k)
            want_ids, want_f, _ = oracle.topk_closeness(rp, ci, k)
            np.testing.assert_array_equal(ids, want_ids, err_msg="%s k=%d" % (name, k))
            np.testing.assert_array_equal(f, want_f, err_msg="%s k=%d" % (name, k))


def test_top1_is_greedy_s0(gcm):
    rp, ci = graphgen.rmat(13, 16.0, seed=3)
    with gcm.Graph(rp, ci) as G:
        ids, f, _ = G.top_closeness(1)
        grp, _, _ = G.greedy(1)
    assert ids[0] == grp[0]
    assert f[0] == oracle.farness(rp, ci, [int(grp[0])])


@pytest.mark.parametrize("lanes", [-1, 0, 64, 256])
def test_top_closeness_search_paths(gcm, lanes):
    """Shallow R-MAT graphs: the wide bottom-up batches (64 or 256 lanes, also
    with every level in full), the 64-lane path (-1) and the automatic choice."""
    for rp, ci in (graphgen.rmat(15, 16.0, seed=7), graphgen.rmat(16, 8.0, seed=9)):
        with gcm.Graph(rp, ci) as G:
            for k in (10, 100, 300):
                want_ids, want_f, _ = oracle.topk_closeness(rp, ci, k)
                for full in (False, True) if lanes > 0 else (False,):
                    ids, f, st = G.top_closeness(k, round0_lanes=lanes, r0_full_levels=full)
                    np.testing.assert_array_equal(ids, want_ids, err_msg="lanes %d k %d" % (lanes, k))
                    np.testing.assert_array_equal(f, want_f)
                    if lanes > 0:
                        assert st["r0_width"] in (0, lanes)


def test_top_closeness_errors(gcm):
    rp, ci = sg.path(10)
    with gcm.Graph(rp, ci) as G:
        for k in (0, 11):
            with pytest.raises(gcm.GcError) as e:
                G.top_closeness(k)
            assert e.value.code == gcm.GC_EINVAL
        ids, f, _ = G.top_closeness(10)  # the handle stays usable
        np.testing.assert_array_equal(ids, oracle.topk_closeness(rp, ci, 10)[0])


@pytest.mark.parametrize("which", ["ba2000_k10", "rmat16_k50"])
def test_group_vs_topk_overlap(gcm, which):
    """How many members of the greedy group are also among the k most central
    vertices by closeness and by degree (the paper compares these sets on its
    graphs).  The greedy group's first member is the top-1 closeness vertex;
    the counts are printed for the record."""
    if which == "ba2000_k10":
        (rp, ci), k = graphgen.ba_n2000_m5(), 10
    else:
        (rp, ci), k = graphgen.rmat(16, 16.0, seed=1), 50
    deg = np.diff(rp)
    top_deg = set(sorted(range(rp.size - 1), key=lambda v: (-deg[v], v))[:k])
    with gcm.Graph(rp, ci) as G:
        grp, f_grp, _ = G.greedy(k)
        ids, f, _ = G.top_closeness(k)
    want = oracle.topk_closeness(rp, ci, k)
    np.testing.assert_array_equal(ids, want[0])
    grp_set, top_cl = set(grp.tolist()), set(ids.tolist())
    assert grp[0] == ids[0]
    # the group of the k most central vertices is never better than the greedy group here
    f_topk = oracle.farness(rp, ci, ids.tolist())
    print("\n%s: |greedy & top-k closeness| = %d, |greedy & top-k degree| = %d, "
          "|top-k closeness & top-k degree| = %d of k = %d; farness greedy %d, top-k closeness set %d"
          % (which, len(grp_set & top_cl), len(grp_set & top_deg), len(top_cl & top_deg), k, f_grp, f_topk))
    assert f_grp <= f_topk
