"""Batched solving: many graphs of uneven size and k in one persistent launch
(optionally replayed from a captured CUDA graph).  Every graph's group must
equal the CPU oracle's on that graph alone."""
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


def mixed_batch():
    graphs = [graphgen.barabasi_albert(800 + 97 * i, 1 + i % 4, 10 + i) for i in range(6)]
    graphs += [graphgen.rmat(9 + i % 4, 4.0 + 3 * i, seed=20 + i) for i in range(6)]
    graphs += [sg.path(30), sg.star(25), sg.cycle(17), sg.grid(6, 9), sg.caterpillar(7, 2), sg.complete(5),
               graphgen.grid_road(25, 31, 0.2, 0.01, 4)]
    ks = [1 + (7 * i) % 23 for i in range(len(graphs))]
    ks = [min(k, rp.size - 1) for k, (rp, _) in zip(ks, graphs)]
    ks[0], ks[1] = 1, 2  # the round-0-only and round-1-only cases
    return graphs, ks


def oracle_groups(graphs, ks):
    out = []
    for (rp, ci), k in zip(graphs, ks):
        g, ft, _, _ = oracle.greedypp(rp, ci, k)
        out.append((g, int(ft[-1])))
    return out


def test_batch_matches_oracle(gcm):
    graphs, ks = mixed_batch()
    ref = oracle_groups(graphs, ks)
    with gcm.Batch(graphs) as B:
        # grid_min_n: 1 = every graph's lazy rounds grid-wide, -1 = all CTA-local;
        # bound: round 1 from two-hop bounds (default) or over every vertex
        for act, lanes, gmin, bound in ((0, 0, 0, True), (2, 16, 1, True), (64, 64, -1, True), (0, 0, 1, True),
                                        (0, 0, 0, False), (2, 16, 1, False)):
            groups, far, st = B.greedy(ks, active_target=act, lanes=lanes, grid_min_n=gmin, round1_bound=bound)
            for i, ((g, f), got) in enumerate(zip(ref, groups)):
                np.testing.assert_array_equal(got, g, err_msg="graph %d (act %d, gmin %d, bound %s)"
                                              % (i, act, gmin, bound))
                assert far[i] == f


def test_batch_capture_replay(gcm):
    graphs, ks = mixed_batch()
    ref = oracle_groups(graphs, ks)
    with gcm.Batch(graphs) as B:
        for call in range(3):
            groups, far, st = B.greedy(ks, capture=True)
            assert st["graph_replay"] == 1
            for (g, f), got, ff in zip(ref, groups, far):
                np.testing.assert_array_equal(got, g)
                assert ff == f
        # changing ks re-captures
        ks2 = [max(1, k - 1) for k in ks]
        ref2 = oracle_groups(graphs, ks2)
        groups, far, st = B.greedy(ks2, capture=True)
        for (g, f), got in zip(ref2, groups):
            np.testing.assert_array_equal(got, g)


def test_batch_errors(gcm):
    graphs, ks = mixed_batch()
    with gcm.Batch(graphs[:3]) as B:
        with pytest.raises(gcm.GcError) as e:
            B.greedy([0, 1, 1])
        assert e.value.code == gcm.GC_EINVAL
    rp, ci = sg.disjoint_union(sg.path(3), sg.path(3))
    with gcm.Batch([rp, ci] and [(rp, ci), sg.path(4)]) as B:
        with pytest.raises(gcm.GcError) as e:
            B.greedy([1, 1])
        assert e.value.code == gcm.GC_EDISCONNECTED


def test_autotune_batch(gcm, tmp_path):
    from paper_1710_01144_gb300 import autotune

    graphs, ks = mixed_batch()
    sizes = [rp.size - 1 for rp, _ in graphs]
    cache = str(tmp_path / "tune.json")
    space = [{"lanes": 64, "A": 1024}, {"lanes": 16, "A": 4}]
    with gcm.Batch(graphs) as B:
        best, entry = autotune.tune_batch(B, ks, sizes, reps=1, cache=cache, space=space)
        assert best in [{"lanes": s["lanes"], "A": s["A"]} for s in space]
        assert len(entry["trials"]) == 2
        again, _ = autotune.tune_batch(B, ks, sizes, cache=cache, space=space)  # from the cache
        assert again == best


def test_greedy_batch_over_handles(gcm):
    """gc_greedy_batch: the batched solve over graphs already loaded as handles
    (host-copied and adopted device arrays mixed); each group equals the
    oracle's, and the handles still answer on their own afterwards."""
    import torch

    graphs, ks = mixed_batch()
    ref = oracle_groups(graphs, ks)
    handles, keep = [], []
    for i, (rp, ci) in enumerate(graphs):
        if i % 3 == 2:  # adopted device arrays
            trp, tci = torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda()
            keep.append((trp, tci))
            handles.append(gcm.Graph(trp, tci, adopt=True))
        else:
            handles.append(gcm.Graph(rp, ci))
    try:
        for _ in range(2):
            groups, far, _ = gcm.greedy_batch(handles, ks)
            for (g, f), got, fv in zip(ref, groups, far):
                np.testing.assert_array_equal(got, g)
                assert fv == f
        got, f, _ = handles[3].greedy(ks[3])
        np.testing.assert_array_equal(got, ref[3][0])
        bad = list(ks)
        bad[4] = graphs[4][0].size  # k > n
        with pytest.raises(gcm.GcError) as e:
            gcm.greedy_batch(handles, bad)
        assert e.value.code == gcm.GC_EINVAL
    finally:
        for G in handles:
            G.close()
