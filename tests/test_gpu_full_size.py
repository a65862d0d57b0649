"""Parity at the full sizes of the evaluation workloads where the plain oracle
cannot run the whole greedy: sampled outputs the oracle computes one by one
(exact gains by full BFS, group farness), plus the full greedy where CPU
Greedy++ finishes in reasonable time."""
import numpy as np
import pytest

import oracle
from paper_1710_01144_gb300 import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gcm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1710_01144_gb300 import build, gc

    build.build()
    return gc


def _sampled(gcm, rp, ci, seed, n_group, n_cand):
    n = rp.size - 1
    rng = np.random.default_rng(seed)
    deg = np.diff(rp)
    # groups mixing high-degree and random vertices, candidates spread over the graph
    S = np.unique(np.concatenate([np.argsort(-deg)[:2], rng.choice(n, size=n_group, replace=False)])).astype(np.int32)
    cand = np.concatenate([rng.choice(n, size=n_cand, replace=False), S[:2], np.argsort(-deg)[2:6]]).astype(np.int32)
    with gcm.Graph(rp, ci) as G:
        assert G.farness(S) == oracle.farness(rp, ci, S)
        got = G.gains(S, cand)
    np.testing.assert_array_equal(got, oracle.gains(rp, ci, S, cand))


def test_road_grid_2048_sampled_gains(gcm):
    """Road-like 2048 x 2048 grid (20% of edges deleted, 1% diagonals, LCC):
    deep BFS (thousands of levels) through the 64-lane kernel."""
    rp, ci = graphgen.road_grid_2048()
    assert rp.size - 1 > 4_000_000
    _sampled(gcm, rp, ci, seed=3, n_group=6, n_cand=58)


def test_road_grid_192_greedy(gcm):
    """A 192 x 192 road-like grid (deep BFS, large pruned regions), whole
    greedy (k=12) against CPU Greedy++."""
    rp, ci = graphgen.grid_road(192, 192, 0.2, 0.01, 1)
    grp, ft, _, _ = oracle.greedypp(rp, ci, 12)
    with gcm.Graph(rp, ci) as G:
        got, f, _ = G.greedy(12)
    np.testing.assert_array_equal(got, grp)
    assert f == ft[-1]


def test_rmat24_sampled_gains(gcm):
    """R-MAT scale 24, edge factor 16 (about 10M vertices, 0.5G entries)."""
    rp, ci = graphgen.rmat_s24_ef16()
    assert rp.size - 1 > 5_000_000
    _sampled(gcm, rp, ci, seed=5, n_group=4, n_cand=60)


def test_mixed_batch_subset_vs_oracle(gcm):
    """The 48 smallest graphs of the mixed 256-graph workload, solved in one
    batched launch, against CPU Greedy++ graph by graph."""
    items = sorted(graphgen.batch_params(256, seed=1), key=lambda it: it.n_target)[:48]
    graphs = [graphgen.batch_graph(it) for it in items]
    ks = [min(it.k, rp.size - 1) for it, (rp, _) in zip(items, graphs)]
    with gcm.Batch(graphs) as B:
        groups, far, _ = B.greedy(ks, capture=True)
    for (rp, ci), k, got, f in zip(graphs, ks, groups, far):
        g, ft, _, _ = oracle.greedypp(rp, ci, k)
        np.testing.assert_array_equal(got, g)
        assert f == ft[-1]


def _golden(name):
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, _, val = line.partition(" ")
        out[key] = val.split()
    return out


def _csr_sha256(rp, ci):
    import hashlib

    h = hashlib.sha256()
    h.update(rp.astype("<i4").tobytes())
    h.update(ci.astype("<i4").tobytes())
    return h.hexdigest()


def test_greedy_rmat24_k50_full_size(gcm):
    """R-MAT scale 24, edge factor 16 (8.86M vertices, 521M entries), k = 50:
    the whole group and its farness against CPU Greedy++, whose answer is
    stored in tests/golden/rmat24_ef16_k50.txt (written by make_rmat24_k50.py,
    which calls only the oracle).  The graph must be the one the oracle saw.
    Default launch configuration, then the host-driven lazy steps, then the
    64-lane round 0."""
    gold = _golden("rmat24_ef16_k50.txt")
    rp, ci = graphgen.rmat_s24_ef16()
    assert rp.size - 1 == int(gold["n"][0]) and ci.size == int(gold["nnz"][0])
    assert _csr_sha256(rp, ci) == gold["sha256"][0]
    grp = np.array([int(x) for x in gold["group"]], dtype=np.int32)
    ft = np.array([int(x) for x in gold["farness"]], dtype=np.int64)
    with gcm.Graph(rp, ci) as G:
        for kw in ({}, {"step_mode": 1, "eval_per_step": 128}, {"round0_lanes": -1}, {"r0_probe": False}):
            got, f, st = G.greedy(50, **kw)
            np.testing.assert_array_equal(got, grp)
            assert f == ft[-1]
            if not kw:  # the persistent rounds' d_S updates come from the claim log (up to overflow)
                assert 0 < st["lazy_log_picks"] <= 48
                assert st["r0_probe_cut"] > 0  # the far-vertex probe cut round-0 lanes
        # the farness of the first ten picks, recomputed by one oracle BFS
        assert G.farness(grp[:10]) == ft[9] == oracle.farness(rp, ci, grp[:10])


def test_mixed_batch_all_256_vs_oracle(gcm):
    """The whole 256-graph mixed workload (25M vertices) in one batched launch,
    replayed from a captured CUDA graph, against CPU Greedy++'s answers stored
    in tests/golden/batch256_groups.txt (written by make_batch256.py, which
    calls only the oracle)."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch256_groups.txt")
    gold = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        d = {f[j]: f[j + 1] for j in range(3, 13, 2)}
        gold.append((int(d["n"]), int(d["nnz"]), int(d["k"]), d["sha256"], int(d["farness"]),
                     np.array([int(x) for x in f[f.index("group") + 1:]], dtype=np.int32)))
    assert len(gold) == 256
    items = graphgen.batch_params(256, seed=1)
    graphs = [graphgen.batch_graph(it) for it in items]
    for (rp, ci), (n, nnz, k, sha, _, _) in zip(graphs, gold):
        assert rp.size - 1 == n and ci.size == nnz and _csr_sha256(rp, ci)[:32] == sha
    ks = [g[2] for g in gold]
    with gcm.Batch(graphs) as B:
        for _ in range(2):  # record, then replay the captured graph
            groups, far, st = B.greedy(ks, capture=True)
            for i, (got, g) in enumerate(zip(groups, gold)):
                np.testing.assert_array_equal(got, g[5], err_msg="graph %d" % i)
                assert far[i] == g[4]
        assert st["graph_replay"] == 1
