"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element and bit-exact (all quantities are integers)."""
import numpy as np
import pytest

import oracle
from paper_1710_01144_gb300 import graphgen
from tests import smallgraphs as sg

pytestmark = pytest.mark.gpu

# (eval_per_step, step_lanes, step_mode, active_target) of the lazy rounds:
# defaults (persistent device kernel), host-driven CTA-per-batch steps,
# host-driven grid-wide steps, and the persistent kernel with a tiny active
# list so that it must stop and have the list rebuilt many times
STEP_VARIANTS = [(0, 0, 0, 0), (64, 8, 1, 0), (0, 0, 2, 0), (128, 1, 1, 0), (0, 0, 3, 64), (0, 0, 3, 1)]
# (the neighbour bound is on in all of them; test_greedy_bound_off turns it off)


@pytest.fixture(scope="module")
def gcm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1710_01144_gb300 import build, gc

    build.build()
    return gc


def small_cases():
    return [("path37", sg.path(37)), ("cycle20", sg.cycle(20)), ("star70", sg.star(70)),
            ("grid9x13", sg.grid(9, 13)), ("cater", sg.caterpillar(12, 3)), ("k9", sg.complete(9)),
            ("tree", sg.tree_random(500, 3)), ("gnp", sg.gnp_connected(150, 0.03, 5)),
            ("ba", graphgen.barabasi_albert(700, 3, 7)), ("rmat10", graphgen.rmat(10, 8.0, seed=3)),
            ("road", graphgen.grid_road(40, 33, 0.2, 0.01, 5))]


@pytest.mark.parametrize("name,g", small_cases())
def test_farness(gcm, name, g):
    rp, ci = g
    n = rp.size - 1
    rng = np.random.default_rng(1)
    with gcm.Graph(rp, ci, validate=True) as G:
        for size in (1, 2, 5, min(17, n)):
            S = rng.choice(n, size=size, replace=False)
            assert G.farness(S) == oracle.farness(rp, ci, S)
        assert G.farness([0, 0, 0]) == oracle.farness(rp, ci, [0])


@pytest.mark.parametrize("name,g", small_cases())
def test_gains_all_candidates(gcm, name, g):
    rp, ci = g
    n = rp.size - 1
    rng = np.random.default_rng(2)
    with gcm.Graph(rp, ci) as G:
        for size in (1, 3, 8):
            S = rng.choice(n, size=min(size, n), replace=False)
            cand = np.arange(n, dtype=np.int32)
            np.testing.assert_array_equal(G.gains(S, cand), oracle.gains(rp, ci, S, cand))


def test_gains_ragged_repeats_members(gcm):
    rp, ci = graphgen.barabasi_albert(3000, 4, 11)
    n = rp.size - 1
    rng = np.random.default_rng(3)
    S = rng.choice(n, size=6, replace=False)
    with gcm.Graph(rp, ci) as G:
        for m in (0, 1, 63, 64, 65, 129, 1000, 4097):
            cand = rng.integers(0, n, size=m).astype(np.int32)
            if m > 3:
                cand[:3] = S[:3]  # members -> 0
                cand[3] = cand[4]  # a repeat
            got = G.gains(S, cand)
            assert got.shape == (m,)
            np.testing.assert_array_equal(got, oracle.gains(rp, ci, S, cand))
        # more candidates than vertices (chunked)
        cand = rng.integers(0, n, size=2 * n + 5).astype(np.int32)
        np.testing.assert_array_equal(G.gains(S, cand), oracle.gains(rp, ci, S, cand))


@pytest.mark.parametrize("name,g", small_cases())
def test_greedy_equals_plain_oracle(gcm, name, g):
    rp, ci = g
    n = rp.size - 1
    k = min(12, n)
    grp, ft, _ = oracle.greedy_plain(rp, ci, k)
    with gcm.Graph(rp, ci) as G:
        for eps, lanes, mode, act in STEP_VARIANTS:
            got, f, st = G.greedy(k, eval_per_step=eps, step_lanes=lanes, step_mode=mode, active_target=act)
            np.testing.assert_array_equal(got, grp)
            assert f == ft[-1]
            assert st["rounds"] == k


@pytest.mark.parametrize("name,g", small_cases() + [("rmat13", graphgen.rmat(13, 16.0, seed=4))])
def test_round1_bound_same_group(gcm, name, g):
    """Round 1 with the two-hop bounds (the 64 largest first, then every
    candidate whose bound reaches the best exact gain) returns the oracle's
    group, as the every-vertex round 1 does; on R-MAT it evaluates far fewer
    candidates."""
    rp, ci = g
    k = min(12, rp.size - 1)
    grp, ft, _ = oracle.greedy_plain(rp, ci, k)
    with gcm.Graph(rp, ci) as G:
        a, fa, sa = G.greedy(k)
        b, fb, sb = G.greedy(k, round1_bound=False)
    np.testing.assert_array_equal(a, grp)
    np.testing.assert_array_equal(b, grp)
    assert fa == fb == ft[-1]
    if name == "rmat13":
        assert sa["evals"] * 2 < sb["evals"]


@pytest.mark.parametrize("n", [37, 64, 101])
def test_round0_deep_graphs_repeated(gcm, n):
    """Round 0 (top-1 closeness) on paths and cycles, many times over: the
    grid-wide BFScut batches run dozens of levels, one barrier each, and every
    CTA must take the same cut decisions at every level (a lane that some CTAs
    cut and others keep ends short of n and reads as a disconnected graph).
    Closed forms: f({v}) on a path = v(v+1)/2 + (n-1-v)(n-v)/2, minimised at
    (n-1)//2; on a cycle every vertex has floor(n^2/4), so s0 = 0."""
    v = (n - 1) // 2
    cases = [(sg.path(n), v, v * (v + 1) // 2 + (n - 1 - v) * (n - v) // 2), (sg.cycle(n), 0, n * n // 4)]
    for (rp, ci), s0, f0 in cases:
        with gcm.Graph(rp, ci) as G:
            for _ in range(40):
                grp, f, _ = G.greedy(1)
                assert int(grp[0]) == s0 and f == f0


@pytest.mark.parametrize("name,g", small_cases())
def test_greedy_step_forms(gcm, name, g):
    """Persistent rounds with wide steps (a 64-lane batch per CTA) or grid-wide
    steps, each with every d_S update on one CTA or always grid-wide, and with
    the automatic choice."""
    rp, ci = g
    k = min(12, rp.size - 1)
    grp, ft, _ = oracle.greedy_plain(rp, ci, k)
    with gcm.Graph(rp, ci) as G:
        for form, local, pruned in ((2, 1 << 30, True), (1, -1, True), (2, -1, False), (1, 1 << 30, False),
                                    (0, 4096, True)):
            got, f, _ = G.greedy(k, step_form=form, local_update_max_gain=local, pruned_adjacency=pruned)
            np.testing.assert_array_equal(got, grp)
            assert f == ft[-1]


@pytest.mark.parametrize("name,g", small_cases() + [("rmat13", graphgen.rmat(13, 16.0, seed=4))])
def test_greedy_claim_log(gcm, name, g):
    """d_S updates of the persistent rounds from the claim log of the pick's
    gain batch, against the relabel BFS from the pick: the oracle's group and
    farness, and the same number of lowered labels (the same vertices).  With
    grid-wide steps every pick of rounds >= 2 comes from the log, also across
    the relaunches that rebuild a tiny active list; a log capped at 16 entries
    mixes both updates; wide steps (the automatic form on deep graphs) keep no
    log.  The host checks every update's decrease against the pick's gain."""
    rp, ci = g
    k = min(12, rp.size - 1)
    grp, ft, _ = oracle.greedy_plain(rp, ci, k)
    relabels = set()
    with gcm.Graph(rp, ci) as G:
        for form, act, log, cap in ((1, 0, False, 0), (1, 0, True, 0), (1, 64, True, 0), (1, 1, True, 0),
                                    (1, 0, True, 16), (2, 0, True, 0), (0, 0, True, 0)):
            got, f, st = G.greedy(k, step_form=form, active_target=act, step_mode=3 if act else 0,
                                  claim_log=log, claim_log_cap=cap)
            np.testing.assert_array_equal(got, grp)
            assert f == ft[-1]
            relabels.add(st["lazy_upd_relabels"])
            picks = st["lazy_log_picks"]
            if not log or form == 2:
                assert picks == 0, (form, act, log, cap, picks)
            elif form == 1 and cap == 0:
                assert picks == max(0, k - 2), (form, act, log, cap, picks)
            else:  # a capped log, or the automatic form (wide steps on deep graphs)
                assert picks in range(max(0, k - 2) + 1), (form, act, log, cap, picks)
            if picks == max(0, k - 2) and k > 2:
                assert st["lazy_upd_frontier"] == 0  # no relabel BFS ran
    assert len(relabels) == 1


@pytest.mark.parametrize("name,g", small_cases())
def test_greedy_bound_off(gcm, name, g):
    rp, ci = g
    n = rp.size - 1
    k = min(12, n)
    grp, ft, _ = oracle.greedy_plain(rp, ci, k)
    with gcm.Graph(rp, ci) as G:
        got, f, st = G.greedy(k, expand_bound=False, round1_heavy=-1)
        np.testing.assert_array_equal(got, grp)
        assert f == ft[-1]


def test_greedy_ba2000_k10(gcm):
    """The small evaluation workload: BA n=2000, m=5, seed 1, k=10."""
    rp, ci = graphgen.ba_n2000_m5()
    grp, ft, _ = oracle.greedy_plain(rp, ci, 10)
    with gcm.Graph(rp, ci, validate=True) as G:
        got, f, _ = G.greedy(10)
    np.testing.assert_array_equal(got, grp)
    assert f == ft[-1]


@pytest.mark.parametrize("scale,k", [(12, 30), (14, 40)])
def test_greedy_rmat_vs_greedypp(gcm, scale, k):
    rp, ci = graphgen.rmat(scale, 16.0, seed=5)
    grp, ft, _, _ = oracle.greedypp(rp, ci, k)
    with gcm.Graph(rp, ci) as G:
        for eps, lanes, mode, act in STEP_VARIANTS + [(1024, 64, 1, 0)]:
            got, f, _ = G.greedy(k, eval_per_step=eps, step_lanes=lanes, step_mode=mode, active_target=act,
                                 round1_heavy=-1 if mode == 1 else 0)
            np.testing.assert_array_equal(got, grp)
            assert f == ft[-1]


def test_greedy_rmat20_k100_full_size(gcm):
    """R-MAT scale 20 (ef 16, seed 1), k = 100: the benchmark workload, in the
    benchmark's launch configuration, against CPU Greedy++ (itself pinned to
    the plain oracle).  Prefixes are the k = 10 and k = 50 answers."""
    rp, ci = graphgen.rmat_s20_ef16()
    grp, ft, _, _ = oracle.greedypp(rp, ci, 100)
    with gcm.Graph(rp, ci) as G:
        got, f, st = G.greedy(100)
        np.testing.assert_array_equal(got, grp)
        assert f == ft[-1]
        assert st["lazy_log_picks"] == 98  # every d_S update of rounds 2..99 from the claim log
        g1, f1, s1 = G.greedy(100, claim_log=False)
        np.testing.assert_array_equal(g1, grp)
        assert f1 == ft[-1] and s1["lazy_log_picks"] == 0
        assert s1["lazy_upd_relabels"] == st["lazy_upd_relabels"]
        for mode, heavy, bound, form, local, pruned in ((1, -1, False, 0, 0, True), (2, 64, True, 0, 0, False),
                                                        (3, 4096, True, 1, -1, True), (3, 0, False, 2, 1 << 30, False)):
            g2, f2, _ = G.greedy(100, step_mode=mode, round1_heavy=heavy, expand_bound=bound,
                                 step_form=form, local_update_max_gain=local, pruned_adjacency=pruned)
            np.testing.assert_array_equal(g2, grp)
            assert f2 == ft[-1]
        # farness of the prefixes by the library's own BFS, against the trace
        for kk in (10, 50):
            assert G.farness(got[:kk]) == ft[kk - 1]
        # sampled exact gains at full size
        rng = np.random.default_rng(9)
        cand = rng.integers(0, rp.size - 1, size=300).astype(np.int32)
        np.testing.assert_array_equal(G.gains(got[:10], cand), oracle.gains(rp, ci, got[:10], cand))


def test_errors(gcm):
    rp, ci = sg.path(10)
    with gcm.Graph(rp, ci) as G:
        for bad in (0, 11, -1):
            with pytest.raises(gcm.GcError) as e:
                G.greedy(bad)
            assert e.value.code == gcm.GC_EINVAL
        with pytest.raises(gcm.GcError) as e:
            G.farness([10])
        assert e.value.code == gcm.GC_EINVAL
        with pytest.raises(gcm.GcError) as e:
            G.gains([], [1])
        assert e.value.code == gcm.GC_EINVAL
        with pytest.raises(gcm.GcError) as e:
            G.gains([1], [12])
        assert e.value.code == gcm.GC_EINVAL
        assert G.greedy(10)[1] == 0  # k = n: every vertex in the group
    rp, ci = sg.disjoint_union(sg.path(4), sg.cycle(5))
    with pytest.raises(gcm.GcError) as e:
        gcm.Graph(rp, ci, validate=True)
    assert e.value.code == gcm.GC_EDISCONNECTED
    with gcm.Graph(rp, ci) as G:
        with pytest.raises(gcm.GcError) as e:
            G.farness([0])
        assert e.value.code == gcm.GC_EDISCONNECTED
        with pytest.raises(gcm.GcError) as e:
            G.greedy(2)
        assert e.value.code == gcm.GC_EDISCONNECTED
    # malformed CSR: asymmetric edge, self-loop, unsorted row, bad row_ptr
    bad = [
        (np.array([0, 1, 1], np.int32), np.array([1], np.int32)),
        (np.array([0, 2, 3], np.int32), np.array([0, 1, 0], np.int32)),
        (np.array([0, 2, 3, 4], np.int32), np.array([2, 1, 0, 0], np.int32)),
        (np.array([0, 2, 1, 3], np.int32), np.array([1, 2, 0], np.int32)),
    ]
    for rp, ci in bad:
        with pytest.raises(gcm.GcError) as e:
            gcm.Graph(rp, ci, validate=True)
        assert e.value.code == gcm.GC_EINVAL


def test_device_pointers_and_adopt(gcm):
    import torch

    rp, ci = graphgen.rmat(11, 8.0, seed=8)
    n = rp.size - 1
    trp = torch.from_numpy(rp).cuda()
    tci = torch.from_numpy(ci).cuda()
    S = np.array([0, 5, 9], np.int32)
    cand = np.arange(n, dtype=np.int32)
    ref = oracle.gains(rp, ci, S, cand)
    for adopt in (False, True):
        with gcm.Graph(trp, tci, validate=True, adopt=adopt) as G:
            out = torch.empty(n, dtype=torch.int64, device="cuda")
            G.gains_device(torch.from_numpy(S).cuda(), torch.from_numpy(cand).cuda(), out)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("name,g", small_cases())
def test_upper_bounds_match_restatement(gcm, name, g):
    """gc_gain_upper_bounds element by element against the numpy restatement of
    the two-hop bound (tests/test_round1_bound.py), for groups of 1 to 5
    vertices: one vertex goes through the round-1 kernel, larger groups through
    the refresh kernels of later rounds.  The restatement itself is checked
    against the oracle's exact gains on CPU."""
    from tests.test_round1_bound import bound

    rp, ci = g
    n = rp.size - 1
    rng = np.random.default_rng(17)
    with gcm.Graph(rp, ci) as G:
        for size in (1, 2, 3, 5):
            if size >= n:
                continue
            S = rng.choice(n, size=size, replace=False).astype(np.int32)
            d = oracle.bfs(rp, ci, S).astype(np.int64)
            np.testing.assert_array_equal(G.upper_bounds(S), bound(rp, ci, d))


def test_wait_expiry_returns_timeout_and_handle_stays_usable(gcm):
    """Every device-side wait has a time limit.  With a limit of 1 us the grid
    barriers of a deep graph's BFS levels cannot all be met: the call returns
    GC_ETIMEOUT (no fault, no hang), and the next call on the same handle with
    the default limit returns the oracle's group."""
    rp, ci = sg.path(6000)
    grp, ft, _ = oracle.greedy_plain(rp, ci, 3)
    with gcm.Graph(rp, ci) as G:
        for _ in range(2):
            with pytest.raises(gcm.GcError) as e:
                G.greedy(3, timeout_us=1)
            assert e.value.code == gcm.GC_ETIMEOUT
            got, f, _ = G.greedy(3)
            np.testing.assert_array_equal(got, grp)
            assert f == ft[-1]


def round0_cases():
    return [("ba20000m1", graphgen.barabasi_albert(20000, 1, 5)), ("gnp400", sg.gnp_connected(400, 0.02, 3)),
            ("ba3000m2", graphgen.barabasi_albert(3000, 2, 3)), ("tree", sg.tree_random(900, 3)),
            ("rmat12", graphgen.rmat(12, 16.0, seed=1)), ("star70", sg.star(70)), ("k9", sg.complete(9))]


@pytest.mark.parametrize("name,g", round0_cases() + [("rmat14", graphgen.rmat(14, 16.0, seed=2)),
                                                     ("rmat15", graphgen.rmat(15, 16.0, seed=3))])
@pytest.mark.parametrize("lanes", [64, 256])
def test_round0_probe_on_off(gcm, name, g, lanes):
    """Round 0 with and without the far-vertex probe before the count-only
    distance-2 pass (vertices proven at distance >= 3 raise the BFScut bound
    and cut lanes early): the oracle's s0 and farness, its top-5 closeness,
    and the same group."""
    rp, ci = g
    s0, f0, _ = oracle.top1_closeness(rp, ci)
    k = 3
    grp, ft, _, _ = oracle.greedypp(rp, ci, k)
    ids, fs, _ = oracle.topk_closeness(rp, ci, 5)
    with gcm.Graph(rp, ci) as G:
        for probe in (True, False):
            got, f, st = G.greedy(k, round0_lanes=lanes, r0_probe=probe)
            np.testing.assert_array_equal(got, grp)
            assert f == ft[-1]
            if not probe:
                assert st["r0_probes"] == 0
            got1, f1, _ = G.greedy(1, round0_lanes=lanes, r0_probe=probe)
            assert got1[0] == s0 and f1 == f0
            ti, tf = G.top_closeness(5, round0_lanes=lanes, r0_probe=probe)[:2]
            np.testing.assert_array_equal(ti, ids)
            np.testing.assert_array_equal(tf, fs)


@pytest.mark.parametrize("name,g", round0_cases())
@pytest.mark.parametrize("lanes", [64, 128, 256, 512, -1])
def test_round0_wide_lane_widths(gcm, name, g, lanes):
    """Round 0 (top-1 closeness, BFScut) by the wide bottom-up kernel at every
    batch width, and by the 64-lane path (-1): the same s0 and farness as the
    oracle, then the same group.  The 20,000-vertex tree leaves every vertex a
    survivor of the degree bound, so many batches and deferred lanes run."""
    rp, ci = g
    s0, f0, _ = oracle.top1_closeness(rp, ci)
    k = 4
    grp, ft, _, _ = oracle.greedypp(rp, ci, k)
    assert grp[0] == s0 and ft[0] == f0
    with gcm.Graph(rp, ci) as G:
        got, f, st = G.greedy(k, round0_lanes=lanes)
        np.testing.assert_array_equal(got, grp)
        assert f == ft[-1]
        if lanes > 0 and name == "ba20000m1":
            assert st["r0_batches"] >= 2
        got1, f1, _ = G.greedy(1, round0_lanes=lanes)
        assert got1[0] == s0 and f1 == f0


# ---- gain kernel at 128 and 256 candidates per batch (gc_set_gain_lanes) ----

@pytest.mark.parametrize("lanes", [128, 256])
@pytest.mark.parametrize("name,g", small_cases())
def test_gains_wide_lanes(gcm, name, g, lanes):
    """Two or four lane words per vertex: the same exact gains as the oracle's
    full BFS for every candidate, groups of 1, 3 and 8 vertices."""
    rp, ci = g
    n = rp.size - 1
    rng = np.random.default_rng(2)
    with gcm.Graph(rp, ci) as G:
        G.set_gain_lanes(lanes)
        for size in (1, 3, 8):
            S = rng.choice(n, size=min(size, n), replace=False)
            cand = np.arange(n, dtype=np.int32)
            np.testing.assert_array_equal(G.gains(S, cand), oracle.gains(rp, ci, S, cand))


@pytest.mark.parametrize("lanes", [128, 256])
def test_gains_wide_ragged_repeats_members(gcm, lanes):
    """Partial last batches, members of S, a repeated candidate inside one
    batch, more candidates than vertices, and the width switched back and
    forth on one handle."""
    rp, ci = graphgen.barabasi_albert(3000, 4, 11)
    n = rp.size - 1
    rng = np.random.default_rng(3)
    S = rng.choice(n, size=6, replace=False)
    with gcm.Graph(rp, ci) as G:
        for m in (0, 1, 127, 128, 129, 255, 256, 257, 1000, 4097):
            G.set_gain_lanes(lanes)
            cand = rng.integers(0, n, size=m).astype(np.int32)
            if m > 3:
                cand[:3] = S[:3]
                cand[3] = cand[4]
            ref = oracle.gains(rp, ci, S, cand)
            np.testing.assert_array_equal(G.gains(S, cand), ref)
            G.set_gain_lanes(64)
            np.testing.assert_array_equal(G.gains(S, cand), ref)
        G.set_gain_lanes(lanes)
        cand = rng.integers(0, n, size=2 * n + 5).astype(np.int32)
        np.testing.assert_array_equal(G.gains(S, cand), oracle.gains(rp, ci, S, cand))
        with pytest.raises(gcm.GcError):
            G.set_gain_lanes(96)


@pytest.mark.parametrize("lanes", [128, 256])
def test_gains_wide_rmat14_sampled(gcm, lanes):
    """R-MAT scale 14 (hub rows much longer than a CTA's 512 threads): 3000
    seeded candidates, several batches and a ragged tail, against the oracle;
    every vertex against the 64-lane kernel."""
    rp, ci = graphgen.rmat(14, 16.0, seed=6)
    n = rp.size - 1
    rng = np.random.default_rng(8)
    S = rng.choice(n, size=4, replace=False)
    cand = rng.choice(n, size=3000, replace=False).astype(np.int32)
    with gcm.Graph(rp, ci) as G:
        G.set_gain_lanes(lanes)
        np.testing.assert_array_equal(G.gains(S, cand), oracle.gains(rp, ci, S, cand))
        allv = np.arange(n, dtype=np.int32)
        wide = G.gains(S, allv)
        G.set_gain_lanes(64)
        np.testing.assert_array_equal(wide, G.gains(S, allv))


@pytest.mark.parametrize("lanes", [128, 256])
@pytest.mark.parametrize("name,g", small_cases() + [("rmat13", graphgen.rmat(13, 16.0, seed=4))])
def test_greedy_wide_lanes(gcm, name, g, lanes):
    """Greedy whose round 1 (every vertex, no bounds) and host-driven lazy
    steps run on the wide kernel: the oracle's group and farness."""
    rp, ci = g
    k = min(12, rp.size - 1)
    grp, ft, _ = oracle.greedy_plain(rp, ci, k)
    with gcm.Graph(rp, ci) as G:
        G.set_gain_lanes(lanes)
        for kw in ({"round1_bound": False, "step_mode": 1, "eval_per_step": 256, "step_lanes": 64},
                   {"step_mode": 1, "eval_per_step": 512, "step_lanes": 64}, {}):
            got, f, st = G.greedy(k, **kw)
            np.testing.assert_array_equal(got, grp)
            assert f == ft[-1]


def test_autotune_gain_lanes(gcm, tmp_path):
    """The width tuner times 64, 128 and 256 lanes, checks that they agree,
    caches the winner and leaves the handle at it; the oracle's gains."""
    from paper_1710_01144_gb300 import autotune

    rp, ci = graphgen.barabasi_albert(3000, 4, 11)
    n = rp.size - 1
    S = np.array([5, 77, 1234], dtype=np.int32)
    cand = np.arange(n, dtype=np.int32)
    cache = str(tmp_path / "tune.json")
    with gcm.Graph(rp, ci) as G:
        best, entry = autotune.tune_gain_lanes(G, S, cand, reps=1, cache=cache)
        assert best["gain_lanes"] in (64, 128, 256) and len(entry["trials"]) == 3
        np.testing.assert_array_equal(G.gains(S, cand), oracle.gains(rp, ci, S, cand))
        again, _ = autotune.tune_gain_lanes(G, S, cand, cache=cache)
        assert again == best
