"""gc_marginal_gains_static: the allocation-free gains entry point.

Some callers cannot allocate device memory: plugins confined to a host
application's own allocator or memory budget, and request paths where
allocator calls (which can synchronise the device) are not allowed.  The
static variant keeps its scratch in a fixed array inside libgc.so; this file
checks it, through the C ABI, against the ordinary gc_marginal_gains and the
CPU oracle on calls in a row, at its size limit, and on the inputs whose
device-side failure it reports by writing -1 to every output.  It is
collected last so that a run stopping at the first failure has already run
everything else.
"""
import numpy as np
import pytest

import oracle
from paper_1710_01144_gb300 import graphgen
from tests import smallgraphs as sg

pytestmark = pytest.mark.gpu

MAX_N = 1_048_496  # largest n the fixed scratch array holds (documented in include/gc.h)


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1710_01144_gb300 import build, gc

    build.build()
    return torch, gc


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _static_gains(torch, gc, rp, ci, S, cand):
    out = torch.full((max(len(cand), 1),), -7, dtype=torch.int64, device="cuda")
    gc.gains_static(_dev(torch, rp), _dev(torch, ci), _dev(torch, S), _dev(torch, cand), out[:len(cand)])
    torch.cuda.synchronize()
    return out[:len(cand)].cpu().numpy()


def test_static_gains_match_allocating_entry_point_twice(env):
    torch, gc = env
    rng = np.random.default_rng(21)
    # two calls in a row, the second on a smaller graph so that state left
    # behind by the first (another n, another layout) would show up
    cases = [graphgen.rmat(13, 16.0, seed=4), graphgen.barabasi_albert(1500, 3, 2)]
    for rp, ci in cases:
        n = rp.size - 1
        S = rng.choice(n, size=4, replace=False).astype(np.int32)
        cand = rng.integers(0, n, size=777).astype(np.int32)
        with gc.Graph(rp, ci) as G:
            ref = G.gains(S, cand)
        got = _static_gains(torch, gc, rp, ci, S, cand)
        np.testing.assert_array_equal(got, ref)
        np.testing.assert_array_equal(got, oracle.gains(rp, ci, S, cand))
    # and the same inputs twice on one graph
    rp, ci = sg.grid(30, 41)
    n = rp.size - 1
    S = np.array([5, 600], np.int32)
    cand = np.arange(n, dtype=np.int32)
    with gc.Graph(rp, ci) as G:
        ref = G.gains(S, cand)
    np.testing.assert_array_equal(ref, oracle.gains(rp, ci, S, cand))
    for _ in range(2):
        np.testing.assert_array_equal(_static_gains(torch, gc, rp, ci, S, cand), ref)


def _star(n):
    """Star K_{1,n-1} with centre 0 as an int32 CSR."""
    rp = np.empty(n + 1, dtype=np.int64)
    rp[0] = 0
    rp[1] = n - 1
    rp[2:] = n - 1 + np.arange(1, n, dtype=np.int64)
    ci = np.concatenate([np.arange(1, n, dtype=np.int32), np.zeros(n - 1, dtype=np.int32)])
    return rp.astype(np.int32), ci


def test_static_gains_size_limit(env):
    """The largest documented n runs (and matches the oracle); one more vertex
    is rejected with GC_ERANGE before anything runs."""
    torch, gc = env
    rp, ci = _star(MAX_N)
    S = np.array([7], np.int32)
    cand = np.array([0, 1, 7, 12345, MAX_N - 1], np.int32)
    got = _static_gains(torch, gc, rp, ci, S, cand)
    np.testing.assert_array_equal(got, oracle.gains(rp, ci, S, cand))
    rp1, ci1 = _star(MAX_N + 1)
    with pytest.raises(gc.GcError) as e:
        _static_gains(torch, gc, rp1, ci1, S, cand)
    assert e.value.code == gc.GC_ERANGE


def test_static_gains_reject_too_large(env):
    torch, gc = env
    n = 3_000_000  # more vertices than the fixed scratch can hold
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    S = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(gc.GcError) as e:
        gc.gains_static(rp, ci, S, S, out)
    assert e.value.code == gc.GC_ERANGE


def test_static_gains_failed_bfs_gives_minus_one(env):
    """An id of S outside [0, n) or a group that does not reach every vertex
    leaves d(., S) undefined: every output is -1, and the next call on valid
    inputs is correct again."""
    torch, gc = env
    rp, ci = sg.grid(12, 9)
    n = rp.size - 1
    cand = np.arange(n, dtype=np.int32)
    got = _static_gains(torch, gc, rp, ci, np.array([3, n + 5], np.int32), cand)
    assert (got == -1).all()
    # two disjoint paths: S in the first never reaches the second
    a = sg.path(20)
    rp2 = np.concatenate([a[0], a[0][1:] + a[1].size]).astype(np.int32)
    ci2 = np.concatenate([a[1], a[1] + 20]).astype(np.int32)
    got = _static_gains(torch, gc, rp2, ci2, np.array([4], np.int32), np.arange(40, dtype=np.int32))
    assert (got == -1).all()
    S = np.array([5, 60], np.int32)
    np.testing.assert_array_equal(_static_gains(torch, gc, rp, ci, S, cand), oracle.gains(rp, ci, S, cand))
