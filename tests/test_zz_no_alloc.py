"""gc_marginal_gains_static: the allocation-free gains entry point.

Some callers cannot allocate device memory (code that runs while another
component captures the stream into a CUDA graph, or that must stay inside a
host application's own allocator).  The static variant keeps its scratch in a
fixed array inside libgc.so; this file checks it, through the C ABI, against
the ordinary gc_marginal_gains on two calls in a row.  It is collected last so
that a run stopping at the first failure has already run everything else.
"""
import numpy as np
import pytest

from paper_1710_01144_gb300 import graphgen
from tests import smallgraphs as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1710_01144_gb300 import build, gc

    build.build()
    return torch, gc


def _static_gains(torch, gc, rp, ci, S, cand):
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    out = torch.full((len(cand),), -7, dtype=torch.int64, device="cuda")
    gc.gains_static(d(rp), d(ci), d(S), d(cand), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


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
    # and the same inputs twice on one graph
    rp, ci = sg.grid(30, 41)
    n = rp.size - 1
    S = np.array([5, 600], np.int32)
    cand = np.arange(n, dtype=np.int32)
    with gc.Graph(rp, ci) as G:
        ref = G.gains(S, cand)
    for _ in range(2):
        np.testing.assert_array_equal(_static_gains(torch, gc, rp, ci, S, cand), ref)


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
