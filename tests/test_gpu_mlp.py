"""GPU kernels of the proposal network against the float64 reference, and the
proposal's effect on Greedy++ (the group must not change)."""
import numpy as np
import pytest

import oracle
from oracle import mlp as mref
from paper_1710_01144_gb300 import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1710_01144_gb300 import build, gc

    build.build()
    return torch, gc


def _blocks():
    """(start, end) of each parameter block (W1, b1, W2, b2, W3, b3)."""
    out, o = [], 0
    for _, shape in mref.SIZES:
        k = int(np.prod(shape))
        out.append((o, o + k))
        o += k
    return out


def test_forward_grad_adam_match_reference(env):
    torch, gc = env
    rng = np.random.default_rng(11)
    p = mref.init_params(2)
    net = gc.Mlp(max_batch=512)
    net.set_params(p.astype(np.float32))
    p32 = net.get_params().astype(np.float64)  # the float32-rounded parameters
    for m in (1, 37, 512):
        X = rng.normal(size=(m, 8)).astype(np.float32)
        y = rng.normal(size=m).astype(np.float32)
        Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
        out = torch.empty(m, dtype=torch.float32, device="cuda")
        net.forward(Xd, out)
        torch.cuda.synchronize()
        ref = mref.forward(p32, X.astype(np.float64))
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)
        g, loss = net.grad(Xd, yd)
        gref = mref.grad(p32, X.astype(np.float64), y.astype(np.float64))
        assert abs(loss - mref.loss(p32, X, y)) <= 1e-4 * max(1.0, abs(loss))
        # element by element, each parameter block against its own scale
        # (float32 sums over m samples), so that a wrong entry of a small
        # block such as b3 or one column of W3 cannot hide in the norm
        for lo, hi in _blocks():
            scale = np.abs(gref[lo:hi]).max() + 1e-12
            np.testing.assert_allclose(g[lo:hi], gref[lo:hi], rtol=1e-3, atol=2e-5 * scale)
    # one Adam step against the reference
    X = rng.normal(size=(256, 8)).astype(np.float32)
    y = rng.normal(size=256).astype(np.float32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    net.set_params(p32.astype(np.float32))
    gref = mref.grad(p32, X.astype(np.float64), y.astype(np.float64))
    pref, _, _ = mref.adam_step(p32, gref, np.zeros_like(p32), np.zeros_like(p32), 1, lr=1e-3)
    net.adam_step(Xd, yd, 1e-3)
    got = net.get_params().astype(np.float64)
    # where |g| is not tiny the step is -lr*sign(g); compare the step itself
    big = np.abs(gref) > 1e-5
    np.testing.assert_allclose((got - p32)[big], (pref - p32)[big], rtol=1e-3, atol=1e-7)
    net.close()


def test_features_match_reference(env):
    torch, gc = env
    rng = np.random.default_rng(5)
    rp, ci = graphgen.rmat(10, 8.0, seed=2)
    n = rp.size - 1
    deg = np.diff(rp)
    dS = rng.integers(0, 6, size=n).astype(np.int32)
    ub = rng.integers(-1, 10**6, size=n).astype(np.int64)
    stamp = rng.integers(0, 9, size=n).astype(np.int32)
    two_hop = rng.integers(0, 10**5, size=n).astype(np.int64)
    mx = (dS + rng.integers(0, 3, size=n)).astype(np.int32)
    cand = rng.integers(0, n, size=300).astype(np.int32)
    d = lambda a: torch.from_numpy(a).cuda()
    X = torch.empty((cand.size, 8), dtype=torch.float32, device="cuda")
    gc.candidate_features(d(rp), d(dS), d(ub), d(stamp), d(two_hop), d(mx), d(cand), 9, 1234, X)
    torch.cuda.synchronize()
    ref = mref.features(deg[cand], dS[cand], ub[cand], stamp[cand], two_hop[cand], mx[cand], 9, 1234)
    np.testing.assert_allclose(X.cpu().numpy(), ref, rtol=1e-6, atol=1e-5)


def _record_and_train(torch, gc, graphs, k, epochs=30):
    Xs, ys = [], []
    for rp, ci in graphs:
        cap = 200_000
        X = torch.zeros((cap, 8), dtype=torch.float32, device="cuda")
        y = torch.zeros(cap, dtype=torch.float32, device="cuda")
        with gc.Graph(rp, ci) as G:
            G.set_recorder(X, y)
            G.greedy(k, step_mode=1, eval_per_step=64, step_lanes=8)
            m = G.recorded()
            G.set_recorder(None, None)
        Xs.append(X[:m].clone())
        ys.append(y[:m].clone())
    X = torch.cat(Xs)
    y = torch.cat(ys)
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(0)).cuda()
    X, y = X[perm].contiguous(), y[perm].contiguous()
    net = gc.Mlp(max_batch=1024)
    net.set_params(mref.init_params(0).astype(np.float32))
    _, loss0 = net.grad(X[:1024], y[:1024])
    loss = net.train(X, y, epochs=epochs, batch=1024, lr=2e-3, seed=3)
    return net, X.shape[0], loss0, loss


def test_trained_proposal_keeps_group_and_reports_gain(env, capsys):
    """Trained on exact gains of other seeds of the same graph families, the
    proposal chooses round 1's first exact batch (and, with fill 16, part of
    every lazy batch).  The group must equal the oracle's with and without it;
    the evaluation counts and times with and without it are printed."""
    torch, gc = env
    from paper_1710_01144_gb300 import proposal

    train = [graphgen.rmat(13, 16.0, seed=s) for s in (2, 3)] + [graphgen.barabasi_albert(6000, 4, s) for s in (5, 6)]
    net, (m, loss0, loss) = proposal.train(train, k=40)
    assert m > 500
    assert loss < 0.5 * loss0  # the network learned something about the gains
    for name, (rp, ci), k in (("rmat14", graphgen.rmat(14, 16.0, seed=1), 60),
                              ("ba8000", graphgen.barabasi_albert(8000, 4, 1), 30)):
        grp, ft, _, _ = oracle.greedypp(rp, ci, k)
        with gc.Graph(rp, ci) as G:
            g0, f0, s0 = G.greedy(k)
            for fill in (0, 16):
                G.set_proposal(net, fill)
                g1, f1, s1 = G.greedy(k, use_proposal=True)
                np.testing.assert_array_equal(g1, grp)
                assert f1 == ft[-1]
                with capsys.disabled():
                    print("\nproposal on %s (fill %d): samples %d, loss %.4f -> %.4f; evals %d -> %d, "
                          "steps %d -> %d, round-1 ms %.2f -> %.2f, total ms %.2f -> %.2f"
                          % (name, fill, m, loss0, loss, s0["evals"], s1["evals"], s0["steps"], s1["steps"],
                             s0["ms_round1"], s1["ms_round1"], s0["ms_total"], s1["ms_total"]))
            G.set_proposal(None)
        np.testing.assert_array_equal(g0, grp)
        assert f0 == ft[-1]
    net.close()
