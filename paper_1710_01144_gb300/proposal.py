"""Training of the candidate-proposal network on exact gains produced by the
method itself (host-driven lazy steps record, for every candidate they
evaluate, its features at selection time and log1p of its exact gain)."""
from __future__ import annotations

import numpy as np

from . import gc


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initial parameters (float32), layout of include/gc.h."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0, np.sqrt(2 / 8), (8, 64))
    w2 = rng.normal(0, np.sqrt(2 / 64), (64, 64))
    w3 = rng.normal(0, np.sqrt(1 / 64), 64)
    return np.concatenate([w1.ravel(), np.zeros(64), w2.ravel(), np.zeros(64), w3, np.zeros(1)]).astype(np.float32)


def record(graphs, k: int, cap: int = 400_000, lazy_rounds: bool = True):
    """(X, y) CUDA tensors of recorded samples: per graph, the 1024 largest
    round-1 two-hop bounds with their exact gains (a default-mode call) and,
    with lazy_rounds, every candidate of the host-driven lazy steps of rounds
    >= 2."""
    import torch

    Xs, ys = [], []
    for rp, ci in graphs:
        X = torch.zeros((cap, 8), dtype=torch.float32, device="cuda")
        y = torch.zeros(cap, dtype=torch.float32, device="cuda")
        with gc.Graph(rp, ci) as G:
            G.set_recorder(X, y)
            G.greedy(min(k, 2))
            if lazy_rounds:
                G.greedy(k, step_mode=1, eval_per_step=64, step_lanes=8)
            m = G.recorded()
            G.set_recorder(None, None)
        Xs.append(X[:m].clone())
        ys.append(y[:m].clone())
    X = torch.cat(Xs)
    y = torch.cat(ys)
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(0)).cuda()
    return X[perm].contiguous(), y[perm].contiguous()


def train(graphs, k: int = 100, epochs: int = 30, batch: int = 1024, lr: float = 2e-3, seed: int = 3):
    """A trained gc.Mlp and (samples, initial loss, final loss)."""
    X, y = record(graphs, k)
    net = gc.Mlp(max_batch=batch)
    net.set_params(init_params(0))
    _, loss0 = net.grad(X[:batch], y[:batch])
    loss = net.train(X, y, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return net, (int(X.shape[0]), loss0, loss)
