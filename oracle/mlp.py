"""Float64 reference of the candidate-proposal network (not in the paper).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA kernels of the
proposal network (features, forward, gradient, Adam) element by element.

Network: 8 features -> 64 (ReLU) -> 64 (ReLU) -> 1, float32 on the GPU.
Parameter vector (4801 floats, this order):
    W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3[1]
    h1 = relu(x W1 + b1);  h2 = relu(h1 W2 + b2);  out = h2 . W3 + b3
Loss: mean squared error  L = (1/m) sum_i (out_i - y_i)^2.
Adam (Kingma & Ba): m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
    p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Features of a candidate v in round r (all float):
    0 log1p(deg v)            1 d_S[v]               2 log1p(max(ub[v], 0))
    3 r - stamp[v]            4 log1p(two_hop[v])    5 mx[v] - d_S[v]
    6 log1p(prev_gain)        7 feature 2 - feature 6
where two_hop[v] = sum over neighbours w of (deg w - 1), mx[v] = max d_S over
neighbours, prev_gain = gain of the previous round's pick.
"""
from __future__ import annotations

import numpy as np

IN, H = 8, 64
SIZES = [("W1", (IN, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)  # 4801


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(seed: int = 0):
    """He-style initialisation (used by tests as a starting point)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, np.sqrt(2 / IN), (IN, H)), "b1": np.zeros(H),
         "W2": rng.normal(0, np.sqrt(2 / H), (H, H)), "b2": np.zeros(H),
         "W3": rng.normal(0, np.sqrt(1 / H), (H,)), "b3": np.zeros(1)}
    return pack(d)


def forward(p, X):
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"] + w["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ w["W2"] + w["b2"]
    h2 = np.maximum(z2, 0)
    return h2 @ w["W3"] + w["b3"][0]


def loss(p, X, y):
    d = forward(p, X) - np.asarray(y, dtype=np.float64)
    return float(np.mean(d * d))


def grad(p, X, y):
    """Gradient of the mean squared error with respect to the parameter vector."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = X.shape[0]
    z1 = X @ w["W1"] + w["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ w["W2"] + w["b2"]
    h2 = np.maximum(z2, 0)
    out = h2 @ w["W3"] + w["b3"][0]
    dout = 2.0 * (out - y) / m
    g = {"W3": h2.T @ dout, "b3": np.array([dout.sum()])}
    dh2 = np.outer(dout, w["W3"]) * (z2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"].T) * (z1 > 0)
    g["W1"] = X.T @ dh1
    g["b1"] = dh1.sum(axis=0)
    return pack(g)


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def features(deg, dS, ub, stamp, two_hop, mx, rnd, prev_gain):
    """Feature matrix (float64) for vertices with the given per-vertex arrays."""
    deg = np.asarray(deg, dtype=np.float64)
    dS = np.asarray(dS, dtype=np.float64)
    ub = np.maximum(np.asarray(ub, dtype=np.float64), 0)
    f = np.zeros((deg.size, IN))
    f[:, 0] = np.log1p(deg)
    f[:, 1] = dS
    f[:, 2] = np.log1p(ub)
    f[:, 3] = rnd - np.asarray(stamp, dtype=np.float64)
    f[:, 4] = np.log1p(np.asarray(two_hop, dtype=np.float64))
    f[:, 5] = np.asarray(mx, dtype=np.float64) - dS
    f[:, 6] = np.log1p(max(float(prev_gain), 0.0))
    f[:, 7] = f[:, 2] - f[:, 6]
    return f
