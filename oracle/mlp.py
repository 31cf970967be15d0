"""Surrogate network oracle -- TEST INFRASTRUCTURE ONLY (plain numpy, float64).

The network maps a chromosome's feature vector x (in_dim values) to a
predicted normalised makespan: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
y = w3 . h2 + b3, trained on the mean squared error with Adam (Kingma & Ba,
"Adam: A Method for Stochastic Optimization", 2015).

`rounded=True` reproduces where the GPU path stores BF16 values: the input,
W1, W2 and both hidden activations are rounded to BF16 (round to nearest
even), everything else is exact (float64 here; FP32 accumulation on the GPU).
The gradients are those of that function with the hidden activations'
rounding treated as identity (straight-through), plus BF16 rounding of the
backpropagated hidden-layer signals, which is where the GPU rounds them.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    out = u.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    out[nan] = np.nan
    return out


def init_params_philox(in_dim: int, h1: int, h2: int, seed: int) -> dict:
    """The library's documented weight initialisation restated with the
    oracle's own Philox: He-uniform (He et al. 2015; limit sqrt(6 / fan_in)
    in float32), element (o, i) of layer L (1: W1, 2: W2, 3: w3 as one row)
    from draw i of the stream (seed, purpose 14, island L, generation 0,
    cell o), u = ((x >> 8) - 2^23) / 2^23, value lim * u (then * 0.1 for w3),
    each product rounded once to float32; biases 0."""
    from oracle import draw

    def layer(rows, cols, fan_in, L, scale=None):
        lim = np.sqrt(np.float32(6.0) / np.float32(fan_in), dtype=np.float32)
        W = np.zeros((rows, cols), dtype=np.float32)
        for o in range(rows):
            x = np.array([draw(seed, 14, L, 0, o, i) for i in range(cols)], dtype=np.int64)
            u = (((x >> 8) - (1 << 23)).astype(np.float32) * np.float32(1.0 / 8388608.0)).astype(np.float32)
            v = (lim * u).astype(np.float32)
            if scale is not None:
                v = (v * np.float32(scale)).astype(np.float32)
            W[o] = v
        return W
    return {"W1": layer(h1, in_dim, in_dim, 1), "b1": np.zeros(h1, np.float32),
            "W2": layer(h2, h1, h1, 2), "b2": np.zeros(h2, np.float32),
            "w3": layer(1, h2, h2, 3, scale=0.1)[0], "b3": np.float32(0.0)}


def forward(params: dict, X, rounded: bool = True):
    X = np.asarray(X, dtype=np.float64)
    r = bf16_round if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    Xr = r(X)
    W1, W2 = r(params["W1"]), r(params["W2"])
    Z1 = Xr @ W1.T + np.asarray(params["b1"], np.float64)
    H1 = r(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + np.asarray(params["b2"], np.float64)
    H2 = r(np.maximum(Z2, 0.0))
    y = H2 @ np.asarray(params["w3"], np.float64) + float(params["b3"])
    return y, {"X": Xr, "W1": W1, "W2": W2, "H1": H1, "H2": H2, "Z1": Z1, "Z2": Z2}


def loss_and_grads(params: dict, X, t, rounded: bool = True):
    """MSE loss and its gradients with respect to every parameter."""
    y, c = forward(params, X, rounded)
    t = np.asarray(t, dtype=np.float64)
    B = len(t)
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B
    r = bf16_round if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    w3 = np.asarray(params["w3"], np.float64)
    gw3 = c["H2"].T @ dy
    gb3 = dy.sum()
    dZ2 = r(np.outer(dy, w3) * (c["H2"] > 0))
    gW2 = dZ2.T @ c["H1"]
    gb2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ c["W2"]
    dZ1 = dH1 * (c["H1"] > 0)
    gW1 = r(dZ1).T @ c["X"]
    gb1 = dZ1.sum(axis=0)
    return loss, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "w3": gw3, "b3": gb3}


def adam_step(params: dict, grads: dict, state: dict, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> dict:
    """One Adam update (in float64); state holds m, v and t."""
    t = state.get("t", 0) + 1
    out = {}
    for k, g in grads.items():
        m = b1 * state.get(("m", k), 0.0) + (1 - b1) * np.asarray(g, np.float64)
        v = b2 * state.get(("v", k), 0.0) + (1 - b2) * np.asarray(g, np.float64) ** 2
        state[("m", k)], state[("v", k)] = m, v
        out[k] = np.asarray(params[k], np.float64) - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    state["t"] = t
    return out


def instance_features(n: int, S: int, M, p, width: int = 40) -> np.ndarray:
    """The network's instance summary: per stage s < 12 the triple
    (M_s / 10, mean_j p[j][s] / 99, load_s / (M_s * LB)), then n / 500,
    S / 20, LB / sum p, zero-padded to `width` (float32)."""
    p = np.asarray(p, dtype=np.float64).reshape(n, S)
    M = np.asarray(M, dtype=np.float64)
    loads = p.sum(axis=0)
    lb = max(p.sum(axis=1).max(), max(np.ceil(loads[s] / M[s]) for s in range(S)))
    f = np.zeros(width, dtype=np.float64)
    k = 0
    for s in range(min(S, 12)):
        f[k:k + 3] = (M[s] / 10.0, loads[s] / n / 99.0, loads[s] / (M[s] * lb))
        k += 3
    f[36:39] = (n / 500.0, S / 20.0, lb / p.sum())
    return f.astype(np.float32)


def features(rows: np.ndarray, n: int, P: int, inst_feat: np.ndarray) -> np.ndarray:
    """Network input of job orders: x[j] = position of job j / (n - 1) for j < n
    (0 when n = 1), zero for n <= j < P, then the instance features; rounded
    to BF16 as the GPU stores them."""
    rows = np.asarray(rows)
    X = np.zeros((rows.shape[0], P + len(inst_feat)), dtype=np.float32)
    denom = np.float32(max(n - 1, 1))
    pos = (np.arange(n, dtype=np.float32) / denom).astype(np.float32)
    for r in range(rows.shape[0]):
        X[r, rows[r, :n].astype(np.int64)] = pos
    X[:, P:] = inst_feat
    return bf16_round(X)
