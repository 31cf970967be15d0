"""Pins of the surrogate-network oracle (oracle/mlp.py): BF16 rounding against
torch's conversion, a hand-computed tiny network, and gradients against
central finite differences of the unrounded network."""
import numpy as np
import pytest

from ffs_workloads import mlp_params
from oracle import mlp


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 10, 5000), rng.normal(0, 1e-3, 5000), [0.0, -0.0, 1.0, 3.0, 65504.0,
                                                                             1.00390625, 1.01171875]])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), want)
    # ties to even at the half-way points between BF16 neighbours of 1.0
    assert mlp.bf16_round(np.float32(1.00390625))[()] == 1.0
    assert mlp.bf16_round(np.float32(1.01171875))[()] == 1.015625


def test_tiny_network_by_hand():
    p = {"W1": np.array([[1.0, -1.0], [0.5, 0.5]], np.float32), "b1": np.array([0.0, -1.0], np.float32),
         "W2": np.array([[2.0, 1.0]], np.float32), "b2": np.array([0.5], np.float32),
         "w3": np.array([3.0], np.float32), "b3": np.float32(-1.0)}
    X = np.array([[2.0, 1.0], [1.0, 3.0]])
    # row 0: z1 = (1, 0.5), h1 = (1, 0.5); z2 = 2.5 + 0.5 = 3, h2 = 3; y = 9 - 1 = 8
    # row 1: z1 = (-2, 1), h1 = (0, 1); z2 = 1 + 0.5 = 1.5; y = 4.5 - 1 = 3.5
    y, _ = mlp.forward(p, X, rounded=False)
    assert y.tolist() == [8.0, 3.5]
    loss, g = mlp.loss_and_grads(p, X, [7.0, 3.5], rounded=False)
    assert loss == 0.5
    assert g["b3"] == 1.0                      # dy = (2*1/2, 0)
    assert g["w3"].tolist() == [3.0]           # h2 of row 0


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    p = mlp_params(7, 64, 64, seed=3)
    p["b1"] = rng.normal(0, 0.1, 64).astype(np.float32)
    p["b2"] = rng.normal(0, 0.1, 64).astype(np.float32)
    X = rng.normal(0, 1, (16, 7))
    t = rng.normal(0, 1, 16)
    _, g = mlp.loss_and_grads(p, X, t, rounded=False)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        base = np.asarray(p[k], np.float64)
        flat = base.reshape(-1)
        for idx in rng.choice(flat.size, min(6, flat.size), replace=False):
            pp, pm = dict(p), dict(p)
            a, b = flat.copy(), flat.copy()
            a[idx] += h
            b[idx] -= h
            pp[k] = a.reshape(base.shape) if base.shape else a[0]
            pm[k] = b.reshape(base.shape) if base.shape else b[0]
            num = (mlp.loss_and_grads(pp, X, t, rounded=False)[0] - mlp.loss_and_grads(pm, X, t, rounded=False)[0]) / (2 * h)
            ana = np.asarray(g[k]).reshape(-1)[idx]
            assert abs(num - ana) <= 1e-5 + 1e-4 * abs(ana), (k, idx, num, ana)


def test_adam_first_step_is_signed_lr():
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -4.0, 0.0])}
    out = mlp.adam_step(p, g, {}, lr=0.01)
    # first Adam step: m_hat = g, v_hat = g^2 -> update = lr * sign(g) (0 for g = 0)
    assert np.allclose(out["a"], [0.99, -1.99, 0.5], atol=1e-9)


def test_philox_initialisation_follows_its_definition():
    """init_params_philox: values inside (-lim, lim) with lim = sqrt(6 / fan_in)
    (He-uniform), spread like a uniform draw, w3 scaled by 0.1, biases 0, and
    element (o, i) taken from the documented Philox counter."""
    import oracle
    p = mlp.init_params_philox(48, 64, 64, seed=3)
    for k, fan in (("W1", 48), ("W2", 64)):
        lim = np.sqrt(6.0 / fan)
        W = p[k].astype(np.float64)
        assert np.all(np.abs(W) <= lim)
        assert abs(W.mean()) < 0.05 * lim
        assert abs(W.var() / (lim * lim / 3.0) - 1.0) < 0.1          # variance of U(-lim, lim)
    assert np.all(np.abs(p["w3"]) <= 0.1 * np.sqrt(6.0 / 64))
    assert not p["b1"].any() and not p["b2"].any() and float(p["b3"]) == 0.0
    # element (o = 5, i = 6) of W2: word 6 mod 4 of the block with counter (6 / 4, 5, 0, 2 | 14 << 24)
    x = int(oracle.philox([1, 5, 0, 2 | (14 << 24)], [3, 0])[2])
    u = ((x >> 8) - (1 << 23)) / 8388608.0
    lim = float(np.sqrt(np.float32(6.0) / np.float32(64), dtype=np.float32))
    assert abs(float(p["W2"][5, 6]) - lim * u) <= 1e-7 * lim
