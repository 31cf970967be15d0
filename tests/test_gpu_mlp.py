"""Tensor-core GEMM and surrogate network against the float64 oracle
(oracle/mlp.py), element by element, within bounds derived from BF16 inputs
and FP32 accumulation.

Bounds.  A GPU value that is a sum of products (a GEMM entry, a gradient
summed over the batch) differs from the oracle's by FP32 accumulation error
(at most K * 2^-24 of the sum of the absolute terms) plus, rarely, a BF16
rounding decision taken on the other side of a rounding boundary (one BF16
ulp, 2^-8 relative, on one term) or an activation exactly at the ReLU's kink
(one whole term of the B in a batch gradient).  So the check is
|gpu - oracle| <= rtol * sum_k |term_k| + atol with rtol = 1e-2 (the 1e-2
relative error of the network's reading of the surrogate) and a small
absolute floor.  Adam's update is compared in FP32 terms: the oracle's
float64 step given the GPU's gradients, to a few FP32 ulps of each parameter
plus 1e-4 of the step (beta2 = 0.999 is 1.3e-5 off in FP32)."""
import numpy as np
import pytest
import torch

from ffs_workloads import mlp_params
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

RTOL = 1e-2


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 256, 128), (300, 192, 540), (1024, 512, 576),
                                   (128, 576, 1024), (77, 128, 16), (512, 256, 512),
                                   # at least one row tile per SM: the persistent form (two
                                   # accumulators; 128- and 256-column tiles, ragged rows and K)
                                   (32768, 512, 576), (20000, 256, 512), (19584, 384, 200),
                                   (40000, 128, 64)])
def test_gemm_matches_float64(gpu, M, N, K):
    rng = np.random.default_rng(M + N + K)
    lda = (K + 7) // 8 * 8
    A = np.zeros((M, lda), np.float32)
    B = np.zeros((N, lda), np.float32)
    A[:, :K] = rng.normal(0, 1, (M, K))
    B[:, :K] = rng.normal(0, 1, (N, K))
    Ab, Bb = _bf16(A), _bf16(B)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    gpu.ffs_gemm_bf16(Ab, lda, Bb, lda, D, N, M, N, K, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    Ar = Ab.float().cpu().numpy().astype(np.float64)[:, :K]
    Br = Bb.float().cpu().numpy().astype(np.float64)[:, :K]
    want = Ar @ Br.T
    bound = (np.abs(Ar) @ np.abs(Br).T) * (K * 2.0 ** -24) + 1e-6   # FP32 accumulation error bound
    got = D.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - want) <= bound), float(np.max(np.abs(got - want) - bound))


def _features(rng, B, in_dim):
    return rng.uniform(0, 1, (B, in_dim)).astype(np.float32)


def _padded(X, ldx):
    Xp = np.zeros((X.shape[0], ldx), np.float32)
    Xp[:, :X.shape[1]] = X
    return _bf16(Xp)


def test_mlp_init_matches_oracle_philox_bit_exactly(gpu):
    in_dim, h1, h2 = 540, 512, 256
    m = gpu.MLP(in_dim, h1, h2, 256)
    m.init(3)
    got = m.get()
    want = omlp.init_params_philox(in_dim, h1, h2, 3)
    for k in ("W1", "b1", "W2", "b2", "w3"):
        assert np.array_equal(got[k].view(np.uint32), np.asarray(want[k], np.float32).view(np.uint32)), k
    assert float(got["b3"]) == 0.0 and m.adam_steps() == 0


@pytest.mark.parametrize("B", [1000, 20000])    # 20000: both layers on the persistent GEMM
def test_mlp_forward_matches_oracle(gpu, B):
    in_dim, h1, h2 = 540, 512, 256
    p = mlp_params(in_dim, h1, h2, seed=1)
    rng = np.random.default_rng(2)
    p["b1"] = rng.normal(0, 0.05, h1).astype(np.float32)
    p["b2"] = rng.normal(0, 0.05, h2).astype(np.float32)
    p["b3"] = np.float32(0.25)
    m = gpu.MLP(in_dim, h1, h2, max(2048, (B + 127) // 128 * 128))
    m.set_params(p)
    back = m.get()
    assert np.array_equal(back["W1"], p["W1"]) and np.array_equal(back["w3"], p["w3"])
    X = _features(rng, B, in_dim)
    y = torch.zeros(B, dtype=torch.float32, device="cuda")
    gpu.ffs_mlp_forward(m, _padded(X, 544), 544, B, y)
    gpu.ffs_mlp_check(m)
    got = y.cpu().numpy().astype(np.float64)
    want, c = omlp.forward(p, X, rounded=True)
    # per row: y = sum_j H2[j] w3[j] + b3
    terms = np.abs(c["H2"]) @ np.abs(np.asarray(p["w3"], np.float64)) + abs(float(p["b3"]))
    assert np.all(np.abs(got - want) <= RTOL * terms + 1e-6), float(np.max(np.abs(got - want) / terms))
    assert np.max(np.abs(got - want)) <= RTOL * np.mean(np.abs(want))


def _grad_terms(p, X, t):
    """Per gradient entry: (sum over the batch of |each product|, the part of
    it that passes through an ambiguous activation).  An activation is
    ambiguous when its pre-activation Z lies within 1e-3 of its own sum of
    |terms| of the ReLU's kink -- the room for FP32 accumulation and a few
    BF16 rounding flips (2^-7 each) among its inputs: it may be open on one
    side and closed on the other, so its terms may differ in full."""
    y, c = omlp.forward(p, X, rounded=True)
    dy = np.abs(2.0 * (y - np.asarray(t, np.float64)) / len(t))
    w3 = np.abs(np.asarray(p["w3"], np.float64))
    S1 = np.abs(c["X"]) @ np.abs(c["W1"]).T + np.abs(np.asarray(p["b1"], np.float64))
    S2 = c["H1"] @ np.abs(c["W2"]).T + np.abs(np.asarray(p["b2"], np.float64))
    amb1 = np.abs(c["Z1"]) <= 1e-3 * S1
    amb2 = np.abs(c["Z2"]) <= 1e-3 * S2
    open1, open2 = (c["H1"] > 0) | amb1, (c["H2"] > 0) | amb2
    H1 = np.maximum(c["H1"], np.where(amb1, 1e-3 * S1, 0.0))     # largest value an ambiguous unit may take
    H2 = np.maximum(c["H2"], np.where(amb2, 1e-3 * S2, 0.0))
    dZ2 = np.outer(dy, w3) * open2
    dZ2a = np.outer(dy, w3) * amb2
    dH1 = dZ2 @ np.abs(c["W2"])
    dH1a = dZ2a @ np.abs(c["W2"])
    dZ1 = dH1 * open1
    dZ1a = dH1a * open1 + dH1 * amb1
    X = np.abs(c["X"])
    total = {"W1": dZ1.T @ X, "b1": dZ1.sum(axis=0), "W2": dZ2.T @ H1, "b2": dZ2.sum(axis=0),
             "w3": H2.T @ dy, "b3": dy.sum()}
    amb = {"W1": dZ1a.T @ X, "b1": dZ1a.sum(axis=0), "W2": dZ2a.T @ H1 + dZ2.T @ (H1 * amb1),
           "b2": dZ2a.sum(axis=0), "w3": (H2 * amb2).T @ dy, "b3": 0.0}
    return total, amb


def _bound(total, amb):
    T = np.asarray(total, np.float64)
    return RTOL * T + np.asarray(amb, np.float64) + 1e-6 * float(np.max(T))


def _check_elementwise(got, want, bound, what):
    a = np.asarray(got, np.float64)
    b = np.asarray(want, np.float64)
    bad = np.abs(a - b) > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(a - b) / np.maximum(bound, 1e-30))))


def _train_setup(gpu, seed_p, seed_x, B=512):
    in_dim, h1, h2 = 540, 512, 256
    p = mlp_params(in_dim, h1, h2, seed=seed_p)
    rng = np.random.default_rng(seed_x)
    p["b1"] = rng.normal(0, 0.02, h1).astype(np.float32)
    p["b2"] = rng.normal(0, 0.02, h2).astype(np.float32)
    m = gpu.MLP(in_dim, h1, h2, 1024)
    m.set_params(p)
    X = _features(rng, B, in_dim)
    t = (X[:, :50].sum(axis=1) / 25.0 - 1.0).astype(np.float32)
    return m, p, X, t, _padded(X, m.width), torch.from_numpy(t).cuda()


def test_mlp_gradients_match_oracle_elementwise(gpu):
    m, p, X, t, Xd, td = _train_setup(gpu, 5, 6)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gpu.ffs_mlp_train_step(m, Xd, m.width, td, len(t), 0.0, loss)
    gpu.ffs_mlp_check(m)
    g = m.get(grads=True)
    oloss, og = omlp.loss_and_grads(p, X, t, rounded=True)
    assert abs(float(loss.item()) - oloss) <= RTOL * oloss
    total, amb = _grad_terms(p, X, t)
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        _check_elementwise(g[k], og[k], _bound(total[k], amb[k]), k)
    # lr = 0: the parameters do not move
    after = m.get()
    assert all(np.array_equal(after[k], p[k]) for k in ("W1", "W2", "w3"))


def test_mlp_adam_steps_match_oracle_elementwise(gpu):
    """Three training steps with lr = 1e-3.  After each: the moments and the
    parameters against oracle.adam_step fed the GPU's gradients (the update's
    arithmetic), and after the first step, the parameters against the
    oracle's own gradient-and-update wherever that gradient's sign is
    decided (|g| above its element bound)."""
    lr = 1e-3
    m, p, X, t, Xd, td = _train_setup(gpu, 9, 10)
    keys = ("W1", "b1", "W2", "b2", "w3", "b3")
    state = {}
    prev = {k: np.asarray(p[k], np.float64) for k in keys}
    mags = {k: 0.0 for k in keys}
    _, og1 = omlp.loss_and_grads(p, X, t, rounded=True)
    total1, amb1 = _grad_terms(p, X, t)
    for step in (1, 2, 3):
        gpu.ffs_mlp_train_step(m, Xd, m.width, td, len(t), lr, None)
        gpu.ffs_mlp_check(m)
        assert m.adam_steps() == step
        g = m.get(grads=True)
        want = omlp.adam_step(prev, {k: np.asarray(g[k], np.float64) for k in keys}, state, lr)
        got, m1, m2 = m.get(), m.get(which=2), m.get(which=3)
        for k in keys:
            gk = np.abs(np.asarray(g[k], np.float64))
            mags[k] = 0.9 * mags[k] + 0.1 * gk      # sum of |terms| behind the first moment
            assert np.all(np.abs(m1[k] - state[("m", k)]) <= 1e-4 * mags[k] + 1e-30), (k, step)
            assert np.all(np.abs(m2[k] - state[("v", k)]) <= 1e-4 * state[("v", k)] + 1e-38), (k, step)
            tol = step * (4 * 2.0 ** -24 * np.abs(want[k]) + 1e-4 * lr)
            err = np.abs(np.asarray(got[k], np.float64) - want[k])
            assert np.all(err <= tol), (k, step, float(np.max(err - tol)))
        prev = want
        if step == 1:
            oracle1 = omlp.adam_step({k: np.asarray(p[k], np.float64) for k in keys}, og1, {}, lr)
            for k in keys:
                gb = np.asarray(og1[k], np.float64)
                bnd = _bound(total1[k], amb1[k])
                # |g| above twice its element bound: the GPU's gradient has the same sign.
                # The first step is lr g / (|g| + eps); near eps = 1e-8 it still moves
                # with |g|, by lr eps dg / (|g| - dg + eps)^2 for a gradient error dg.
                decided = np.abs(gb) > 2 * bnd
                sens = lr * 1e-8 * bnd / (np.abs(gb) - bnd + 1e-8) ** 2
                err = np.abs(np.asarray(got[k], np.float64) - oracle1[k])
                tol1 = 4 * 2.0 ** -24 * np.abs(oracle1[k]) + 1e-4 * lr + sens
                assert np.all(err[decided] <= tol1[decided]), (k, float(np.max((err - tol1)[decided])))
                if k != "b3":
                    assert decided.mean() > 0.2, (k, float(decided.mean()))


def test_mlp_training_reduces_loss(gpu):
    m, p, X, t, Xd, td = _train_setup(gpu, 5, 6)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gpu.ffs_mlp_train_step(m, Xd, m.width, td, len(t), 0.0, loss)
    first = float(loss.item())
    for _ in range(150):
        gpu.ffs_mlp_train_step(m, Xd, m.width, td, len(t), 1e-3, loss)
    gpu.ffs_mlp_check(m)
    assert float(loss.item()) < 0.2 * first


def test_mlp_state_save_load_resumes_bit_exactly(gpu):
    """Save after 2 steps, take 3 more; a fresh network loaded from the blob
    takes the same 3 steps to the same parameters and moments, bit for bit."""
    m, p, X, t, Xd, td = _train_setup(gpu, 12, 13)
    for _ in range(2):
        gpu.ffs_mlp_train_step(m, Xd, m.width, td, len(t), 1e-3, None)
    blob = m.save()
    for _ in range(3):
        gpu.ffs_mlp_train_step(m, Xd, m.width, td, len(t), 1e-3, None)
    m2 = gpu.MLP(540, 512, 256, 1024)
    m2.init(77)
    m2.load_state(blob)
    assert m2.adam_steps() == 2
    for _ in range(3):
        gpu.ffs_mlp_train_step(m2, Xd, m2.width, td, len(t), 1e-3, None)
    for which in (0, 2, 3):
        a, b = m.get(which=which), m2.get(which=which)
        for k in a:
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), (which, k)
    small = gpu.MLP(540, 256, 256, 256)
    with pytest.raises(gpu.FFSError) as e:
        small.load_state(blob)
    assert e.value.status == gpu.FFS_EINVAL
