"""Tensor-core GEMM and surrogate network against the float64 oracle
(oracle/mlp.py), within tolerances derived from BF16 inputs and FP32
accumulation."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 256, 128), (300, 192, 540), (1024, 512, 576),
                                   (128, 576, 1024), (77, 128, 16), (512, 256, 512)])
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


def test_mlp_forward_matches_oracle(gpu):
    in_dim, h1, h2 = 540, 512, 256
    p = omlp.init_params(in_dim, h1, h2, seed=1)
    rng = np.random.default_rng(2)
    p["b1"] = rng.normal(0, 0.05, h1).astype(np.float32)
    p["b2"] = rng.normal(0, 0.05, h2).astype(np.float32)
    m = gpu.MLP(in_dim, h1, h2, 2048)
    m.set_params(p)
    back = m.get()
    assert np.array_equal(back["W1"], p["W1"]) and np.array_equal(back["w3"], p["w3"])
    B = 1000
    X = _features(rng, B, in_dim)
    ldx = 544
    Xp = np.zeros((B, ldx), np.float32)
    Xp[:, :in_dim] = X
    y = torch.zeros(B, dtype=torch.float32, device="cuda")
    gpu.ffs_mlp_forward(m, _bf16(Xp), ldx, B, y)
    gpu.ffs_mlp_check(m)
    got = y.cpu().numpy().astype(np.float64)
    want, _ = omlp.forward(p, X, rounded=True)
    scale = np.mean(np.abs(want)) + 1e-3
    assert np.max(np.abs(got - want)) <= 2e-2 * scale, (np.max(np.abs(got - want)), scale)


def test_mlp_gradients_match_oracle_and_training_reduces_loss(gpu):
    in_dim, h1, h2 = 540, 512, 256
    p = omlp.init_params(in_dim, h1, h2, seed=5)
    m = gpu.MLP(in_dim, h1, h2, 1024)
    m.set_params(p)
    rng = np.random.default_rng(6)
    B = 512
    X = _features(rng, B, in_dim)
    t = (X[:, :50].sum(axis=1) / 25.0 - 1.0).astype(np.float32)
    ldx = m.width
    Xp = np.zeros((B, ldx), np.float32)
    Xp[:, :in_dim] = X
    Xd = _bf16(Xp)
    td = torch.from_numpy(t).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gpu.ffs_mlp_train_step(m, Xd, ldx, td, B, 0.0, loss)
    gpu.ffs_mlp_check(m)
    g = m.get(grads=True)
    oloss, og = omlp.loss_and_grads(p, X, t, rounded=True)
    assert abs(float(loss.item()) - oloss) <= 1e-2 * oloss
    for k in ("W1", "b1", "W2", "b2", "w3"):
        a, b = np.asarray(g[k], np.float64), np.asarray(og[k], np.float64)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-12)
        assert rel <= 3e-2, (k, rel)
    assert abs(float(g["b3"]) - float(og["b3"])) <= 1e-3 * (abs(float(og["b3"])) + 1e-3)
    first = float(loss.item())
    for _ in range(150):
        gpu.ffs_mlp_train_step(m, Xd, ldx, td, B, 1e-3, loss)
    gpu.ffs_mlp_check(m)
    assert float(loss.item()) < 0.2 * first
