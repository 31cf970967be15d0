"""GPU evaluation of the paper's genotype (n*S machine-assignment strings on
unrelated machines) against the CPU oracle, bit-exact, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as orc
from conftest import dev
from ffs_workloads import make_assign_instance, random_assignments

pytestmark = pytest.mark.gpu

SHAPES = [
    # n, S, m_lo, m_hi, N
    (1, 1, 1, 1, 5),
    (1, 4, 1, 3, 9),
    (7, 1, 3, 3, 33),
    (20, 5, 1, 4, 100),
    (40, 3, 32, 32, 70),      # 32 machines, the per-stage maximum
    (100, 10, 2, 5, 300),
    (257, 7, 1, 9, 130),
    (500, 20, 5, 10, 64),
    (100, 4, 32, 32, 50),     # per-thread genes in shared memory, table slice not
    (3000, 2, 2, 3, 20),      # genes read from the stage-major copy in global memory
    (20, 5, 1, 4, 40000),     # more rows than one chunk
]


def _pair(spec, gpu, release=None, due=None, wt=0):
    return (orc.AssignInstance(spec.n, spec.S, spec.M, spec.p_u, release, due, wt),
            gpu.AssignInstance(spec.n, spec.S, spec.M, spec.p_u, release, due, wt))


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[0]}x{s[1]}m{s[2]}-{s[3]}N{s[4]}" for s in SHAPES])
def test_assign_eval_matches_oracle(gpu, shape):
    n, S, mlo, mhi, N = shape
    spec = make_assign_instance(n, S, mlo, mhi, seed=n * 13 + S)
    o, g = _pair(spec, gpu)
    pop = random_assignments(n, S, spec.M, N, seed=N + n)
    out = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    gpu.ffs_assign_eval(g, dev(pop), N, pop.shape[1], out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().astype(np.int64), orc.eval_population_assign(o, pop))


def test_assign_eval_objective_with_release_and_due(gpu):
    rng = np.random.default_rng(3)
    for trial in range(4):
        n, S = int(rng.integers(2, 120)), int(rng.integers(1, 8))
        spec = make_assign_instance(n, S, 1, 6, seed=40 + trial)
        R = rng.integers(0, 300, size=n).astype(np.int32)
        D = (R + rng.integers(0, 400, size=n)).astype(np.int32)
        o, g = _pair(spec, gpu, R, D, 7)
        pop = random_assignments(n, S, spec.M, 200, seed=trial)
        out = torch.zeros(200, dtype=torch.int32, device="cuda")
        gpu.ffs_assign_eval(g, dev(pop), 200, pop.shape[1], out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), orc.eval_population_assign(o, pop)), trial


def test_assign_golden_examples(gpu, golden):
    for ex in golden("assign_examples.json")["examples"]:
        g = gpu.AssignInstance(ex["n"], ex["S"], ex["M"], ex["p_u"], ex.get("release"), ex.get("due"),
                               ex.get("wt", 0))
        pop = np.zeros((1, 8), dtype=np.int16)
        pop[0, :len(ex["genes"])] = ex["genes"]
        out = torch.zeros(1, dtype=torch.int32, device="cuda")
        gpu.ffs_assign_eval(g, dev(pop), 1, 8, out)
        torch.cuda.synchronize()
        assert int(out.item()) == ex["objective"], ex["name"]


def test_assign_invalid_genes_empty_and_errors(gpu):
    spec = make_assign_instance(10, 3, 2, 3, seed=9)
    o, g = _pair(spec, gpu)
    pop = random_assignments(10, 3, spec.M, 20, ld=32, seed=1)
    pop[:, 30:] = 12345          # padding is never read as genes
    pop[3, 4] = 99               # machine out of range -> -1
    pop[5, 0] = -1               # negative -> -1
    out = torch.zeros(20, dtype=torch.int32, device="cuda")
    gpu.ffs_assign_eval(g, dev(pop), 20, 32, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[3] == -1 and got[5] == -1
    ok = [i for i in range(20) if i not in (3, 5)]
    assert np.array_equal(got[ok].astype(np.int64), orc.eval_population_assign(o, pop[ok]))
    gpu.ffs_assign_eval(g, dev(pop), 0, 32, out)        # N = 0 is a no-op
    with pytest.raises(gpu.FFSError):
        gpu.ffs_assign_eval(g, dev(pop), 20, 24, out)   # ld < n * S
    with pytest.raises(gpu.FFSError):
        gpu.ffs_assign_eval(g, dev(pop), 20, 36, out)   # ld not a multiple of 8
    with pytest.raises(gpu.FFSError):
        gpu.AssignInstance(2, 1, [2], [[1, 0], [1, 1]])          # a time < 1
    with pytest.raises(gpu.FFSError):
        gpu.AssignInstance(2, 1, [33], np.ones((2, 33)))         # more than 32 machines
    with pytest.raises(gpu.FFSError):
        gpu.AssignInstance(2, 2, [1, 1], [[65535, 65535], [65535, 65535]], due=[0, 0], wt=10000)   # objective > int32


def test_assign_full_size_sampled(gpu):
    """500 jobs x 20 stages (10000 genes per row), 16384 rows: 150 sampled rows
    and the first and last against the oracle."""
    spec = make_assign_instance(500, 20, 5, 10, seed=1)
    o, g = _pair(spec, gpu)
    N = 16384
    pop = random_assignments(500, 20, spec.M, N, seed=5)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    gpu.ffs_assign_eval(g, dev(pop), N, pop.shape[1], out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.int64)
    rng = np.random.default_rng(6)
    idx = np.concatenate([[0, N - 1], rng.choice(N, 150, replace=False)])
    assert np.array_equal(got[idx], orc.eval_population_assign(o, pop[idx]))
    assert got.min() > 0
