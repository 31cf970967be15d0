"""The stage-parallel decoder (variant 5: lane s of a group runs stage s of
one chromosome) against the CPU oracle, element by element: edge shapes
(one job, one stage, M_s >= n, 32 machines, 32 stages), ragged counts of
chromosomes, the paper's objective with release and due times, invalid
genes."""
import numpy as np
import pytest
import torch

import oracle as orc
from conftest import dev
from ffs_workloads import make_instance, random_population

pytestmark = pytest.mark.gpu

SHAPES = [
    # n, S, m_lo, m_hi, N
    (1, 1, 1, 1, 5),
    (1, 7, 1, 3, 33),
    (9, 1, 2, 5, 100),
    (12, 3, 20, 32, 64),        # M_s >= n: clamped to n
    (40, 4, 32, 32, 97),        # 32 machines per stage (the 32-slot heap)
    (37, 5, 1, 1, 31),          # permutation flow shop
    (100, 10, 2, 5, 1000),      # the 100 x 10 family: 3 chromosomes per warp
    (60, 11, 2, 9, 257),        # 2 per warp, 10 idle lanes
    (80, 17, 3, 6, 129),        # one per warp
    (33, 32, 1, 4, 70),         # 32 stages: every lane of the warp
    (500, 20, 5, 10, 300),      # the 500 x 20 family
    (300, 4, 2, 2, 512),        # the paper's shape
]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[0]}x{s[1]}m{s[2]}-{s[3]}N{s[4]}" for s in SHAPES])
def test_lanes_decoder_matches_oracle(gpu, shape):
    n, S, lo, hi, N = shape
    spec = make_instance(n, S, lo, hi, seed=n + 3 * S)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    pop = random_population(n, N, seed=N)
    out = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    gpu.ffs_population_eval_tuned(g, dev(pop), N, pop.shape[1], out, 0, 0, 5)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().astype(np.int64), orc.eval_population(o, pop))


@pytest.mark.parametrize("shape", [(300, 4, 2, 2, 256), (50, 6, 1, 4, 77), (20, 3, 5, 5, 40)])
def test_lanes_decoder_objective(gpu, shape):
    """Release times (stage 1 starts at max(machine free, R_j)), due times and
    WT x total tardiness."""
    n, S, lo, hi, N = shape
    spec = make_instance(n, S, lo, hi, p_lo=1, p_hi=5 if n == 300 else 40, seed=S)
    rng = np.random.default_rng(n)
    pbar = spec.p.sum(axis=1)
    R = rng.integers(0, int(pbar.sum()) // 4 + 1, size=n).astype(np.int32)
    D = (R + np.floor(pbar * (1.0 + 2.0 * rng.random(n)))).astype(np.int32)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p, release=R, due=D, wt=100)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p, release=R, due=D, wt=100)
    pop = random_population(n, N, seed=3)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    gpu.ffs_population_eval_tuned(g, dev(pop), N, pop.shape[1], out, 0, 0, 5)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().astype(np.int64), orc.eval_population(o, pop))


def test_lanes_decoder_invalid_genes_and_routing(gpu):
    spec = make_instance(30, 6, 2, 4, seed=5)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    pop = random_population(30, 50, seed=2)
    pop[4, 3] = 30
    pop[9, 0] = -1
    pop[49, 29] = 31000
    want = orc.eval_population(o, pop)
    assert want[4] == want[9] == want[49] == -1
    for variant in (5, 0, 3):         # stage-parallel, the library's choice, one lane per chromosome
        out = torch.empty(50, dtype=torch.int32, device="cuda")
        gpu.ffs_population_eval_tuned(g, dev(pop), 50, pop.shape[1], out, 0, 0, variant)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), want), variant
    with pytest.raises(gpu.FFSError):
        gpu.ffs_population_eval_tuned(g, dev(pop), 50, pop.shape[1], out, 0, 0, 6)
    many = make_instance(10, 33, 1, 2, seed=1)
    g33 = gpu.Instance(many.n, many.S, many.M, many.p)
    p33 = random_population(10, 4, seed=1)
    with pytest.raises(gpu.FFSError) as e:
        gpu.ffs_population_eval_tuned(g33, dev(p33), 4, p33.shape[1], out, 0, 0, 5)
    assert e.value.status == gpu.FFS_EUNSUPPORTED
    # the library's choice for a 33-stage instance is one chromosome per lane
    o33 = orc.Instance(many.n, many.S, many.M, many.p)
    gpu.ffs_population_eval(g33, dev(p33), 4, p33.shape[1], out)
    torch.cuda.synchronize()
    assert np.array_equal(out[:4].cpu().numpy().astype(np.int64), orc.eval_population(o33, p33))
