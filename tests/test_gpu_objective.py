"""GPU parity for the paper's objective (arXiv:1903.10722, Section 3, Table 1):
release times at the first stage, due times, WT * total tardiness + C_max.
Bit-exact against the CPU oracle over instance shapes, launch shapes and
decoder variants (the first stage reads release times, the last stage sums
tardiness, in both the one-stage and the stage-pair decoder), then through
the cellular, pseudo and dual-island generations."""
import numpy as np
import pytest
import torch

import oracle as orc
from conftest import dev
from ffs_workloads import make_instance, make_paper_instance, random_population

pytestmark = pytest.mark.gpu


def _with_objective(spec, seed):
    """A Table-1 style objective on any instance: R ~ U{0..Pbar/4}, D = R + Pbar_j (1 + U[0,2))."""
    rng = np.random.default_rng(seed)
    pbar_j = spec.p.sum(axis=1).astype(np.int64)
    R = rng.integers(0, max(1, int(pbar_j.sum()) // 4) + 1, size=spec.n)
    D = R + np.floor(pbar_j * (1.0 + 2.0 * rng.random(spec.n))).astype(np.int64)
    return R.astype(np.int32), D.astype(np.int32)


def _pair(spec, gpu, R, D, wt):
    return (orc.Instance(spec.n, spec.S, spec.M, spec.p, release=R, due=D, wt=wt),
            gpu.Instance(spec.n, spec.S, spec.M, spec.p, release=R, due=D, wt=wt))


SHAPES = [
    # n, S, m_lo, m_hi, N
    (300, 4, 2, 2, 200),      # the paper's 300 x 4 x 2 shape (Table 1 instance below)
    (100, 10, 2, 5, 300),
    (33, 1, 2, 5, 70),        # one stage: release and tardiness in the same stage
    (57, 3, 1, 32, 90),       # catch-all heap size
    (500, 20, 5, 10, 96),
]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[0]}x{s[1]}" for s in SHAPES])
def test_objective_eval_matches_oracle(gpu, shape):
    n, S, mlo, mhi, N = shape
    spec = (make_paper_instance(n, S, mlo, seed=2) if (n, S) == (300, 4)
            else make_instance(n, S, mlo, mhi, seed=n + S))
    R, D = (spec.release, spec.due) if spec.release is not None else _with_objective(spec, n)
    # the largest WT <= 100 whose objective bound fits int32 (the library checks the same bound)
    horizon = int(R.max()) + int(spec.p.sum())
    wt = int(min(100, (2 ** 31 - 1 - horizon) // (n * horizon)))
    assert wt >= 1
    pop = random_population(n, N, seed=n * 7)
    d = dev(pop)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    for rel, due, wt in [(R, D, wt), (None, D, 1), (R, None, 0)]:
        o, g = _pair(spec, gpu, rel, due, wt)
        want = orc.eval_population(o, pop)
        for chunk, threads, variant in [(0, 0, 0), (8, 128, 1), (8, 128, 2), (16, 256, 3), (16, 448, 4),
                                        (0, 64, 1), (0, 64, 2)]:
            out.fill_(-7)
            try:
                gpu.ffs_population_eval_tuned(g, d, N, pop.shape[1], out, chunk, threads, variant)
            except gpu.FFSError as e:
                assert e.status == gpu.FFS_EUNSUPPORTED and (chunk, threads) != (0, 0)
                continue
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.int64)
            assert np.array_equal(got, want), (rel is None, due is None, chunk, threads, variant,
                                               np.flatnonzero(got != want)[:5])


def test_objective_rejects_overflow(gpu):
    spec = make_instance(50, 3, 2, 3, seed=1)
    R = np.zeros(50, dtype=np.int32)
    D = np.zeros(50, dtype=np.int32)
    with pytest.raises(gpu.FFSError) as e:
        gpu.Instance(spec.n, spec.S, spec.M, spec.p, release=R, due=D, wt=2 ** 30)
    assert e.value.status == gpu.FFS_EOVERFLOW
    with pytest.raises(gpu.FFSError) as e:
        gpu.Instance(spec.n, spec.S, spec.M, spec.p, release=R - 1, due=D, wt=1)
    assert e.value.status == gpu.FFS_EINVAL


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_objective_islands_match_oracle(gpu, variant):
    """The paper's configuration, scaled down: a Table-1 instance, a cellular
    and a pseudo island, penetration migration (theta = 1.00) every 3 generations."""
    spec = make_paper_instance(60, 4, 2, seed=5)
    o, g = _pair(spec, gpu, spec.release, spec.due, spec.wt)
    p = gpu.ffs_params_default()
    p.seed, p.decode_variant = 11, variant
    p.decode_chunk, p.block_threads = (16, 128) if variant else (0, 0)
    p.migration_mode, p.migration_gap = gpu.FFS_MIG_PENETRATION, 3
    p.theta_num, p.theta_den = 1, 1
    oprm = orc.Params(seed=11)
    isl = gpu.Islands(g, p, 1, 8, 8, 1, 64)
    ga = orc.IslandGA(o, oprm, 1, 8, 8, 1, 64)
    for gen in range(1, 10):
        gpu.ffs_island_step(isl, -1, 1)
        ga.step()
        if gen % 3 == 0:
            ga.migrate_penetration(1, 1)
        for i in range(isl.n_islands):
            pop, ms = gpu.island_tensors(isl, i)
            torch.cuda.synchronize()
            assert np.array_equal(pop.cpu().numpy(), ga.pops[i][:, :spec.n]), (gen, i)
            assert np.array_equal(ms.cpu().numpy().astype(np.int64), ga.mss[i]), (gen, i)
    assert gpu.ffs_islands_best(isl)[0] == ga.best()
