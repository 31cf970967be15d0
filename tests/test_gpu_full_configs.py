"""Whole-population parity at the measured configurations, at full length or
with every row compared (integer results: exact equality).

  * 100 jobs x 10 stages (64x64 cellular + pseudo 4096, ring migration of 2%
    every 50 generations): all 1000 generations, every row of both islands
    compared every 50 generations.
  * 500 jobs x 20 stages (4 x 128x128 cellular + 4 x 16384 pseudo = 131072
    chromosomes) at the launch shape bench.py times (384 threads, chunk 104,
    one stage at a time with saved heaps in tensor memory): 3 generations
    with ring migration after every generation, every row of every island.
  * 256 uneven instances (n in [20, 500], S in [5, 20], M_s in [2, 10],
    32x32 tori) at the library's default launch shape: 10 generations, every
    row of 16 instances spread over the range of n x S.

The oracle splits each generation's independent cells and pairs over a
thread pool (its C calls release the GIL); every step it takes is the
plain sequential definition."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle as orc
from ffs_workloads import make_batch, workload_instance

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def pool():
    with ThreadPoolExecutor(THREADS) as ex:
        yield ex


def _compare_islands(gpu, isl, ga, n, tag, islands=None):
    for i in (islands if islands is not None else range(isl.n_islands)):
        pop, ms = gpu.island_tensors(isl, i)
        torch.cuda.synchronize()
        assert np.array_equal(pop.cpu().numpy(), ga.pops[i][:, :n]), (tag, i)
        assert np.array_equal(ms.cpu().numpy().astype(np.int64), ga.mss[i]), (tag, i)


def test_dual_100x10_all_1000_generations(gpu, pool):
    spec = workload_instance("dual_100x10")
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.migration_mode, prm.migration_gap = gpu.FFS_MIG_RING, 50
    isl = gpu.Islands(g, prm, 1, 64, 64, 1, 4096)
    ga = orc.IslandGA(o, orc.Params(seed=7), 1, 64, 64, 1, 4096, pool=pool, parts=THREADS)
    _compare_islands(gpu, isl, ga, spec.n, 0)
    for block in range(20):
        gpu.ffs_island_step(isl, -1, 50)
        for _ in range(50):
            ga.step_threads(pool, THREADS)
        ga.migrate_ring(prm.ring_num, prm.ring_den)       # after generation 50 (block + 1)
        _compare_islands(gpu, isl, ga, spec.n, 50 * (block + 1))
    assert isl.generation() == 1000
    assert gpu.ffs_islands_best(isl)[0] == ga.best()
    assert gpu.ffs_islands_decoded(isl) == ga.decoded


def test_scale_500x20_three_generations_every_row(gpu, pool):
    spec = workload_instance("scale_500x20")
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.migration_mode, prm.migration_gap = gpu.FFS_MIG_RING, 1
    prm.block_threads, prm.decode_chunk, prm.decode_variant = 384, 104, 3
    isl = gpu.Islands(g, prm, 4, 128, 128, 4, 16384)
    ga = orc.IslandGA(o, orc.Params(seed=7), 4, 128, 128, 4, 16384, pool=pool, parts=THREADS)
    _compare_islands(gpu, isl, ga, spec.n, 0)
    for gen in (1, 2, 3):
        gpu.ffs_island_step(isl, -1, 1)
        ga.step_threads(pool, THREADS)
        ga.migrate_ring(prm.ring_num, prm.ring_den)
        _compare_islands(gpu, isl, ga, spec.n, gen)
    assert gpu.ffs_islands_decoded(isl) == ga.decoded


def test_batch_256_ten_generations_sixteen_instances(gpu, pool):
    specs = make_batch(256, seed=1)
    rows = cols = 32
    prm = gpu.ffs_params_default()
    oprm = orc.Params(seed=7)
    b = gpu.Batch(specs, prm, rows, cols)      # the library's default launch shape
    order = sorted(range(len(specs)), key=lambda i: specs[i].n * specs[i].S)
    chosen = order[::16]
    assert len(chosen) == 16
    states = {}
    for i in chosen:
        s = specs[i]
        o = orc.Instance(s.n, s.S, s.M, s.p)
        ld = (s.n + 7) // 8 * 8
        pop = np.zeros((rows * cols, ld), dtype=np.int16)
        for c in range(rows * cols):
            pop[c, :s.n] = orc.init_chromosome(7, i, c, s.n)
        states[i] = [o, pop, orc.eval_population_threads(o, pop, pool, THREADS)]

    def compare(tag):
        for i in chosen:
            pop, ms = gpu.batch_tensors(b, i)
            torch.cuda.synchronize()
            assert np.array_equal(pop.cpu().numpy(), states[i][1][:, :specs[i].n]), (tag, i)
            assert np.array_equal(ms.cpu().numpy().astype(np.int64), states[i][2]), (tag, i)

    compare(0)
    for gen in range(1, 11):
        gpu.ffs_batch_step(b, 1)
        for i in chosen:
            o, pop, ms = states[i]
            pop, ms, _ = orc.cellular_generation_threads(o, oprm, i, gen, rows, cols, pop, ms, pool, THREADS)
            states[i] = [o, pop, ms]
        compare(gen)
    best = gpu.ffs_batch_best(b)
    for i in chosen:
        assert best[i] == states[i][2].min()
    gpu.ffs_batch_check(b)
