"""GPU GA parity against the CPU oracle, bit-exact: Philox draws, initial
populations, cellular and pseudo generations (stateless calls), the islands
handle (CUDA-graph generations with ring and penetration migration) over
whole runs, and sampled cells at the 500 x 20 scale."""
import numpy as np
import pytest
import torch

import oracle as orc
from conftest import dev
from ffs_workloads import make_instance, random_population

pytestmark = pytest.mark.gpu


def _pair(spec, ffs):
    return orc.Instance(spec.n, spec.S, spec.M, spec.p), ffs.Instance(spec.n, spec.S, spec.M, spec.p)


def _params(ffs, seed=7, cell_pc=1.0, cell_pm=0.05, pseudo_pc=0.75, le=False, always=False,
            mode=1, gap=50, ring=(2, 100), theta=(1, 1), decode_variant=0, chunk=0, threads=0):
    p = ffs.ffs_params_default()
    p.decode_variant = decode_variant
    p.decode_chunk, p.block_threads = chunk, threads
    p.seed = seed
    p.cell_pc, p.cell_pm, p.pseudo_pc = ffs.threshold(cell_pc), ffs.threshold(cell_pm), ffs.threshold(pseudo_pc)
    p.cell_replace_le, p.pseudo_always = int(le), int(always)
    p.migration_mode, p.migration_gap = mode, gap
    p.ring_num, p.ring_den = ring
    p.theta_num, p.theta_den = theta
    o = orc.Params(seed=seed, cell_pc=cell_pc, cell_pm=cell_pm, pseudo_pc=pseudo_pc,
                   cell_replace_le=le, pseudo_always=always)
    return p, o


def test_philox_draws_match_oracle(gpu):
    out = torch.zeros((37, 11), dtype=torch.int64, device="cuda").to(torch.int32)
    for seed, purpose, isl, gen, cell0 in [(7, 2, 0, 1, 0), (2**63 + 5, 3, 5, 999, 77), (0, 1, 2**23, 0, 2**31)]:
        gpu.ffs_philox_draws(seed, purpose, isl, gen, cell0, 37, 11, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        for c in (0, 1, 17, 36):
            want = [orc.draw(seed, purpose, isl, gen, (cell0 + c) & 0xFFFFFFFF, d) for d in range(11)]
            assert got[c].tolist() == want


def test_population_init_matches_oracle(gpu):
    spec = make_instance(37, 3, 1, 3, seed=2)
    _, g = _pair(spec, gpu)
    ld = 40
    pop = torch.full((20, ld), 99, dtype=torch.int16, device="cuda")
    gpu.ffs_population_init(g, 7, 3, 0, 20, ld, pop)
    torch.cuda.synchronize()
    got = pop.cpu().numpy()
    for c in range(20):
        assert got[c, :37].tolist() == orc.init_chromosome(7, 3, c, 37).tolist()
        assert not got[c, 37:].any()
    gpu.ffs_population_init(g, 11, 1, 1, 20, ld, pop)
    torch.cuda.synchronize()
    got = pop.cpu().numpy()
    for k in range(10):
        a, b = orc.init_pseudo_pair(11, 1, k, 37)
        assert got[2 * k, :37].tolist() == a.tolist() and got[2 * k + 1, :37].tolist() == b.tolist()


@pytest.mark.parametrize("variant", [dict(), dict(cell_pc=0.6, cell_pm=1.0), dict(le=True, cell_pm=0.3),
                                     dict(cell_pc=0.0, cell_pm=0.0), dict(decode_variant=1),
                                     dict(decode_variant=2, cell_pm=0.5), dict(decode_variant=3),
                                     dict(decode_variant=4)])
def test_cellular_generations_match_oracle(gpu, variant):
    spec = make_instance(20, 5, 3, 3, seed=1)
    o, g = _pair(spec, gpu)
    prm, oprm = _params(gpu, **variant)
    rows, cols, ld = 8, 8, 24
    pop = np.zeros((64, ld), dtype=np.int16)
    for c in range(64):
        pop[c, :20] = orc.init_chromosome(7, 0, c, 20)
    ms = orc.eval_population(o, pop)
    a, b = dev(pop), torch.zeros((64, ld), dtype=torch.int16, device="cuda")
    ma, mb = dev(ms.astype(np.int32)), torch.zeros(64, dtype=torch.int32, device="cuda")
    for gen in range(1, 31):
        pop, ms, _ = orc.cellular_generation(o, oprm, 0, gen, rows, cols, pop, ms)
        gpu.ffs_cellular_step(g, prm, 0, gen, rows, cols, ld, a, ma, b, mb)
        torch.cuda.synchronize()
        assert np.array_equal(b.cpu().numpy()[:, :20], pop[:, :20]), gen
        assert np.array_equal(mb.cpu().numpy().astype(np.int64), ms), gen
        a, b, ma, mb = b, a, mb, ma


@pytest.mark.parametrize("always,dvar", [(False, 0), (True, 0), (False, 1), (False, 3)])
@pytest.mark.parametrize("shape", [(20, 5, 3, 3, 64), (100, 10, 2, 5, 512), (33, 4, 1, 6, 130), (45, 7, 1, 20, 96)])
def test_pseudo_generations_match_oracle(gpu, always, dvar, shape):
    n, S, mlo, mhi, size = shape
    spec = make_instance(n, S, mlo, mhi, seed=n + S)
    o, g = _pair(spec, gpu)
    prm, oprm = _params(gpu, seed=5, always=always, decode_variant=dvar)
    ld = (n + 7) // 8 * 8
    pop = np.zeros((size, ld), dtype=np.int16)
    for k in range(size // 2):
        x, y = orc.init_pseudo_pair(5, 1, k, n)
        pop[2 * k, :n], pop[2 * k + 1, :n] = x, y
    ms = orc.eval_population(o, pop)
    scratch = torch.empty(gpu.ffs_pseudo_scratch_bytes(size, ld), dtype=torch.uint8, device="cuda")
    a, b = dev(pop), torch.zeros((size, ld), dtype=torch.int16, device="cuda")
    ma, mb = dev(ms.astype(np.int32)), torch.zeros(size, dtype=torch.int32, device="cuda")
    for gen in range(1, 11):
        pop, ms, _ = orc.pseudo_generation(o, oprm, 1, gen, pop, ms)
        gpu.ffs_pseudo_step(g, prm, 1, gen, size, ld, a, ma, b, mb, scratch)
        torch.cuda.synchronize()
        assert np.array_equal(b.cpu().numpy()[:, :n], pop[:, :n]), gen
        assert np.array_equal(mb.cpu().numpy().astype(np.int64), ms), gen
        a, b, ma, mb = b, a, mb, ma


def _islands_vs_oracle(gpu, spec, prm, oprm, n_cell, rows, cols, n_pseudo, psize, gens, gap, mode,
                       check_every=1):
    o, g = _pair(spec, gpu)
    isl = gpu.Islands(g, prm, n_cell, rows, cols, n_pseudo, psize)
    ga = orc.IslandGA(o, oprm, n_cell, rows, cols, n_pseudo, psize)
    assert isl.kinds == ga.kinds and isl.sizes == ga.sizes

    def compare(tag):
        for i in range(isl.n_islands):
            pop, ms = gpu.island_tensors(isl, i)
            torch.cuda.synchronize()
            assert np.array_equal(pop.cpu().numpy(), ga.pops[i][:, :spec.n]), (tag, i)
            assert np.array_equal(ms.cpu().numpy().astype(np.int64), ga.mss[i]), (tag, i)

    compare("init")
    done = 0
    while done < gens:
        step = min(check_every, gens - done)
        gpu.ffs_island_step(isl, -1, step)
        for _ in range(step):
            ga.step()
            done += 1
            if gap and done % gap == 0 and len(ga.kinds) > 1:
                if mode == gpu.FFS_MIG_RING:
                    ga.migrate_ring(prm.ring_num, prm.ring_den)
                else:
                    ga.migrate_penetration(prm.theta_num, prm.theta_den)
        compare(done)
    assert isl.generation() == gens
    best = gpu.ffs_islands_best(isl)
    assert best[0] == ga.best()
    decoded = gpu.ffs_islands_decoded(isl)
    assert decoded == ga.decoded
    return isl, ga


def test_islands_tiny_100_generations(gpu):
    """20 x 5, 3 machines per stage, one 8x8 cellular island, 100 generations, seed 7."""
    spec = make_instance(20, 5, 3, 3, seed=1)
    prm, oprm = _params(gpu, mode=0, gap=0)
    _islands_vs_oracle(gpu, spec, prm, oprm, 1, 8, 8, 0, 0, 100, 0, 0, check_every=1)


def test_islands_dual_ring(gpu):
    """100 x 10, M_s in [2,5]: 64x64 cellular + pseudo 4096, ring 2% every 50 generations."""
    spec = make_instance(100, 10, 2, 5, seed=1)
    prm, oprm = _params(gpu, mode=1, gap=50)
    _islands_vs_oracle(gpu, spec, prm, oprm, 1, 64, 64, 1, 4096, 120, 50, 1, check_every=10)


def test_islands_penetration_multi(gpu):
    spec = make_instance(30, 4, 1, 3, seed=3)
    prm, oprm = _params(gpu, seed=9, mode=2, gap=4, theta=(1, 1))
    _islands_vs_oracle(gpu, spec, prm, oprm, 2, 6, 6, 2, 36, 24, 4, 2, check_every=2)


def test_islands_ring_uneven_three(gpu):
    spec = make_instance(12, 3, 1, 4, seed=8)
    prm, oprm = _params(gpu, seed=3, mode=1, gap=3, ring=(10, 100))
    _islands_vs_oracle(gpu, spec, prm, oprm, 2, 5, 4, 1, 30, 12, 3, 1, check_every=3)


def test_islands_fused_generation_flags(gpu):
    """Both kinds in one generation (breeding launch + decode launch) with the
    replace-if-not-worse flag and the children-always-replace flag."""
    spec = make_instance(40, 6, 2, 4, seed=14)
    prm, oprm = _params(gpu, seed=21, le=True, always=True, cell_pm=0.4, mode=1, gap=3)
    _islands_vs_oracle(gpu, spec, prm, oprm, 2, 8, 8, 2, 48, 9, 3, 1, check_every=3)


@pytest.mark.parametrize("mode", [1, 2])
def test_islands_odd_sizes_migration(gpu, mode):
    """Islands of an odd number of rows (5 x 5 tori): the ranking's per-island
    key offsets and shared-memory staging take their odd-length paths."""
    spec = make_instance(18, 4, 1, 4, seed=16)
    prm, oprm = _params(gpu, seed=13, mode=mode, gap=2, ring=(10, 100), theta=(1, 1))
    _islands_vs_oracle(gpu, spec, prm, oprm, 2, 5, 5, 2, 26, 6, 2, mode, check_every=2)


def test_islands_more_than_one_batch_of_a_kind(gpu):
    """17 cellular islands (more than one launch batch) beside a pseudo island:
    generations take the per-kind launches instead of the fused pair."""
    spec = make_instance(16, 3, 1, 3, seed=15)
    prm, oprm = _params(gpu, seed=3, mode=1, gap=2, ring=(10, 100))
    _islands_vs_oracle(gpu, spec, prm, oprm, 17, 4, 4, 1, 16, 4, 2, 1, check_every=2)


@pytest.mark.parametrize("mode", [1, 2])
def test_islands_migration_full_size_islands(gpu, mode):
    """Migration every generation between islands of 16384 rows (128 x 128
    tori and 16384-row pseudo islands), the bench's island size: the ranking
    sorts eight chunks per island and merges them."""
    spec = make_instance(20, 5, 2, 4, seed=5)
    prm, oprm = _params(gpu, seed=5, mode=mode, gap=1, ring=(2, 100), theta=(1, 1))
    _islands_vs_oracle(gpu, spec, prm, oprm, 2, 128, 128, 2, 16384, 3, 1, mode, check_every=1)


@pytest.mark.parametrize("variant,threads,n_pseudo", [(4, 128, 1), (3, 256, 1), (4, 512, 0), (3, 128, 0)])
def test_islands_tensor_memory_heaps(gpu, variant, threads, n_pseudo):
    """Chunked decoding (8 jobs per round) with the saved heaps in tensor
    memory, in the fused decode launch (cellular + pseudo) and the cellular
    kernel alone."""
    spec = make_instance(60, 9, 1, 6, seed=12)
    prm, oprm = _params(gpu, seed=4, mode=1, gap=5, decode_variant=variant, chunk=8, threads=threads)
    o, g = _pair(spec, gpu)
    assert gpu.ffs_decode_plan(g, 2 if n_pseudo else 1, 8, threads, variant)["tmem_cols"] > 0
    _islands_vs_oracle(gpu, spec, prm, oprm, 2, 12, 12, n_pseudo, 64 if n_pseudo else 0, 12, 5, 1,
                       check_every=3)


def test_explicit_migrate_and_set_get(gpu):
    spec = make_instance(16, 3, 2, 3, seed=6)
    o, g = _pair(spec, gpu)
    prm, oprm = _params(gpu, mode=0, gap=0)
    isl = gpu.Islands(g, prm, 1, 4, 4, 1, 16)
    ga = orc.IslandGA(o, oprm, 1, 4, 4, 1, 16)
    gpu.ffs_island_step(isl, -1, 3)
    for _ in range(3):
        ga.step()
    gpu.ffs_migrate(isl, gpu.FFS_MIG_PENETRATION)
    ga.migrate_penetration()
    gpu.ffs_migrate(isl, gpu.FFS_MIG_RING)
    ga.migrate_ring(2, 100)   # the handle's fraction: 2% of 16 rows -> k = 1
    for i in range(2):
        pop, ms = gpu.island_tensors(isl, i)
        torch.cuda.synchronize()
        assert np.array_equal(pop.cpu().numpy(), ga.pops[i][:, :16])
        assert np.array_equal(ms.cpu().numpy().astype(np.int64), ga.mss[i])
    # host round trip through set/get
    host_pop = np.ascontiguousarray(ga.pops[1][:, :16][::-1])
    host_ms = np.ascontiguousarray(ga.mss[1][::-1].astype(np.int32))
    gpu.ffs_islands_set(isl, 1, host_pop, 16, host_ms)
    back_pop = np.zeros_like(host_pop)
    back_ms = np.zeros_like(host_ms)
    gpu.ffs_islands_get(isl, 1, back_pop, 16, back_ms)
    torch.cuda.synchronize()
    assert np.array_equal(back_pop, host_pop) and np.array_equal(back_ms, host_ms)
    # single-island stepping diverges generation counts; all-island step then refuses
    gpu.ffs_island_step(isl, 0, 1)
    with pytest.raises(gpu.FFSError):
        gpu.ffs_island_step(isl, -1, 1)


@pytest.mark.parametrize("shape", [(0, 0, 0), (384, 128, 3), (384, 104, 3)], ids=["library", "bench128", "bench104"])
def test_scale_500x20_sampled_generation(gpu, shape):
    """4 x 128^2 cellular + 4 x 16384 pseudo at 500 x 20: one generation of
    every island, checked on sampled cells and pairs with the oracle, at the
    library's launch shape and at the one bench.py times (384 threads,
    chunk 128, variant 3)."""
    spec = make_instance(500, 20, 5, 10, seed=1)
    o, g = _pair(spec, gpu)
    threads, chunk, variant = shape
    prm, oprm = _params(gpu, mode=0, gap=0, decode_variant=variant, chunk=chunk, threads=threads)
    isl = gpu.Islands(g, prm, 4, 128, 128, 4, 16384)
    before = [gpu.island_tensors(isl, i) for i in range(isl.n_islands)]
    before = [(p.cpu().numpy(), m.cpu().numpy().astype(np.int64)) for p, m in before]
    # initial rows are the oracle's initial rows
    for i in (0, 1, 6, 7):
        for c in (0, 5, 16383):
            if isl.kinds[i] == "cellular":
                assert before[i][0][c].tolist() == orc.init_chromosome(7, i, c, 500).tolist()
    gpu.ffs_island_step(isl, -1, 1)
    after = [gpu.island_tensors(isl, i) for i in range(isl.n_islands)]
    after = [(p.cpu().numpy(), m.cpu().numpy().astype(np.int64)) for p, m in after]
    rng = np.random.default_rng(2)
    for i in (0, 2):   # ring order [cell 0, pseudo 0, cell 1, ...]: cellular islands 0 and 1
        pop, ms = before[i]
        for c in rng.choice(16384, 40, replace=False).tolist() + [0, 127, 16383]:
            x = [orc.draw(7, orc.PURPOSE_CELLULAR, i, 1, c, d) for d in range(10)]
            child, _ = orc.cellular_child(o, oprm, 128, 128, c, x, pop, ms)
            mc = orc.decode(o, child)
            if mc < ms[c]:
                assert after[i][0][c].tolist() == child.tolist() and after[i][1][c] == mc
            else:
                assert after[i][0][c].tolist() == pop[c].tolist() and after[i][1][c] == ms[c]
    for i in (1, 7):
        pop, ms = before[i]
        for k in rng.choice(8192, 30, replace=False).tolist() + [0, 8191]:
            a, b = pop[2 * k], pop[2 * k + 1]
            x0, x1, x2 = (orc.draw(7, orc.PURPOSE_PSEUDO, i, 1, k, d) for d in range(3))
            if not orc.bernoulli(x0, oprm._c().pseudo_pc):
                want = [(a, ms[2 * k]), (b, ms[2 * k + 1])]
            else:
                u, v = orc.uniform(x1, 500), orc.uniform(x2, 500)
                c1 = orc.order_crossover(a, b, min(u, v), max(u, v))
                c2 = orc.order_crossover(b, a, min(u, v), max(u, v))
                fam = [(c1, orc.decode(o, c1)), (c2, orc.decode(o, c2)), (a, ms[2 * k]), (b, ms[2 * k + 1])]
                pick = orc.family_best2([f[1] for f in fam])
                want = [fam[pick[0]], fam[pick[1]]]
            for t in range(2):
                assert after[i][0][2 * k + t].tolist() == want[t][0].tolist()
                assert after[i][1][2 * k + t] == want[t][1]


def test_get_set_all_islands(gpu):
    """ffs_islands_get_all / set_all move every island's rows in ring order in one call."""
    spec = make_instance(24, 3, 2, 3, seed=2)
    o, g = _pair(spec, gpu)
    prm, _ = _params(gpu, mode=0, gap=0)
    isl = gpu.Islands(g, prm, 2, 4, 4, 1, 10)
    gpu.ffs_island_step(isl, -1, 2)
    total = sum(isl.sizes)
    pop = torch.zeros((total, isl.ld), dtype=torch.int16)
    ms = torch.zeros(total, dtype=torch.int32)
    gpu.ffs_islands_get_all(isl, pop, isl.ld, ms)
    torch.cuda.synchronize()
    row = 0
    for i in range(isl.n_islands):
        p_i, m_i = gpu.island_tensors(isl, i)
        torch.cuda.synchronize()
        N = isl.sizes[i]
        assert np.array_equal(pop[row:row + N, :spec.n].numpy(), p_i.cpu().numpy())
        assert np.array_equal(ms[row:row + N].numpy(), m_i.cpu().numpy())
        row += N
    rev = torch.flip(pop, dims=[0]).contiguous()
    rms = torch.flip(ms, dims=[0]).contiguous()
    gpu.ffs_islands_set_all(isl, rev, isl.ld, rms)
    back = torch.zeros_like(pop)
    bms = torch.zeros_like(ms)
    gpu.ffs_islands_get_all(isl, back, isl.ld, bms)
    torch.cuda.synchronize()
    assert torch.equal(back, rev) and torch.equal(bms, rms)
