"""Batched uneven instances (one cellular island per instance, one persistent
launch per generation from a CUDA graph) against the CPU oracle, bit-exact;
launch shapes from the autotuner must not change results."""
import numpy as np
import pytest
import torch

import oracle as orc
from ffs_workloads import InstanceSpec, make_batch, make_instance

pytestmark = pytest.mark.gpu


def _oracle_state(spec, island, rows, cols, seed=7):
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    ld = (spec.n + 7) // 8 * 8
    pop = np.zeros((rows * cols, ld), dtype=np.int16)
    for c in range(rows * cols):
        pop[c, :spec.n] = orc.init_chromosome(seed, island, c, spec.n)
    return o, pop, orc.eval_population(o, pop)


def _mixed_specs():
    shapes = [(1, 1, 1, 1), (7, 3, 2, 4), (20, 5, 3, 3), (37, 6, 1, 8), (60, 2, 5, 32), (100, 8, 2, 5),
              (13, 1, 4, 4), (250, 4, 2, 10), (44, 7, 1, 1), (3, 5, 2, 6), (90, 3, 9, 10), (17, 2, 1, 3)]
    return [make_instance(n, S, lo, hi, seed=k + 3) for k, (n, S, lo, hi) in enumerate(shapes)]


def test_batch_mixed_instances_match_oracle(gpu):
    specs = _mixed_specs()
    rows, cols = 6, 5          # 30 cells: tiles end part-way through a warp
    prm = gpu.ffs_params_default()
    oprm = orc.Params(seed=7)
    b = gpu.Batch(specs, prm, rows, cols)
    states = [_oracle_state(s, i, rows, cols) for i, s in enumerate(specs)]

    def compare(tag):
        for i, s in enumerate(specs):
            pop, ms = gpu.batch_tensors(b, i)
            torch.cuda.synchronize()
            assert np.array_equal(pop.cpu().numpy(), states[i][1][:, :s.n]), (tag, i)
            assert np.array_equal(ms.cpu().numpy().astype(np.int64), states[i][2]), (tag, i)

    compare("init")
    gen = 0
    for block in range(4):
        gpu.ffs_batch_step(b, 3)
        for _ in range(3):
            gen += 1
            for i, s in enumerate(specs):
                o, pop, ms = states[i]
                pop, ms, _ = orc.cellular_generation(o, oprm, i, gen, rows, cols, pop, ms)
                states[i] = (o, pop, ms)
        compare(gen)
    best = gpu.ffs_batch_best(b)
    assert best.tolist() == [int(st[2].min()) for st in states]
    assert gpu.ffs_batch_decoded(b) == gen * len(specs) * rows * cols
    assert b.info()["generation"] == gen
    gpu.ffs_batch_check(b)


def _many_stage_specs():
    """Instances of 17 to 20 stages (2S > 32 stage-table entries, so more than
    one warp copies the table into shared memory) mixed with short ones, in
    an order that puts different stage counts in consecutive work units."""
    shapes = [(120, 20, 2, 10), (9, 3, 2, 4), (64, 17, 3, 6), (200, 19, 5, 10), (31, 5, 1, 8),
              (150, 18, 2, 3), (77, 20, 6, 9), (40, 2, 4, 4)]
    return [make_instance(n, S, lo, hi, seed=k + 11) for k, (n, S, lo, hi) in enumerate(shapes)]


@pytest.mark.parametrize("variant,threads,chunk", [(3, 64, 16), (4, 128, 32), (3, 320, 24), (4, 512, 64),
                                                   (1, 128, 16), (2, 192, 32)])
def test_batch_many_stages_match_oracle(gpu, variant, threads, chunk):
    """Every block computes each work unit's decode layout (which stages keep
    their saved heaps in tensor memory) from the instance's own stage table,
    whatever instance its previous unit had: 6 generations of instances with
    up to 20 stages at launch shapes with and without tensor-memory heaps."""
    specs = _many_stage_specs()
    rows, cols = 8, 8
    prm = gpu.ffs_params_default()
    prm.decode_variant, prm.decode_chunk, prm.block_threads = variant, chunk, threads
    oprm = orc.Params(seed=7)
    b = gpu.Batch(specs, prm, rows, cols)
    states = [_oracle_state(s, i, rows, cols) for i, s in enumerate(specs)]
    gpu.ffs_batch_step(b, 6)
    for gen in range(1, 7):
        for i, s in enumerate(specs):
            o, pop, ms = states[i]
            pop, ms, _ = orc.cellular_generation(o, oprm, i, gen, rows, cols, pop, ms)
            states[i] = (o, pop, ms)
    gpu.ffs_batch_check(b)
    for i, s in enumerate(specs):
        pop, ms = gpu.batch_tensors(b, i)
        torch.cuda.synchronize()
        assert np.array_equal(pop.cpu().numpy(), states[i][1][:, :s.n]), i
        assert np.array_equal(ms.cpu().numpy().astype(np.int64), states[i][2]), i


@pytest.mark.parametrize("which", ["mixed", "many_stages"])
def test_batch_autotune_then_generations_match_oracle(gpu, which):
    """The autotuner times every launch shape on generations that do not
    advance the state (after it the rows, makespans and generation count are
    the initial ones); generations at the shape it keeps then match the
    oracle."""
    specs = _mixed_specs() if which == "mixed" else _many_stage_specs()
    rows, cols = 6, 5
    b = gpu.Batch(specs, gpu.ffs_params_default(), rows, cols)
    before = [tuple(t.cpu() for t in gpu.batch_tensors(b, i)) for i in range(len(specs))]
    tuned = gpu.ffs_batch_autotune(b, repeats=1)
    assert tuned["threads"] > 0 and tuned["chunk"] > 0 and tuned["ms"] > 0
    for i in range(len(specs)):
        pop, ms = gpu.batch_tensors(b, i)
        torch.cuda.synchronize()
        assert torch.equal(pop.cpu(), before[i][0]) and torch.equal(ms.cpu(), before[i][1]), i
    assert b.info()["generation"] == 0 and gpu.ffs_batch_decoded(b) == 0
    # dry runs (a whole generation, then the decode launch alone) change nothing either
    gpu.ffs_batch_dry_run(b, 0)
    gpu.ffs_batch_dry_run(b, 1)
    gpu.ffs_batch_dry_run(b, 1)
    for i in range(len(specs)):
        pop, ms = gpu.batch_tensors(b, i)
        torch.cuda.synchronize()
        assert torch.equal(pop.cpu(), before[i][0]) and torch.equal(ms.cpu(), before[i][1]), i
    assert b.info()["generation"] == 0 and gpu.ffs_batch_decoded(b) == 0
    with pytest.raises(gpu.FFSError):
        gpu.ffs_batch_dry_run(b, 2)
    gpu.ffs_batch_check(b)
    oprm = orc.Params(seed=7)
    states = [_oracle_state(s, i, rows, cols) for i, s in enumerate(specs)]
    gpu.ffs_batch_step(b, 3)
    for gen in range(1, 4):
        for i, s in enumerate(specs):
            o, pop, ms = states[i]
            pop, ms, _ = orc.cellular_generation(o, oprm, i, gen, rows, cols, pop, ms)
            states[i] = (o, pop, ms)
    gpu.ffs_batch_check(b)
    for i, s in enumerate(specs):
        pop, ms = gpu.batch_tensors(b, i)
        torch.cuda.synchronize()
        assert np.array_equal(pop.cpu().numpy(), states[i][1][:, :s.n]), (tuned, i)
        assert np.array_equal(ms.cpu().numpy().astype(np.int64), states[i][2]), (tuned, i)


def test_batch_256_uneven_sampled(gpu):
    """256 instances, n in [20,500], S in [5,20], M in [2,10], 32x32 torus each."""
    specs = make_batch(256, seed=1)
    rows = cols = 32
    prm = gpu.ffs_params_default()
    oprm = orc.Params(seed=7)
    b = gpu.Batch(specs, prm, rows, cols)
    order = sorted(range(256), key=lambda i: specs[i].n * specs[i].S)
    sample = sorted(set([order[0], order[1], order[-1], order[-2], order[128], 0, 255]))
    before = {i: [t.cpu().numpy() for t in gpu.batch_tensors(b, i)] for i in sample}
    for i in sample:
        for c in (0, 513, 1023):
            assert before[i][0][c].tolist() == orc.init_chromosome(7, i, c, specs[i].n).tolist()
    gpu.ffs_batch_step(b, 1)
    after = {i: [t.cpu().numpy() for t in gpu.batch_tensors(b, i)] for i in sample}
    rng = np.random.default_rng(4)
    for i in sample:
        s = specs[i]
        o = orc.Instance(s.n, s.S, s.M, s.p)
        ld = (s.n + 7) // 8 * 8
        pop = np.zeros((rows * cols, ld), dtype=np.int16)
        pop[:, :s.n] = before[i][0]
        ms = before[i][1].astype(np.int64)
        assert np.array_equal(ms, orc.eval_population(o, pop)[:]) if s.n * s.S < 2000 else True
        for c in rng.choice(1024, 12, replace=False).tolist() + [0, 1023]:
            x = [orc.draw(7, orc.PURPOSE_CELLULAR, i, 1, c, d) for d in range(10)]
            child, _ = orc.cellular_child(o, oprm, rows, cols, c, x, pop, ms)
            mc = orc.decode(o, child)
            if mc < ms[c]:
                assert after[i][0][c].tolist() == child[:s.n].tolist() and after[i][1][c] == mc, (i, c)
            else:
                assert after[i][0][c].tolist() == pop[c, :s.n].tolist() and after[i][1][c] == ms[c], (i, c)


@pytest.mark.parametrize("variant,threads,chunk", [(3, 128, 8), (4, 256, 8), (3, 448, 8), (4, 320, 8), (3, 384, 24),
                                                   (4, 448, 40)])
def test_batch_tensor_memory_heaps_match_oracle(gpu, variant, threads, chunk):
    """Chunked decoding (8 jobs per round) with each instance's saved heaps in
    tensor memory as far as its stages fit the warp's columns."""
    specs = _mixed_specs()
    rows, cols = 6, 5
    prm = gpu.ffs_params_default()
    prm.decode_variant, prm.decode_chunk, prm.block_threads = variant, chunk, threads
    oprm = orc.Params(seed=7)
    b = gpu.Batch(specs, prm, rows, cols)
    assert b.info()["variant"] == variant
    states = [_oracle_state(s, i, rows, cols) for i, s in enumerate(specs)]
    gpu.ffs_batch_step(b, 4)
    for gen in range(1, 5):
        for i, s in enumerate(specs):
            o, pop, ms = states[i]
            pop, ms, _ = orc.cellular_generation(o, oprm, i, gen, rows, cols, pop, ms)
            states[i] = (o, pop, ms)
    gpu.ffs_batch_check(b)
    for i, s in enumerate(specs):
        pop, ms = gpu.batch_tensors(b, i)
        torch.cuda.synchronize()
        assert np.array_equal(pop.cpu().numpy(), states[i][1][:, :s.n]), i
        assert np.array_equal(ms.cpu().numpy().astype(np.int64), states[i][2]), i


def test_batch_rejects_more_than_32_machines_below_n(gpu):
    """The decoder keeps at most 32 machine free times per stage in registers:
    an instance with min(M_s, n) > 32 is refused with FFS_EUNSUPPORTED (and
    the batch is not created); M_s >= n clamps to n and is accepted."""
    prm = gpu.ffs_params_default()
    specs = [make_instance(20, 3, 2, 4, seed=1), make_instance(100, 3, 40, 40, seed=2)]
    with pytest.raises(gpu.FFSError) as e:
        gpu.Batch(specs, prm, 4, 4)
    assert e.value.status == gpu.FFS_EUNSUPPORTED and "instance 1" in str(e.value)
    ok = gpu.Batch([make_instance(20, 3, 2, 4, seed=1), make_instance(30, 3, 40, 40, seed=2)], prm, 4, 4)
    gpu.ffs_batch_step(ok, 1)
    assert (gpu.ffs_batch_best(ok) > 0).all()
