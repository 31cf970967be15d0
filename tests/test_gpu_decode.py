"""GPU decoder parity: ffs_population_eval against the CPU oracle, bit-exact
(integer makespans), over instance shapes, launch shapes, ragged sizes and
edge cases; at the 500 x 20 x 131072 scale on sampled rows."""
import numpy as np
import pytest
import torch

import oracle as orc
from conftest import dev
from ffs_workloads import make_instance, random_population

pytestmark = pytest.mark.gpu

SHAPES = [
    # n, S, m_lo, m_hi, N
    (20, 5, 3, 3, 64),        # 8x8 torus instance shape
    (100, 10, 2, 5, 1000),    # 100 x 10 dual-island shape
    (500, 20, 5, 10, 300),    # 500 x 20 scale shape
    (1, 1, 1, 1, 5),
    (1, 3, 2, 4, 7),
    (7, 1, 3, 3, 33),
    (9, 4, 1, 1, 40),         # permutation flow shop
    (13, 3, 20, 40, 50),      # more machines than jobs (clamped)
    (33, 2, 32, 32, 70),      # 32 machines, the register-heap maximum
    (40, 6, 1, 32, 100),
    (257, 7, 2, 9, 130),      # ragged n
    (1000, 5, 2, 7, 65),
]


def _pair(spec, ffs):
    return orc.Instance(spec.n, spec.S, spec.M, spec.p), ffs.Instance(spec.n, spec.S, spec.M, spec.p)


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[0]}x{s[1]}m{s[2]}-{s[3]}N{s[4]}" for s in SHAPES])
def test_eval_matches_oracle(gpu, shape):
    n, S, mlo, mhi, N = shape
    spec = make_instance(n, S, mlo, mhi, seed=n * 31 + S)
    o, g = _pair(spec, gpu)
    pop = random_population(n, N, seed=N + n)
    want = orc.eval_population(o, pop)
    d = dev(pop)
    out = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    shapes = [(0, 0)]
    for chunk in (8, 16, 32, 48, 64, 96, 104, 112, 128):
        if chunk < n:
            shapes.append((chunk, 0))
    for threads in (32, 96, 128, 256, 512):
        shapes.append((0, threads))
    if n > 8:
        shapes.append((8, 64))
    for chunk, threads in ((8, 128), (16, 256), (32, 512), (8, 512), (96, 384), (112, 448), (48, 320)):
        if chunk < n:
            shapes.append((chunk, threads))
    ran = 0
    shapes = [(c, t, v) for (c, t) in shapes for v in (1, 2, 3, 4)]
    for chunk, threads, variant in shapes:
        out.fill_(-7)
        try:
            gpu.ffs_population_eval_tuned(g, d, N, pop.shape[1], out, chunk, threads, variant)
        except gpu.FFSError as e:
            # a forced shape may not fit shared memory; the library's own choice always does
            assert e.status == gpu.FFS_EUNSUPPORTED and (chunk, threads) != (0, 0), (chunk, threads, variant)
            continue
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.int64)
        assert np.array_equal(got, want), (chunk, threads, variant, np.flatnonzero(got != want)[:5])
        ran += 1
    assert ran >= len(shapes) // 2


def test_eval_full_scale_sampled(gpu):
    """500 jobs x 20 stages, 131072 rows (the 4 x 128^2 + 4 x 16384 scale)."""
    spec = make_instance(500, 20, 5, 10, seed=1)
    o, g = _pair(spec, gpu)
    N = 131072
    pop = random_population(500, N, seed=3)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    gpu.ffs_population_eval(g, dev(pop), N, pop.shape[1], out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    rng = np.random.default_rng(5)
    idx = np.concatenate([[0, 1, N - 1], rng.choice(N, 200, replace=False)])
    want = orc.eval_population(o, pop[idx])
    assert np.array_equal(got[idx].astype(np.int64), want)
    lb = orc.lower_bound(o)
    assert got.min() >= lb and got.max() <= int(spec.p.sum())


def test_eval_padding_invalid_genes_and_empty(gpu):
    spec = make_instance(10, 3, 2, 3, seed=9)
    o, g = _pair(spec, gpu)
    ld = 24
    pop = random_population(10, 20, ld=ld, seed=1)
    pop[:, 10:] = 12345          # padding is never read as genes
    pop[3, 4] = 10               # out of range -> -1
    pop[5, 0] = -2               # negative -> -1
    out = torch.zeros(20, dtype=torch.int32, device="cuda")
    gpu.ffs_population_eval(g, dev(pop), 20, ld, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[3] == -1 and got[5] == -1
    assert np.array_equal(got.astype(np.int64), orc.eval_population(o, pop))   # the oracle also gives -1
    gpu.ffs_population_eval(g, dev(pop), 0, ld, out)   # N = 0 is a no-op
    with pytest.raises(gpu.FFSError):
        gpu.ffs_population_eval(g, dev(pop), 20, 12, out)   # ld not a multiple of 8
    with pytest.raises(gpu.FFSError):
        gpu.ffs_population_eval_tuned(g, dev(pop), 20, ld, out, 12, 0, 0)  # chunk not a multiple of 8


def test_eval_golden_examples(gpu, golden):
    for ex in golden("gantt_examples.json")["examples"]:
        g = gpu.Instance(ex["n"], ex["S"], ex["M"], ex["p"])
        pop = np.zeros((1, 8), dtype=np.int16)
        pop[0, :ex["n"]] = ex["perm"]
        out = torch.zeros(1, dtype=torch.int32, device="cuda")
        gpu.ffs_population_eval(g, dev(pop), 1, 8, out)
        torch.cuda.synchronize()
        assert int(out.item()) == ex["cmax"], ex["name"]


def test_eval_host_buffers(gpu):
    spec = make_instance(100, 10, 2, 5, seed=4)
    o, g = _pair(spec, gpu)
    pop = random_population(100, 500, seed=8)
    out = np.zeros(500, dtype=np.int32)
    gpu.ffs_population_eval_host(g, pop, 500, pop.shape[1], out)
    assert np.array_equal(out.astype(np.int64), orc.eval_population(o, pop))


@pytest.mark.parametrize("variant", [3, 4])
def test_saved_heaps_in_tensor_memory(gpu, variant):
    """The 500 x 20 instance at chunk 32: the TMEM variants keep a prefix of the
    saved heaps in tensor memory (more resident threads), and decode exactly;
    so does every block size that allows it."""
    spec = make_instance(500, 20, 5, 10, seed=1)
    o, g = _pair(spec, gpu)
    plain = gpu.ffs_decode_plan(g, 0, 32, 0, variant - 2)
    plan = gpu.ffs_decode_plan(g, 0, 32, 0, variant)
    assert plain["tmem_cols"] == 0 and plan["tmem_cols"] in (128, 256, 512)
    assert plan["threads"] * plan["blocks_per_sm"] > plain["threads"] * plain["blocks_per_sm"]
    N = 700
    pop = random_population(500, N, seed=21)
    want = orc.eval_population(o, pop)
    d = dev(pop)
    out = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    for threads in (96, 128, 256, 320, 448, 512):
        p = gpu.ffs_decode_plan(g, 0, 32, threads, variant)
        assert p["tmem_cols"] > 0, p
        out.fill_(-7)
        gpu.ffs_population_eval_tuned(g, d, N, pop.shape[1], out, 32, threads, variant)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.int64)
        assert np.array_equal(got, want), (threads, np.flatnonzero(got != want)[:5])
