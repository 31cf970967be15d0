"""The GA on the paper's genotype (n*S machine-assignment strings on
unrelated machines) on the GPU against the CPU oracle, bit-exact: initial
rows of both kinds, cellular and pseudo generations (both replacement
rules), the paper's objective with release and due times, and a full-size
500 x 20 string."""
import numpy as np
import pytest
import torch

import oracle as orc
from ffs_workloads import make_assign_instance

pytestmark = pytest.mark.gpu


def _pair(spec, gpu, release=None, due=None, wt=0):
    return (orc.AssignInstance(spec.n, spec.S, spec.M, spec.p_u, release, due, wt),
            gpu.AssignInstance(spec.n, spec.S, spec.M, spec.p_u, release, due, wt))


def _init(gpu, g, spec, N, kind, island, seed=7):
    L = spec.n * spec.S
    ld = (L + 7) // 8 * 8
    pop = torch.full((N, ld), -1, dtype=torch.int16, device="cuda")
    gpu.ffs_assign_population_init(g, seed, island, kind, N, ld, pop)
    torch.cuda.synchronize()
    want = np.zeros((N, ld), dtype=np.int16)
    for r in range(N if kind == 0 else N // 2):
        if kind == 0:
            want[r, :L] = orc.assign_init_row(seed, island, r, spec.n, spec.S, spec.M)
        else:
            want[2 * r, :L], want[2 * r + 1, :L] = orc.assign_init_pair(seed, island, r, spec.n, spec.S, spec.M)
    assert np.array_equal(pop.cpu().numpy(), want)        # padding genes included (0)
    return pop, want, ld


def _params(gpu, le=False, always=False, pm=0.05):
    prm = gpu.ffs_params_default()
    prm.cell_replace_le, prm.pseudo_always = int(le), int(always)
    prm.cell_pm = gpu.threshold(pm)
    return prm, orc.Params(seed=7, cell_pm=pm, cell_replace_le=le, pseudo_always=always)


CELL_SHAPES = [
    # n, S, m_lo, m_hi, rows, cols
    (7, 3, 1, 4, 4, 5),
    (20, 5, 1, 1, 3, 3),      # one machine per stage: crossover only, reassignment is a no-op
    (33, 4, 2, 9, 6, 6),
    (40, 3, 32, 32, 4, 4),    # 32 machines
    (100, 10, 2, 5, 8, 8),
]


@pytest.mark.parametrize("shape", CELL_SHAPES, ids=[f"{s[0]}x{s[1]}m{s[2]}-{s[3]}t{s[4]}x{s[5]}" for s in CELL_SHAPES])
@pytest.mark.parametrize("le", [False, True])
def test_assign_cellular_generations_match_oracle(gpu, shape, le):
    n, S, mlo, mhi, rows, cols = shape
    spec = make_assign_instance(n, S, mlo, mhi, seed=n + S)
    o, g = _pair(spec, gpu)
    N = rows * cols
    pop, opop, ld = _init(gpu, g, spec, N, 0, island=2)
    obj = torch.empty(N, dtype=torch.int32, device="cuda")
    gpu.ffs_assign_eval(g, pop, N, ld, obj)
    oobj = orc.eval_population_assign(o, opop)
    torch.cuda.synchronize()
    assert np.array_equal(obj.cpu().numpy().astype(np.int64), oobj)
    prm, oprm = _params(gpu, le=le, pm=0.4)
    scratch = torch.empty(gpu.ffs_assign_step_scratch_bytes(N, ld), dtype=torch.uint8, device="cuda")
    nxt, nobj = torch.empty_like(pop), torch.empty_like(obj)
    for gen in range(1, 11):
        gpu.ffs_assign_cellular_step(g, prm, 2, gen, rows, cols, ld, pop, obj, nxt, nobj, scratch)
        opop, oobj, _ = orc.assign_cellular_generation(o, oprm, 2, gen, rows, cols, opop, oobj)
        torch.cuda.synchronize()
        assert np.array_equal(nxt.cpu().numpy()[:, :n * S], opop[:, :n * S]), gen
        assert np.array_equal(nobj.cpu().numpy().astype(np.int64), oobj), gen
        pop, nxt, obj, nobj = nxt, pop, nobj, obj


@pytest.mark.parametrize("always", [False, True])
def test_assign_pseudo_generations_match_oracle(gpu, always):
    spec = make_assign_instance(30, 6, 2, 7, seed=9)
    o, g = _pair(spec, gpu)
    N = 48
    pop, opop, ld = _init(gpu, g, spec, N, 1, island=1)
    obj = torch.empty(N, dtype=torch.int32, device="cuda")
    gpu.ffs_assign_eval(g, pop, N, ld, obj)
    oobj = orc.eval_population_assign(o, opop)
    prm, oprm = _params(gpu, always=always)
    scratch = torch.empty(gpu.ffs_assign_step_scratch_bytes(N, ld), dtype=torch.uint8, device="cuda")
    nxt, nobj = torch.empty_like(pop), torch.empty_like(obj)
    for gen in range(1, 9):
        gpu.ffs_assign_pseudo_step(g, prm, 1, gen, N, ld, pop, obj, nxt, nobj, scratch)
        opop, oobj, _ = orc.assign_pseudo_generation(o, oprm, 1, gen, opop, oobj)
        torch.cuda.synchronize()
        assert np.array_equal(nxt.cpu().numpy()[:, :spec.n * spec.S], opop[:, :spec.n * spec.S]), gen
        assert np.array_equal(nobj.cpu().numpy().astype(np.int64), oobj), gen
        pop, nxt, obj, nobj = nxt, pop, nobj, obj


def test_assign_ga_with_the_papers_objective(gpu):
    """300 jobs x 4 stages x 2 unrelated machines, P ~ U[1,5] (the paper's
    Section 5 shape), release and due times, WT = 100: a cellular and a pseudo
    island, 4 generations each."""
    spec = make_assign_instance(300, 4, 2, 2, p_lo=1, p_hi=5, seed=3)
    rng = np.random.default_rng(4)
    rel = rng.integers(0, 400, spec.n).astype(np.int32)
    due = (rel + rng.integers(5, 60, spec.n)).astype(np.int32)
    o, g = _pair(spec, gpu, rel, due, 100)
    prm, oprm = _params(gpu)
    for kind, N, island in ((0, 64, 0), (1, 64, 1)):
        pop, opop, ld = _init(gpu, g, spec, N, kind, island)
        obj = torch.empty(N, dtype=torch.int32, device="cuda")
        gpu.ffs_assign_eval(g, pop, N, ld, obj)
        oobj = orc.eval_population_assign(o, opop)
        scratch = torch.empty(gpu.ffs_assign_step_scratch_bytes(N, ld), dtype=torch.uint8, device="cuda")
        nxt, nobj = torch.empty_like(pop), torch.empty_like(obj)
        for gen in range(1, 5):
            if kind == 0:
                gpu.ffs_assign_cellular_step(g, prm, island, gen, 8, 8, ld, pop, obj, nxt, nobj, scratch)
                opop, oobj, _ = orc.assign_cellular_generation(o, oprm, island, gen, 8, 8, opop, oobj)
            else:
                gpu.ffs_assign_pseudo_step(g, prm, island, gen, N, ld, pop, obj, nxt, nobj, scratch)
                opop, oobj, _ = orc.assign_pseudo_generation(o, oprm, island, gen, opop, oobj)
            torch.cuda.synchronize()
            assert np.array_equal(nobj.cpu().numpy().astype(np.int64), oobj), (kind, gen)
            assert np.array_equal(nxt.cpu().numpy()[:, :spec.n * spec.S], opop[:, :spec.n * spec.S]), (kind, gen)
            pop, nxt, obj, nobj = nxt, pop, nobj, obj


def test_assign_ga_full_size_string(gpu):
    """500 x 20 genes per string (10000), M_s in [5, 10]: two cellular
    generations of a 8 x 8 torus."""
    spec = make_assign_instance(500, 20, 5, 10, seed=1)
    o, g = _pair(spec, gpu)
    rows = cols = 8
    N = rows * cols
    pop, opop, ld = _init(gpu, g, spec, N, 0, island=0)
    obj = torch.empty(N, dtype=torch.int32, device="cuda")
    gpu.ffs_assign_eval(g, pop, N, ld, obj)
    oobj = orc.eval_population_assign(o, opop)
    prm, oprm = _params(gpu, pm=0.5)
    scratch = torch.empty(gpu.ffs_assign_step_scratch_bytes(N, ld), dtype=torch.uint8, device="cuda")
    nxt, nobj = torch.empty_like(pop), torch.empty_like(obj)
    for gen in (1, 2):
        gpu.ffs_assign_cellular_step(g, prm, 0, gen, rows, cols, ld, pop, obj, nxt, nobj, scratch)
        opop, oobj, _ = orc.assign_cellular_generation(o, oprm, 0, gen, rows, cols, opop, oobj)
        torch.cuda.synchronize()
        assert np.array_equal(nobj.cpu().numpy().astype(np.int64), oobj), gen
        assert np.array_equal(nxt.cpu().numpy()[:, :spec.n * spec.S], opop[:, :spec.n * spec.S]), gen
        pop, nxt, obj, nobj = nxt, pop, nobj, obj


def test_assign_ga_argument_errors(gpu):
    spec = make_assign_instance(5, 2, 2, 3, seed=1)
    _, g = _pair(spec, gpu)
    ld = 16
    pop = torch.zeros((4, ld), dtype=torch.int16, device="cuda")
    obj = torch.zeros(4, dtype=torch.int32, device="cuda")
    scratch = torch.empty(gpu.ffs_assign_step_scratch_bytes(4, ld), dtype=torch.uint8, device="cuda")
    prm = gpu.ffs_params_default()
    with pytest.raises(gpu.FFSError) as e:
        gpu.ffs_assign_pseudo_step(g, prm, 0, 1, 3, ld, pop, obj, pop.clone(), obj.clone(), scratch)
    assert e.value.status == gpu.FFS_EINVAL
    with pytest.raises(gpu.FFSError):
        gpu.ffs_assign_cellular_step(g, prm, 0, 1, 2, 2, ld, pop, obj, pop, obj, scratch)   # in place
    with pytest.raises(gpu.FFSError):
        gpu.ffs_assign_population_init(g, 7, 0, 1, 3, ld, pop)                               # odd pair count
    assert gpu.ffs_assign_step_scratch_bytes(-1, 8) == -1
