"""Pins of the oracle's GA on the paper's genotype (Section 4.1, genotype
level: a string of n*S machine genes).  The paper names no operators for it;
the library's readings (random initial machines, complement by reflection,
two-point crossover, one-gene machine reassignment) are pinned here by their
defining properties, hand-worked cases with injected draws, and invariants
of whole generations."""
import numpy as np
import pytest

import oracle as orc
from ffs_workloads import make_assign_instance


def test_complement_is_the_binary_not_for_powers_of_two_and_a_valid_involution():
    for M_s in (1, 2, 4, 8, 16):
        for m in range(M_s):
            assert orc.assign_complement(m, M_s) == (~m) & (M_s - 1)
    for M_s in range(1, 12):
        for m in range(M_s):
            c = orc.assign_complement(m, M_s)
            assert 0 <= c < M_s and orc.assign_complement(c, M_s) == m


def test_two_point_crossover_hand_cases():
    p1, p2 = [1, 2, 3, 4, 5], [6, 7, 8, 9, 0]
    assert orc.two_point(p1, p2, 1, 3).tolist() == [6, 2, 3, 4, 0]
    assert orc.two_point(p1, p2, 2, 2).tolist() == [6, 7, 3, 9, 0]
    assert orc.two_point(p1, p2, 0, 4).tolist() == p1
    assert orc.two_point(p2, p1, 0, 0).tolist() == [6, 2, 3, 4, 5]


def test_reassignment_picks_another_machine_uniformly():
    genes = [0, 1, 2, 3]
    # M_s = 1: no other machine
    assert orc.assign_reassign([0], 0, 1, 123456).tolist() == [0]
    counts = {0: 0, 2: 0, 3: 0}
    rng = np.random.default_rng(3)
    for x in rng.integers(0, 2**32, size=3000, dtype=np.uint64):
        g = orc.assign_reassign(genes, 1, 4, int(x))
        assert g[1] != 1 and 0 <= g[1] < 4
        assert g[[0, 2, 3]].tolist() == [0, 2, 3]
        counts[int(g[1])] += 1
    for v in counts.values():
        assert abs(v - 1000) < 120          # about 4 standard deviations of a 1/3 binomial
    # the smallest draw gives machine 0 unless it is the old one, the largest the last machine
    assert orc.assign_reassign([0], 0, 3, 0).tolist() == [1]
    assert orc.assign_reassign([2], 0, 3, 2**32 - 1).tolist() == [1]


def test_initial_rows_and_complementary_pairs():
    n, S, M = 9, 4, [2, 3, 5, 4]
    rows = np.array([orc.assign_init_row(7, 1, c, n, S, M) for c in range(400)])
    assert rows.shape == (400, n * S)
    for i in range(n * S):
        vals = rows[:, i]
        assert vals.min() >= 0 and vals.max() < M[i % S]
        # every machine of the stage appears (400 draws per gene)
        assert len(set(vals.tolist())) == M[i % S]
    # rows of different cells differ
    assert len({r.tobytes() for r in rows}) == 400
    a, b = orc.assign_init_pair(7, 1, 5, n, S, M)
    assert a.tolist() == orc.assign_init_row(7, 1, 10, n, S, M).tolist()
    assert all(b[i] == M[i % S] - 1 - a[i] for i in range(n * S))


def test_cellular_child_with_injected_draws_by_hand():
    """3 x 4 torus, L = 3 jobs x 2 stages = 6 genes.  Cell 5 (row 1, col 1):
    neighbourhood [5, north 1, south 9, west 4, east 6].  Draws pick slots
    (1, 3) -> rows 1 vs 4 and (2, 0) -> rows 9 vs 5; lower objective wins, the
    first drawn on ties."""
    spec = make_assign_instance(3, 2, 3, 3, seed=4)
    inst = orc.AssignInstance(spec.n, spec.S, spec.M, spec.p_u)
    pop = np.zeros((12, 8), dtype=np.int16)
    for c in range(12):
        pop[c, :6] = [(c + i) % 3 for i in range(6)]
    obj = np.array([50] * 12, dtype=np.int64)
    obj[4], obj[9] = 40, 70      # tournament 1: row 4 beats row 1; tournament 2: row 5 beats row 9

    def x_slot(k):     # a draw whose uniform(5) is k
        return int((2**32 * k) // 5 + 1)

    prm = orc.Params(seed=7, cell_pc=1.0, cell_pm=1.0)
    # cuts from draws 5, 6: uniform(6) -> 4 and 1, so l = 1, r = 4
    cut = lambda v: int((2**32 * v) // 6 + 1)
    # mutation: gene uniform(6) = 3 (stage 1, M = 3), reassign draw 0 -> the smallest other machine
    x = [x_slot(1), x_slot(3), x_slot(2), x_slot(0), 0, cut(4), cut(1), 0, cut(3), 0]
    child = orc.assign_cellular_child(inst, prm, 3, 4, 5, x, pop, obj)
    p1, p2 = pop[4, :6], pop[5, :6]          # winners: row 4 (tournament 1), row 5 (tournament 2)
    want = [p2[0], p1[1], p1[2], p1[3], p1[4], p2[5]]
    old = want[3]
    want[3] = 0 if old != 0 else 1
    assert child.tolist() == want
    # no crossover (pc = 0) and no mutation (pm = 0): a copy of the first winner
    prm0 = orc.Params(seed=7, cell_pc=0.0, cell_pm=0.0)
    assert orc.assign_cellular_child(inst, prm0, 3, 4, 5, x, pop, obj).tolist() == p1.tolist()


def _population(inst, spec, N, kind, island=0, seed=7):
    L = spec.n * spec.S
    ld = (L + 7) // 8 * 8
    pop = np.zeros((N, ld), dtype=np.int16)
    if kind == "cellular":
        for c in range(N):
            pop[c, :L] = orc.assign_init_row(seed, island, c, spec.n, spec.S, spec.M)
    else:
        for k in range(N // 2):
            pop[2 * k, :L], pop[2 * k + 1, :L] = orc.assign_init_pair(seed, island, k, spec.n, spec.S, spec.M)
    return pop, orc.eval_population_assign(inst, pop)


@pytest.mark.parametrize("le", [False, True])
def test_cellular_generations_keep_their_invariants(le):
    spec = make_assign_instance(7, 3, 2, 4, seed=2)
    inst = orc.AssignInstance(spec.n, spec.S, spec.M, spec.p_u)
    rows, cols, L = 4, 5, 7 * 3
    pop, obj = _population(inst, spec, rows * cols, "cellular")
    prm = orc.Params(seed=7, cell_pm=0.5, cell_replace_le=le)
    for g in range(1, 9):
        new, nobj, k = orc.assign_cellular_generation(inst, prm, 0, g, rows, cols, pop, obj)
        assert k == rows * cols
        assert np.all(nobj <= obj)                                   # a cell never worsens
        assert np.array_equal(nobj, orc.eval_population_assign(inst, new))
        for c in range(rows * cols):
            nb = [c] + [((c // cols + dr) % rows) * cols + (c % cols + dc) % cols
                        for dr, dc in ((-1, 0), (1, 0), (0, -1), (0, 1))]
            # every gene comes from that position of a neighbourhood row, but for one mutated gene
            own = sum(1 for i in range(L) if new[c, i] not in {pop[r, i] for r in nb})
            assert own <= 1
            assert all(0 <= new[c, i] < spec.M[i % spec.S] for i in range(L))
        pop, obj = new, nobj


@pytest.mark.parametrize("always", [False, True])
def test_pseudo_generations_keep_their_invariants(always):
    spec = make_assign_instance(6, 4, 2, 3, seed=5)
    inst = orc.AssignInstance(spec.n, spec.S, spec.M, spec.p_u)
    N = 24
    pop, obj = _population(inst, spec, N, "pseudo")
    prm = orc.Params(seed=9, pseudo_always=always)
    for g in range(1, 7):
        new, nobj, k = orc.assign_pseudo_generation(inst, prm, 1, g, pop, obj)
        assert np.array_equal(nobj, orc.eval_population_assign(inst, new))
        for q in range(N // 2):
            a, b = pop[2 * q], pop[2 * q + 1]
            if np.array_equal(new[2 * q], a) and np.array_equal(new[2 * q + 1], b):
                continue                                             # no crossover (or parents kept)
            if not always:
                # the pair keeps its two best: never worse than the parents, best first
                assert nobj[2 * q] <= nobj[2 * q + 1]
                kept, before = sorted([nobj[2 * q], nobj[2 * q + 1]]), sorted([obj[2 * q], obj[2 * q + 1]])
                assert kept[0] <= before[0] and kept[1] <= before[1]
            for row in (new[2 * q], new[2 * q + 1]):
                # a child of two-point crossover: each gene from a or b at its position
                assert all(row[i] in (a[i], b[i]) for i in range(spec.n * spec.S))
        pop, obj = new, nobj
