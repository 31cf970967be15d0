"""Pins of the oracle's genetic operators (arXiv:1903.10722, Sections 4.1-4.2)."""
import numpy as np
import pytest

import oracle as orc


def test_order_crossover_golden(golden):
    for case in golden("operators.json")["order_crossover"]:
        got = orc.order_crossover(case["p1"], case["p2"], case["l"], case["r"])
        assert got.tolist() == case["child"]


def test_order_crossover_properties():
    rng = np.random.default_rng(21)
    for _ in range(300):
        n = int(rng.integers(1, 60))
        p1, p2 = rng.permutation(n), rng.permutation(n)
        a, b = sorted(rng.integers(0, n, size=2).tolist())
        child = orc.order_crossover(p1, p2, a, b).tolist()
        assert sorted(child) == list(range(n))
        assert child[a:b + 1] == p1[a:b + 1].tolist()
        seg = set(p1[a:b + 1].tolist())
        rest_positions = [(b + 1 + t) % n for t in range(n - (b - a + 1))]
        rest_p2 = [g for g in np.roll(p2, -(b + 1)).tolist() if g not in seg]
        assert [child[q] for q in rest_positions] == rest_p2


def test_neighbours_golden(golden):
    g = golden("operators.json")["neighbours_3x4"]
    for c, nb in g["cells"].items():
        assert orc.neighbours(g["rows"], g["cols"], int(c)) == nb


def _slot(k):
    """A draw whose uniform(., 5) is slot k."""
    return -(-k * 2**32 // 5)


def test_cellular_child_tournament_and_operators():
    inst = orc.Instance(5, 1, np.array([1], dtype=np.int32), np.ones((5, 1), dtype=np.int32))
    rows, cols = 3, 3
    pop = np.zeros((9, 8), dtype=np.int16)
    rng = np.random.default_rng(3)
    for c in range(9):
        pop[c, :5] = rng.permutation(5)
    ms = np.array([50, 40, 60, 40, 30, 70, 80, 40, 90], dtype=np.int64)
    # cell 4 (centre): slots 0..4 = [4, 1, 7, 3, 5]
    prm = orc.Params(cell_pc=1.0, cell_pm=0.0)
    # tournament 1: slots N (cell 1, ms 40) vs S (cell 7, ms 40) -> tie -> first drawn (1)
    # tournament 2: slots W (cell 3, ms 40) vs E (cell 5, ms 70) -> cell 3
    # crossover always (pc = 1), cuts 0 and 3; mutation never (x[7] = max)
    x = [_slot(1), _slot(2), _slot(3), _slot(4), 0, 0, _slot(3), 2**32 - 1, 0, 0]
    child, parents = orc.cellular_child(inst, prm, rows, cols, 4, x, pop, ms)
    assert parents == [1, 3]
    assert child.tolist() == orc.order_crossover(pop[1, :5], pop[3, :5], 0, 3).tolist()
    # no crossover (pc = 0): child copies the first parent; a forced swap of positions 0 and 4
    prm2 = orc.Params(cell_pc=0.0, cell_pm=1.0)
    x2 = [_slot(0), _slot(0), _slot(0), _slot(0), 0, 0, 0, 0, 0, 2**32 - 1]
    child2, parents2 = orc.cellular_child(inst, prm2, rows, cols, 4, x2, pop, ms)
    assert parents2 == [4, 4]
    want = pop[4, :5].copy()
    want[0], want[4] = want[4], want[0]
    assert child2.tolist() == want.tolist()


def test_family_best2_golden(golden):
    for case in golden("operators.json")["family_best2"]:
        assert orc.family_best2(case["ms"]) == case["pick"]
