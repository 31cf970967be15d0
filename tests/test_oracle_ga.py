"""Invariants of the oracle's GA generations (arXiv:1903.10722, Sections 4.1-4.2).

The paper prints no GA trajectory, so whole runs are "parity unpinned"; these
tests pin what the method fixes: permutations stay permutations, cellular
replacement never worsens a cell, a pseudo pair keeps its two best, operator
wiring with forced rates, and the optimum from brute force is a floor.
"""
import numpy as np

import oracle as orc
from ffs_workloads import make_instance


def _inst(spec):
    return orc.Instance(spec.n, spec.S, spec.M, spec.p)


def _is_perm_rows(pop, n):
    return all(sorted(r[:n].tolist()) == list(range(n)) for r in pop)


def test_dual_island_invariants():
    inst = _inst(make_instance(12, 4, 1, 3, seed=5))
    ga = orc.IslandGA(inst, orc.Params(seed=3), 1, 4, 4, 1, 16)
    assert ga.kinds == ["cellular", "pseudo"]
    for _ in range(12):
        before = [m.copy() for m in ga.mss]
        prev_pop = [p.copy() for p in ga.pops]
        ga.step()
        for i, k in enumerate(ga.kinds):
            assert _is_perm_rows(ga.pops[i], inst.n)
            assert ga.mss[i].tolist() == orc.eval_population(inst, ga.pops[i]).tolist()
            if k == "cellular":
                assert np.all(ga.mss[i] <= before[i])
            else:
                b2 = before[i].reshape(-1, 2)
                a2 = ga.mss[i].reshape(-1, 2)
                assert np.all(a2.min(axis=1) <= b2.min(axis=1))
                changed = np.any(ga.pops[i].reshape(-1, 2, ga.ld) != prev_pop[i].reshape(-1, 2, ga.ld), axis=(1, 2))
                assert np.all(a2[changed, 0] <= a2[changed, 1])
    ga.migrate_ring(25, 100)
    for i in range(2):
        assert ga.mss[i].tolist() == orc.eval_population(inst, ga.pops[i]).tolist()


def test_cellular_selection_only_copies_neighbours():
    inst = _inst(make_instance(10, 3, 2, 3, seed=6))
    rows, cols = 4, 5
    pop = np.zeros((rows * cols, 16), dtype=np.int16)
    for c in range(rows * cols):
        pop[c, :10] = orc.init_chromosome(1, 0, c, 10)
    ms = orc.eval_population(inst, pop)
    prm = orc.Params(seed=9, cell_pc=0.0, cell_pm=0.0)
    new, new_ms, dec = orc.cellular_generation(inst, prm, 0, 1, rows, cols, pop, ms)
    assert dec == rows * cols
    for c in range(rows * cols):
        nb = orc.neighbours(rows, cols, c)
        assert any(new[c, :10].tolist() == pop[q, :10].tolist() for q in nb)
        assert new_ms[c] == min(ms[c], new_ms[c])
        assert new_ms[c] >= min(ms[q] for q in nb)


def test_pseudo_no_crossover_is_identity_and_always_variant():
    inst = _inst(make_instance(9, 3, 1, 3, seed=7))
    pop = np.zeros((8, 16), dtype=np.int16)
    for q in range(4):
        a, b = orc.init_pseudo_pair(2, 1, q, 9)
        pop[2 * q, :9], pop[2 * q + 1, :9] = a, b
    ms = orc.eval_population(inst, pop)
    same, same_ms, dec = orc.pseudo_generation(inst, orc.Params(pseudo_pc=0.0), 1, 1, pop, ms)
    assert dec == 0 and np.array_equal(same, pop) and np.array_equal(same_ms, ms)
    prm = orc.Params(seed=4, pseudo_pc=1.0, pseudo_always=True)
    new, new_ms, dec = orc.pseudo_generation(inst, prm, 1, 3, pop, ms)
    assert dec == 8
    for q in range(4):
        u = orc.uniform(orc.draw(4, orc.PURPOSE_PSEUDO, 1, 3, q, 1), 9)
        v = orc.uniform(orc.draw(4, orc.PURPOSE_PSEUDO, 1, 3, q, 2), 9)
        l, r = min(u, v), max(u, v)
        assert new[2 * q, :9].tolist() == orc.order_crossover(pop[2 * q, :9], pop[2 * q + 1, :9], l, r).tolist()
        assert new[2 * q + 1, :9].tolist() == orc.order_crossover(pop[2 * q + 1, :9], pop[2 * q, :9], l, r).tolist()


def test_ga_never_beats_bruteforce_optimum():
    spec = make_instance(7, 3, 1, 2, seed=8)
    inst = _inst(spec)
    opt, worst, _ = orc.bruteforce(inst)
    ga = orc.IslandGA(inst, orc.Params(seed=7), 1, 4, 4, 1, 8)
    for g in range(30):
        ga.step()
        if g % 5 == 4:
            ga.migrate_ring()
        for m in ga.mss:
            assert opt <= m.min() and m.max() <= worst
    assert ga.best() >= opt
