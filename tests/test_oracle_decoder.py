"""Pins of the oracle's schedule decoder against facts fixed outside it.

Decoder: stage-wise list scheduling of a job order on a flexible flow shop
(problem statement: arXiv:1903.10722, Section 3).  Pins: hand-worked Gantt
charts, the permutation-flow-shop recurrence, Johnson's two-machine rule,
Graham's list-scheduling bounds, closed forms, schedule invariants and the
machine tie-rule invariance of the makespan.
"""
import heapq
import itertools

import numpy as np
import pytest

import oracle as orc


def _inst(n, S, M, p):
    return orc.Instance(n, S, np.array(M, dtype=np.int32), np.array(p, dtype=np.int32))


def _rand_inst(rng, n, S, mlo, mhi, plo=1, phi=20):
    return _inst(n, S, rng.integers(mlo, mhi + 1, size=S), rng.integers(plo, phi + 1, size=(n, S)))


def test_golden_gantt_charts(golden):
    g = golden("gantt_examples.json")
    for ex in g["examples"]:
        inst = _inst(ex["n"], ex["S"], ex["M"], ex["p"])
        cmax, gantt = orc.decode(inst, ex["perm"], gantt=True)
        assert cmax == ex["cmax"], ex["name"]
        assert gantt.tolist() == ex["gantt"], ex["name"]
        assert orc.lower_bound(inst) == ex["lower_bound"], ex["name"]
        if "all_orders" in ex:
            for k, v in ex["all_orders"].items():
                assert orc.decode(inst, [int(t) for t in k.split(",")]) == v
        if "optimal_order" in ex:
            assert orc.decode(inst, ex["optimal_order"]) == ex["optimal_order_cmax"]
        if "optimum" in ex:
            best, worst, _ = orc.bruteforce(inst)
            assert best == ex["optimum"]
            if "worst" in ex:
                assert worst == ex["worst"]


def _pfs_makespan(p, perm):
    """Permutation flow shop recurrence C(k,s) = max(C(k-1,s), C(k,s-1)) + p."""
    n, S = p.shape
    C = np.zeros((n + 1, S + 1), dtype=np.int64)
    for k in range(1, n + 1):
        j = perm[k - 1]
        for s in range(1, S + 1):
            C[k, s] = max(C[k - 1, s], C[k, s - 1]) + p[j, s - 1]
    return int(C[n, S])


def test_single_machine_stages_match_flow_shop_recurrence():
    rng = np.random.default_rng(11)
    for _ in range(60):
        n, S = int(rng.integers(1, 30)), int(rng.integers(1, 8))
        inst = _inst(n, S, [1] * S, rng.integers(1, 50, size=(n, S)))
        perm = rng.permutation(n)
        assert orc.decode(inst, perm) == _pfs_makespan(inst.p, perm)


def _johnson(p):
    """Johnson (1954): p1 <= p2 first by increasing p1, then the rest by decreasing p2."""
    first = sorted([j for j in range(len(p)) if p[j][0] <= p[j][1]], key=lambda j: (p[j][0], j))
    last = sorted([j for j in range(len(p)) if p[j][0] > p[j][1]], key=lambda j: (-p[j][1], j))
    return first + last


def test_two_machine_flow_shop_optimum_is_johnson():
    rng = np.random.default_rng(12)
    for _ in range(25):
        n = int(rng.integers(2, 8))
        inst = _inst(n, 2, [1, 1], rng.integers(1, 30, size=(n, 2)))
        best, _, _ = orc.bruteforce(inst)
        assert best == _pfs_makespan(inst.p, _johnson(inst.p.tolist()))


def test_single_stage_graham_bounds():
    rng = np.random.default_rng(13)
    for _ in range(25):
        n, m = int(rng.integers(2, 8)), int(rng.integers(2, 4))
        inst = _inst(n, 1, [m], rng.integers(1, 40, size=(n, 1)))
        opt, _, _ = orc.bruteforce(inst)
        p = inst.p[:, 0]
        assert opt >= max(int(p.max()), -(-int(p.sum()) // m))
        for _ in range(5):
            c = orc.decode(inst, rng.permutation(n))
            # Graham 1966: list scheduling is within (2 - 1/m) of the optimum,
            # and within sum/m + (1 - 1/m) max in absolute terms.
            assert c * m <= (2 * m - 1) * opt
            assert c * m <= int(p.sum()) + (m - 1) * int(p.max())


def test_enough_machines_gives_longest_job():
    rng = np.random.default_rng(14)
    for _ in range(30):
        n, S = int(rng.integers(1, 12)), int(rng.integers(1, 6))
        inst = _inst(n, S, rng.integers(n, n + 3, size=S), rng.integers(1, 60, size=(n, S)))
        assert orc.decode(inst, rng.permutation(n)) == int(inst.p.sum(axis=1).max())


def test_equal_times_single_machines_closed_form():
    for n, S, c in [(1, 1, 5), (7, 3, 4), (20, 5, 1), (13, 9, 17)]:
        inst = _inst(n, S, [1] * S, np.full((n, S), c))
        assert orc.decode(inst, np.arange(n)[::-1]) == c * (n + S - 1)


def _check_schedule(inst, gantt, cmax):
    n, S = inst.n, inst.S
    seen = set()
    end_of = {}
    for s, j, m, st, en in gantt.tolist():
        assert (s, j) not in seen
        seen.add((s, j))
        assert 0 <= m < inst.M[s]
        assert en - st == inst.p[j, s]
        assert st >= (end_of[(s - 1, j)] if s > 0 else 0)
        end_of[(s, j)] = en
    assert len(seen) == n * S
    for s in range(S):
        for m in range(int(inst.M[s])):
            iv = sorted((st, en) for ss, j, mm, st, en in gantt.tolist() if ss == s and mm == m)
            for a, b in zip(iv, iv[1:]):
                assert a[1] <= b[0], "machine overlap"
    assert cmax == max(end_of[(S - 1, j)] for j in range(n))
    assert orc.lower_bound(inst) <= cmax <= int(inst.p.sum())


def test_schedule_invariants_random():
    rng = np.random.default_rng(15)
    for _ in range(80):
        n, S = int(rng.integers(1, 40)), int(rng.integers(1, 8))
        inst = _rand_inst(rng, n, S, 1, 6)
        cmax, gantt = orc.decode(inst, rng.permutation(n), gantt=True)
        _check_schedule(inst, gantt, cmax)


def _decode_alt_machine_rule(inst, perm):
    """Same list schedule, but a job takes the lowest-index machine among those
    already free at its release (else the earliest free).  The start time of
    every operation is unchanged, so the makespan must be too."""
    n, S = inst.n, inst.S
    prev = [0] * n
    order = list(perm)
    for s in range(S):
        if s > 0:
            order = sorted(range(n), key=lambda j: (prev[j], j))
        free = [0] * int(inst.M[s])
        cur = [0] * n
        for j in order:
            ready = prev[j] if s > 0 else 0
            idle = [m for m in range(len(free)) if free[m] <= ready]
            m = idle[0] if idle else min(range(len(free)), key=lambda q: (free[q], q))
            cur[j] = max(free[m], ready) + int(inst.p[j, s])
            free[m] = cur[j]
        prev = cur
    return max(prev)


def test_machine_tie_rule_does_not_change_makespan():
    rng = np.random.default_rng(16)
    for _ in range(60):
        n, S = int(rng.integers(1, 30)), int(rng.integers(1, 6))
        inst = _rand_inst(rng, n, S, 1, 5, 1, 6)
        perm = rng.permutation(n)
        assert orc.decode(inst, perm) == _decode_alt_machine_rule(inst, perm)


def _graham_single_stage(p, m, perm):
    h = [0] * m
    for j in perm:
        t = heapq.heappop(h)
        heapq.heappush(h, t + int(p[j]))
    return max(h)


def test_single_stage_is_graham_list_scheduling():
    rng = np.random.default_rng(17)
    for _ in range(40):
        n, m = int(rng.integers(1, 40)), int(rng.integers(1, 9))
        inst = _inst(n, 1, [m], rng.integers(1, 99, size=(n, 1)))
        perm = rng.permutation(n)
        assert orc.decode(inst, perm) == _graham_single_stage(inst.p[:, 0], m, perm)


def test_population_eval_matches_rows():
    rng = np.random.default_rng(18)
    inst = _rand_inst(rng, 9, 3, 1, 3)
    pop = np.zeros((6, 16), dtype=np.int16)
    for i in range(6):
        pop[i, :9] = rng.permutation(9)
    out = orc.eval_population(inst, pop)
    assert out.tolist() == [orc.decode(inst, pop[i, :9]) for i in range(6)]


def test_bruteforce_covers_every_order():
    inst = _inst(4, 2, [2, 1], [[3, 1], [1, 4], [2, 2], [4, 3]])
    vals = [orc.decode(inst, list(q)) for q in itertools.permutations(range(4))]
    best, worst, bp = orc.bruteforce(inst)
    assert best == min(vals) and worst == max(vals)
    assert orc.decode(inst, bp) == best
