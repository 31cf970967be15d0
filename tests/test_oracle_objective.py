"""Pins of the oracle's objective (arXiv:1903.10722, Section 3 and Table 1):
release times at the first stage, due times, WT * total tardiness + C_max.

Pinned against hand-worked schedules (tests/golden/objective_examples.json),
the makespan decoder it must reduce to (no releases, due times never missed),
the definition recomputed from the schedule's own records, and invariants a
wrong sign or dropped term would break."""
import json
import os

import numpy as np
import pytest

import oracle as orc
from ffs_workloads import make_instance, make_paper_instance, random_population

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "objective_examples.json")


def _inst(ex):
    return orc.Instance(ex["n"], ex["S"], np.array(ex["M"]), np.array(ex["p"]),
                        release=None if ex["release"] is None else np.array(ex["release"]),
                        due=np.array(ex["due"]), wt=ex["wt"])


def test_hand_worked_objectives():
    data = json.load(open(GOLDEN))
    for ex in data["examples"]:
        inst = _inst(ex)
        for case in ex["cases"]:
            v, g = orc.decode(inst, case["order"], gantt=True)
            assert v == case["objective"], (ex["name"], case["order"])
            if "gantt" in case:
                assert g.tolist() == case["gantt"]
        if "optimum" in ex:
            assert orc.bruteforce(inst)[0] == ex["optimum"]


def _objective_from_gantt(inst, g):
    """WT * sum_j max(0, C_j - D_j) + C_max from the schedule records."""
    last = g[g[:, 0] == inst.S - 1]
    C = np.zeros(inst.n, dtype=np.int64)
    C[last[:, 1]] = last[:, 4]
    T = np.maximum(0, C - inst.due.astype(np.int64)) if inst.due is not None else np.zeros(inst.n, np.int64)
    return int(inst.wt * T.sum() + C.max())


@pytest.mark.parametrize("seed", range(6))
def test_objective_is_the_definition_on_the_schedule(seed):
    spec = make_paper_instance(40, 4, 2, seed=seed)
    inst = orc.Instance(spec.n, spec.S, spec.M, spec.p, release=spec.release, due=spec.due, wt=spec.wt)
    for row in random_population(spec.n, 5, seed=seed)[:, :spec.n]:
        v, g = orc.decode(inst, row, gantt=True)
        assert v == _objective_from_gantt(inst, g)
        first = g[g[:, 0] == 0]
        # no job starts its first operation before its release time
        assert np.all(first[:, 3] >= inst.release[first[:, 1]])


def test_reduces_to_the_makespan():
    spec = make_instance(30, 5, 2, 4, seed=3)
    plain = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    big = np.full(spec.n, int(spec.p.sum()), dtype=np.int32)     # never missed
    with_due = orc.Instance(spec.n, spec.S, spec.M, spec.p, due=big, wt=100)
    zero_rel = orc.Instance(spec.n, spec.S, spec.M, spec.p, release=np.zeros(spec.n, np.int32), due=big, wt=7)
    pop = random_population(spec.n, 20, seed=4)
    want = orc.eval_population(plain, pop)
    assert np.array_equal(orc.eval_population(with_due, pop), want)
    assert np.array_equal(orc.eval_population(zero_rel, pop), want)


def test_weight_and_due_time_monotonicity():
    spec = make_paper_instance(25, 3, 2, seed=9)
    rows = random_population(spec.n, 8, seed=2)
    base = orc.Instance(spec.n, spec.S, spec.M, spec.p, release=spec.release, due=spec.due, wt=100)
    later = orc.Instance(spec.n, spec.S, spec.M, spec.p, release=spec.release, due=spec.due + 5, wt=100)
    nowt = orc.Instance(spec.n, spec.S, spec.M, spec.p, release=spec.release, due=spec.due, wt=0)
    a, b, c = (orc.eval_population(i, rows) for i in (base, later, nowt))
    assert np.all(b <= a) and np.all(c <= a)
    # WT = 0 leaves C_max, which the tardiness-free instance with the same releases gives too
    cmax = orc.Instance(spec.n, spec.S, spec.M, spec.p, release=spec.release)
    assert np.array_equal(c, orc.eval_population(cmax, rows))
    # later releases can only delay: C_max never drops
    delayed = orc.Instance(spec.n, spec.S, spec.M, spec.p, release=spec.release + 3)
    assert np.all(orc.eval_population(delayed, rows) >= orc.eval_population(cmax, rows))


def test_paper_instance_generator():
    """Table 1: p ~ U[1, 5]; R_j ~ U[0, Pbar]; D_j = R_j + Pbar_j (1 + sigma), sigma ~ U[0, 2]."""
    spec = make_paper_instance(300, 4, 2, seed=1)
    assert spec.p.min() >= 1 and spec.p.max() <= 5 and spec.wt == 100
    pbar_j = spec.p.sum(axis=1)          # identical machines: sum_m P_jsm / M_s = p_js
    pbar = int(pbar_j.sum())
    assert spec.release.min() >= 0 and spec.release.max() <= pbar
    slack = spec.due - spec.release
    assert np.all(slack >= pbar_j) and np.all(slack <= 3 * pbar_j)
