"""Pins of the oracle's decoder for the paper's genotype (Section 4.1: the
n*S machine-assignment string; Section 3: unrelated machines P_jsm), with
machines sequencing their jobs by arrival, ties by job index."""
import numpy as np

import oracle as orc
from ffs_workloads import make_instance


def _assign_from_identical(spec):
    """The unrelated-machine view of an identical-machine instance."""
    W = int(np.sum(spec.M))
    p_u = np.zeros((spec.n, W), dtype=np.int32)
    off = 0
    for s in range(spec.S):
        p_u[:, off:off + spec.M[s]] = spec.p[:, s:s + 1]
        off += spec.M[s]
    return p_u


def test_golden_examples(golden):
    for ex in golden("assign_examples.json")["examples"]:
        inst = orc.AssignInstance(ex["n"], ex["S"], ex["M"], ex["p_u"], ex.get("release"), ex.get("due"),
                                  ex.get("wt", 0))
        v, g = orc.decode_assign(inst, ex["genes"], gantt=True)
        assert v == ex["objective"], ex["name"]
        assert g.tolist() == ex["gantt"], ex["name"]


def test_same_schedule_as_list_scheduling_on_its_own_assignment():
    """On identical machines, list scheduling of the identity order assigns
    every operation a machine; decoding that assignment string gives the
    same schedule, operation by operation (at stage 1 both take the jobs in
    index order, later both by (completion, job), and a machine sees the
    same jobs in the same order)."""
    rng = np.random.default_rng(4)
    for trial in range(30):
        n, S = int(rng.integers(1, 40)), int(rng.integers(1, 7))
        spec = make_instance(n, S, 1, 5, seed=100 + trial)
        inst = orc.Instance(spec.n, spec.S, spec.M, spec.p)
        v, g = orc.decode(inst, np.arange(n, dtype=np.int16), gantt=True)
        genes = np.zeros(n * S, dtype=np.int16)
        for s, j, m, start, end in g:
            genes[j * S + s] = m
        ai = orc.AssignInstance(n, S, spec.M, _assign_from_identical(spec))
        va, ga = orc.decode_assign(ai, genes, gantt=True)
        assert va == v
        key = lambda r: (r[0], r[1])
        assert sorted(map(tuple, ga.tolist()), key=key) == sorted(map(tuple, g.tolist()), key=key)


def test_one_machine_per_stage_is_the_permutation_flow_shop():
    """M_s = 1: the textbook permutation flow shop with jobs in release order,
    C[k][s] = max(C[k-1][s], C[k][s-1]) + p, C[k][-1] = R of the k-th job."""
    rng = np.random.default_rng(5)
    for trial in range(20):
        n, S = int(rng.integers(1, 30)), int(rng.integers(1, 6))
        p = rng.integers(1, 50, size=(n, S))
        R = rng.integers(0, 80, size=n)
        order = sorted(range(n), key=lambda j: (R[j], j))
        C = np.zeros((n, S), dtype=np.int64)
        for k, j in enumerate(order):
            for s in range(S):
                prev_machine = C[order[k - 1], s] if k > 0 else 0
                prev_stage = C[j, s - 1] if s > 0 else R[j]
                C[j, s] = max(prev_machine, prev_stage) + p[j, s]
        inst = orc.AssignInstance(n, S, [1] * S, p, release=R)
        assert orc.decode_assign(inst, np.zeros(n * S, dtype=np.int16)) == int(C[:, -1].max())


def test_schedule_is_feasible_and_follows_the_genes():
    rng = np.random.default_rng(6)
    for trial in range(25):
        n, S = int(rng.integers(2, 25)), int(rng.integers(1, 6))
        M = rng.integers(1, 5, size=S)
        p_u = rng.integers(0, 30, size=(n, int(M.sum())))
        R = rng.integers(0, 40, size=n)
        inst = orc.AssignInstance(n, S, M, p_u, release=R)
        genes = np.array([rng.integers(0, M[s]) for j in range(n) for s in range(S)], dtype=np.int16)
        v, g = orc.decode_assign(inst, genes, gantt=True)
        off = np.concatenate([[0], np.cumsum(M)[:-1]])
        end = {}
        for s, j, m, a, b in g.tolist():
            assert m == genes[j * S + s]
            assert b - a == p_u[j, off[s] + m]
            assert a >= (end[(j, s - 1)] if s > 0 else R[j])
            end[(j, s)] = b
        for s in range(S):
            for m in range(M[s]):
                ops = sorted((a, b) for s2, j, m2, a, b in g.tolist() if s2 == s and m2 == m)
                assert all(ops[i][1] <= ops[i + 1][0] for i in range(len(ops) - 1))
        assert v == max(end[(j, S - 1)] for j in range(n))


def test_out_of_range_gene_is_invalid():
    inst = orc.AssignInstance(2, 2, [2, 1], [[1, 2, 3], [4, 5, 6]])
    assert orc.decode_assign(inst, [0, 0, 1, 0]) >= 0
    assert orc.decode_assign(inst, [2, 0, 1, 0]) == -1
    assert orc.decode_assign(inst, [0, 1, 1, 0]) == -1
    assert orc.decode_assign(inst, [0, 0, -1, 0]) == -1
