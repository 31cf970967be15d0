"""The oracle's screened pseudo generation, pinned to its definition's parts.

- A pair that does not cross is copied unchanged and reports -1. The decision is
  draw 0 of the pair's plain pseudo stream.
- Candidate t of a pair is the order crossover of the pair on the cuts of its own
  stream: draws 1 and 2 of purpose 32 + t.
- The winner is the candidate whose better child scores lowest, the lowest t on
  ties.
- The pair is replaced from the winner's two children as the plain generation
  replaces from its own: family best-2 of the decoded makespans, or the children
  themselves with pseudo_always.
- Every row stays a permutation, and two exact decodes are counted per crossing
  pair.

The expected values are assembled from primitives pinned elsewhere: Philox against
cuRAND's host generator, the order crossover against hand-worked rows, the decoder
against Gantt charts, family best-2 against its ranking rule."""
import numpy as np
import pytest

import oracle as orc
from ffs_workloads import make_instance

SEED, ISLAND, GEN = 7, 1, 3


def _pair_population(n, pairs):
    rows = []
    for k in range(pairs):
        a, b = orc.init_pseudo_pair(SEED, ISLAND, k, n)
        rows += [a, b]
    return np.array(rows, dtype=np.int16)


def _expected(o, prm, pop, ms, scores, K):
    n = o.n
    pairs = pop.shape[0] // 2
    out, out_ms = pop.copy(), ms.copy()
    chosen = np.full(pairs, -1, np.int32)
    cands = np.zeros((pairs * K * 2, n), np.int16)
    decoded = 0
    for k in range(pairs):
        a, b = pop[2 * k], pop[2 * k + 1]
        for t in range(K):
            u = orc.uniform(orc.draw(SEED, 32 + t, ISLAND, GEN, k, 1), n)
            v = orc.uniform(orc.draw(SEED, 32 + t, ISLAND, GEN, k, 2), n)
            l, r = min(u, v), max(u, v)
            cands[(k * K + t) * 2] = orc.order_crossover(a, b, l, r)
            cands[(k * K + t) * 2 + 1] = orc.order_crossover(b, a, l, r)
        if not orc.bernoulli(orc.draw(SEED, 3, ISLAND, GEN, k, 0), orc.threshold(prm.pseudo_pc)):
            continue
        better = np.minimum(scores[k * K * 2:(k + 1) * K * 2:2], scores[k * K * 2 + 1:(k + 1) * K * 2:2])
        t = int(np.argmin(better))   # the first minimum: the lowest t on ties
        chosen[k] = t
        c1, c2 = cands[(k * K + t) * 2], cands[(k * K + t) * 2 + 1]
        m = orc.eval_population(o, np.stack([c1, c2]))
        decoded += 2
        if prm.pseudo_always:
            out[2 * k], out[2 * k + 1] = c1, c2
            out_ms[2 * k], out_ms[2 * k + 1] = m
            continue
        fam = [c1, c2, a, b]
        fms = [m[0], m[1], ms[2 * k], ms[2 * k + 1]]
        f, s = orc.family_best2(fms)
        out[2 * k], out[2 * k + 1] = fam[f], fam[s]
        out_ms[2 * k], out_ms[2 * k + 1] = fms[f], fms[s]
    return out, out_ms, chosen, cands, decoded


@pytest.mark.parametrize("always", [False, True])
@pytest.mark.parametrize("n,S,K,pairs", [(30, 4, 8, 24), (9, 3, 3, 10), (1, 2, 2, 3)])
def test_screened_pseudo_generation_matches_its_definition(always, n, S, K, pairs):
    spec = make_instance(n, S, 2, 4, seed=n)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = orc.Params(seed=SEED, pseudo_always=always)
    pop = _pair_population(n, pairs)
    ms = orc.eval_population(o, pop)
    scores = np.random.default_rng(n + K).normal(0, 1, pairs * K * 2).astype(np.float32)
    got = orc.screened_pseudo_generation(o, prm, ISLAND, GEN, pop, ms, scores, K)
    want = _expected(o, prm, pop, ms, scores, K)
    for g, w in zip(got, want):
        assert np.array_equal(np.asarray(g), np.asarray(w))
    crossed = int((got[2] >= 0).sum())
    assert 0 < crossed < pairs or pairs < 4
    for row in got[0]:
        assert sorted(row.tolist()) == list(range(n))
    assert np.array_equal(got[1], orc.eval_population(o, got[0]))


def test_screened_pseudo_ties_pick_the_lowest_candidate():
    n, K, pairs = 20, 5, 16
    spec = make_instance(n, 3, 2, 3, seed=4)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    pop = _pair_population(n, pairs)
    ms = orc.eval_population(o, pop)
    _, _, chosen, _, _ = orc.screened_pseudo_generation(o, orc.Params(seed=SEED), ISLAND, GEN, pop, ms,
                                                        np.zeros(pairs * K * 2, np.float32), K)
    assert set(chosen.tolist()) <= {-1, 0}
    # one candidate made best by its second child only
    scores = np.ones(pairs * K * 2, np.float32)
    scores[(0 * K + 3) * 2 + 1] = -1.0
    _, _, chosen, _, _ = orc.screened_pseudo_generation(o, orc.Params(seed=SEED), ISLAND, GEN, pop, ms, scores, K)
    assert chosen[0] in (-1, 3)
