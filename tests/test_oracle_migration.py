"""Pins of the oracle's migration (arXiv:1903.10722, Section 4.3, Eq. (1)-(2))."""
import numpy as np

import oracle as orc


def test_penetration_counts_golden(golden):
    for c in golden("operators.json")["penetration"]:
        got = orc.penetration_count(c["cA"], c["cB"], c["N"], c["theta"][0], c["theta"][1])
        assert got == c["count"], c


def test_penetration_against_rational_formula():
    # alpha = 1 - beta with beta = lo/hi; move iff 1 - beta < theta; count = floor(alpha N)
    from fractions import Fraction as F
    rng = np.random.default_rng(31)
    for _ in range(500):
        a, b = (int(v) for v in rng.integers(1, 400, size=2))
        N = int(rng.integers(1, 5000))
        th = F(int(rng.integers(0, 11)), 10)
        got = orc.penetration_count(a, b, N, th.numerator, th.denominator)
        if a == b:
            assert got == 0
            continue
        beta = F(min(a, b), max(a, b))
        want = int((1 - beta) * N) if (1 - beta) < th else 0
        assert abs(got) == want
        assert (got > 0) == (want > 0 and a < b)


def test_ring_golden(golden):
    g = golden("operators.json")["ring"]
    for case in g["cases"]:
        pops, mss = [], []
        for i, ms in enumerate(g["ms"]):
            pop = np.zeros((4, 3), dtype=np.int16)
            pop[:, 0] = [10 * i + c for c in range(4)]
            pops.append(pop)
            mss.append(np.array(ms, dtype=np.int64))
        orc.migrate_ring(pops, mss, 3, case["num"], case["den"])
        assert [m.tolist() for m in mss] == case["ms"]
        assert [p[:, 0].tolist() for p in pops] == case["first_gene"]


def test_penetration_moves_rows():
    popA = np.arange(8 * 2, dtype=np.int16).reshape(8, 2)
    popB = (100 + np.arange(8 * 2, dtype=np.int16)).reshape(8, 2)
    msA = np.array([10, 12, 11, 30, 10, 40, 50, 20], dtype=np.int64)
    msB = np.array([20, 25, 21, 22, 23, 24, 26, 27], dtype=np.int64)
    # best A = 10, best B = 20: beta = 1/2, theta 1 -> floor(8/2) = 4 rows A -> B
    cnt = orc.migrate_penetration(popA, msA, popB, msB, 2)
    assert cnt == 4
    # A ranked: (10,0) (10,4) (11,2) (12,1); B worst first: (27,7) (26,6) (25,1) (24,5)
    assert msB.tolist() == [20, 11, 21, 22, 23, 12, 10, 10]
    assert popB[7].tolist() == [0, 1] and popB[6].tolist() == [8, 9]
    assert popB[1].tolist() == [4, 5] and popB[5].tolist() == [2, 3]


def test_rank_island_ties_by_index():
    assert orc.rank_island(np.array([5, 3, 5, 3, 1])).tolist() == [4, 1, 3, 0, 2]
