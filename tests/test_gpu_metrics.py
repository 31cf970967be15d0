"""Per-island, per-generation metrics (best, worst, sum and count of the
valid makespans, best so far, migrations received) recorded on the device
inside the generation graphs, against the same figures computed from the
oracle's populations generation by generation."""
import numpy as np
import pytest

import oracle as orc
from ffs_workloads import make_instance

pytestmark = pytest.mark.gpu


def _expected(ga, g, best_so_far, mig):
    rows = []
    for i, ms in enumerate(ga.mss):
        best_so_far[i] = min(best_so_far[i], int(ms.min()))
        rows.append([g, int(ms.min()), int(ms.max()), int(ms.sum()), len(ms), best_so_far[i], mig[i][0], mig[i][1]])
    return rows


def _ring_rows(sizes, num, den):
    """Rows island j receives per ring event: k of its predecessor i,
    max(1, floor(num * min(N_i, N_j) / den)) (capped at half the smaller island)."""
    I = len(sizes)
    out = []
    for j in range(I):
        i = (j - 1) % I
        nmin = min(sizes[i], sizes[j])
        out.append(min(max(1, (num * nmin) // den), nmin // 2))
    return out


@pytest.mark.parametrize("mode", ["ring", "penetration"])
def test_recorded_metrics_match_oracle(gpu, mode):
    spec = make_instance(30, 5, 2, 4, seed=6)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    gap = 3
    prm.migration_gap = gap
    prm.migration_mode = gpu.FFS_MIG_RING if mode == "ring" else gpu.FFS_MIG_PENETRATION
    if mode == "ring":
        prm.ring_num, prm.ring_den = 5, 100
    isl = gpu.Islands(g, prm, 2, 8, 8, 2, 64)
    ga = orc.IslandGA(o, orc.Params(seed=7), 2, 8, 8, 2, 64)
    cap, gens = 16, 21
    gpu.ffs_islands_record_stats(isl, cap)
    I = len(ga.mss)
    best_so_far = [1 << 62] * I
    mig = [[0, 0] for _ in range(I)]
    expected = {0: _expected(ga, 0, best_so_far, mig)}
    per_event = _ring_rows(ga.sizes, prm.ring_num, prm.ring_den)
    for gen in range(1, gens + 1):
        ga.step()
        if gen % gap == 0:
            if mode == "ring":
                ga.migrate_ring(prm.ring_num, prm.ring_den)
                for j in range(I):
                    mig[j][0] += 1
                    mig[j][1] += per_event[j]
            else:
                counts = ga.migrate_penetration(prm.theta_num, prm.theta_den)
                for q, c in enumerate(counts):
                    if c:
                        dst = 2 * q + 1 if c > 0 else 2 * q
                        mig[dst][0] += 1
                        mig[dst][1] += abs(c)
        expected[gen] = _expected(ga, gen, best_so_far, mig)
    gpu.ffs_island_step(isl, -1, gens)
    hist = gpu.ffs_islands_stats_history(isl)
    assert hist.shape == (cap, I, gpu.FFS_STAT_WORDS)
    for r in range(cap):
        gen = gens - cap + 1 + r
        assert hist[r].tolist() == expected[gen], gen
    assert sum(m[0] for m in mig) > 0          # migrations happened and were counted
    # the current generation's metrics, and the last record
    now = gpu.ffs_islands_stats(isl)
    assert now.tolist() == expected[gens]
    # switching off frees the ring; on again starts from the current generation
    gpu.ffs_islands_record_stats(isl, 0)
    assert gpu.ffs_islands_stats_history(isl).shape[0] == 0
    gpu.ffs_islands_record_stats(isl, 4)
    gpu.ffs_island_step(isl, -1, 2)
    h2 = gpu.ffs_islands_stats_history(isl)
    assert h2.shape[0] == 3 and h2[:, 0, 0].tolist() == [gens, gens + 1, gens + 2]


def test_metrics_without_recording_and_checkpoint(gpu):
    """ffs_islands_stats works without recording; the best-so-far value and
    the migration counters come back with a checkpoint."""
    spec = make_instance(20, 4, 2, 3, seed=3)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.migration_mode, prm.migration_gap = gpu.FFS_MIG_RING, 2
    isl = gpu.Islands(g, prm, 1, 8, 8, 1, 32)
    s0 = gpu.ffs_islands_stats(isl)
    assert (s0[:, 0] == 0).all() and (s0[:, 6] == 0).all() and (s0[:, 4] == [64, 32]).all()
    gpu.ffs_island_step(isl, -1, 6)
    s1 = gpu.ffs_islands_stats(isl)
    assert (s1[:, 0] == 6).all() and (s1[:, 6] == 3).all() and (s1[:, 5] <= s0[:, 5]).all()
    blob = gpu.ffs_checkpoint_save(isl)
    other = gpu.Islands(g, prm, 1, 8, 8, 1, 32)
    gpu.ffs_checkpoint_load(other, blob)
    assert gpu.ffs_islands_stats(other).tolist() == s1.tolist()
    with pytest.raises(gpu.FFSError):
        gpu.ffs_islands_record_stats(isl, -1)
