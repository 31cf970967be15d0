"""Failure handling, checkpoint/resume and tuning on the GPU: a bounded wait
that must run out reports FFS_ETIMEOUT and leaves the context usable; a run
interrupted and resumed from a host checkpoint equals the uninterrupted run;
autotuned launch shapes do not change results."""
import numpy as np
import pytest
import torch

import oracle as orc
from ffs_workloads import make_instance, random_population

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(gpu):
    rc, status = gpu.ffs_selftest_wait_timeout(1_000_000)   # 1 ms
    assert rc == gpu.FFS_ETIMEOUT and status == 1
    spec = make_instance(30, 4, 2, 3, seed=2)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    pop = random_population(30, 64, seed=1)
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    gpu.ffs_population_eval(g, torch.from_numpy(pop).cuda(), 64, pop.shape[1], out)
    torch.cuda.synchronize()
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), orc.eval_population(o, pop))


def test_int_rate_probe_reports_rates(gpu):
    for kind in range(10):
        r = gpu.ffs_measure_int_rate(kind)
        assert r["lane_ops_per_s"] > 1e12 and r["ms"] > 0


def _snapshot(gpu, isl, n):
    return [tuple(t.cpu().numpy().copy() for t in gpu.island_tensors(isl, i)) for i in range(isl.n_islands)]


def test_checkpoint_resume_is_exact(gpu):
    spec = make_instance(40, 5, 2, 4, seed=4)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.migration_mode, prm.migration_gap = gpu.FFS_MIG_RING, 3
    a = gpu.Islands(g, prm, 2, 8, 8, 2, 64)
    gpu.ffs_island_step(a, -1, 8)
    want = _snapshot(gpu, a, spec.n)
    b = gpu.Islands(g, prm, 2, 8, 8, 2, 64)
    gpu.ffs_island_step(b, -1, 5)
    ckpt = _snapshot(gpu, b, spec.n)
    c = gpu.Islands(g, prm, 2, 8, 8, 2, 64)
    for i, (pop, ms) in enumerate(ckpt):
        gpu.ffs_islands_set(c, i, np.ascontiguousarray(pop), spec.n, np.ascontiguousarray(ms))
    gpu.ffs_islands_set_generation(c, 5)
    gpu.ffs_island_step(c, -1, 3)
    got = _snapshot(gpu, c, spec.n)
    for (wp, wm), (gp, gm) in zip(want, got):
        assert np.array_equal(wp, gp) and np.array_equal(wm, gm)


def test_islands_autotune_keeps_results(gpu):
    spec = make_instance(100, 10, 2, 5, seed=9)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.migration_gap = 4
    a = gpu.Islands(g, prm, 1, 16, 16, 1, 256)
    b = gpu.Islands(g, prm, 1, 16, 16, 1, 256)
    tuned = gpu.ffs_islands_autotune(b, repeats=1)
    assert tuned["threads"] > 0 and tuned["chunk"] > 0 and tuned["ms"] > 0
    gpu.ffs_island_step(a, -1, 9)
    gpu.ffs_island_step(b, -1, 9)
    for (pa, ma), (pb, mb) in zip(_snapshot(gpu, a, spec.n), _snapshot(gpu, b, spec.n)):
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb)
    assert gpu.ffs_islands_decoded(a) == gpu.ffs_islands_decoded(b)
