"""Run by tests/test_gpu_debug_checks.py in a child process with
FFS_DEBUG_CHECKS=1, so that the checked library (libffs_gb300_debug.so) is
the one loaded: the GA paths give the oracle's results with every check
passing, and a row that is not a permutation, given by the host, is
reported."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle as orc  # noqa: E402
import paper_1903_10722_gb300 as gpu  # noqa: E402
from ffs_workloads import make_assign_instance, make_instance  # noqa: E402


def islands(mode):
    spec = make_instance(24, 6, 2, 5, seed=8)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.migration_mode = gpu.FFS_MIG_RING if mode == "ring" else gpu.FFS_MIG_PENETRATION
    prm.migration_gap = 4
    isl = gpu.Islands(g, prm, 2, 8, 8, 2, 64)
    ga = orc.IslandGA(o, orc.Params(seed=7), 2, 8, 8, 2, 64)
    for gen in range(1, 13):
        ga.step()
        if gen % 4 == 0:
            if mode == "ring":
                ga.migrate_ring(prm.ring_num, prm.ring_den)
            else:
                ga.migrate_penetration(prm.theta_num, prm.theta_den)
    gpu.ffs_island_step(isl, -1, 12)
    for i in range(len(ga.mss)):
        pop, ms = gpu.island_tensors(isl, i)
        torch.cuda.synchronize()
        assert np.array_equal(pop.cpu().numpy(), ga.pops[i][:, :spec.n]), (mode, i)
        assert np.array_equal(ms.cpu().numpy().astype(np.int64), ga.mss[i]), (mode, i)
    assert gpu.ffs_debug_check_error() == 0, mode


def batch():
    shapes = [(60, 18, 2, 6), (9, 3, 2, 4), (120, 20, 3, 9), (17, 2, 1, 3)]
    specs = [make_instance(n, S, lo, hi, seed=k + 2) for k, (n, S, lo, hi) in enumerate(shapes)]
    prm = gpu.ffs_params_default()
    prm.decode_variant, prm.decode_chunk, prm.block_threads = 3, 16, 128
    b = gpu.Batch(specs, prm, 6, 6)
    gpu.ffs_batch_step(b, 3)
    oprm = orc.Params(seed=7)
    for i, s in enumerate(specs):
        o = orc.Instance(s.n, s.S, s.M, s.p)
        ld = (s.n + 7) // 8 * 8
        pop = np.zeros((36, ld), dtype=np.int16)
        for c in range(36):
            pop[c, :s.n] = orc.init_chromosome(7, i, c, s.n)
        ms = orc.eval_population(o, pop)
        for gen in range(1, 4):
            pop, ms, _ = orc.cellular_generation(o, oprm, i, gen, 6, 6, pop, ms)
        p, m = gpu.batch_tensors(b, i)
        torch.cuda.synchronize()
        assert np.array_equal(p.cpu().numpy(), pop[:, :s.n]), i
        assert np.array_equal(m.cpu().numpy().astype(np.int64), ms), i
    gpu.ffs_batch_check(b)
    assert gpu.ffs_debug_check_error() == 0


def screened(screen_pseudo=0):
    spec = make_instance(40, 5, 2, 4, seed=5)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.migration_mode, prm.migration_gap = gpu.FFS_MIG_RING, 3
    isl = gpu.Islands(g, prm, 1, 8, 8, 1, 64)
    net = gpu.MLP(540, 512, 256, 64 * 8)
    net.init(3)
    sp = gpu.ffs_surrogate_params_default()
    sp.ring_capacity, sp.train_batch, sp.warmup_generations = 4096, 128, 2
    sp.screen_pseudo = screen_pseudo
    gpu.ffs_islands_attach_surrogate(isl, net, sp)
    gpu.ffs_island_step(isl, -1, 8)
    gpu.ffs_mlp_check(net)
    assert gpu.ffs_debug_check_error() == 0


def assign_ga():
    spec = make_assign_instance(20, 4, 2, 5, seed=4)
    o = orc.AssignInstance(spec.n, spec.S, spec.M, spec.p_u)
    g = gpu.AssignInstance(spec.n, spec.S, spec.M, spec.p_u)
    L = spec.n * spec.S
    ld = (L + 7) // 8 * 8
    N = 16
    prm = gpu.ffs_params_default()
    prm.cell_pm = gpu.threshold(0.5)
    oprm = orc.Params(seed=7, cell_pm=0.5)
    pop = torch.zeros((N, ld), dtype=torch.int16, device="cuda")
    gpu.ffs_assign_population_init(g, 7, 0, 0, N, ld, pop)
    obj = torch.empty(N, dtype=torch.int32, device="cuda")
    gpu.ffs_assign_eval(g, pop, N, ld, obj)
    opop = pop.cpu().numpy()
    oobj = orc.eval_population_assign(o, opop)
    scratch = torch.empty(gpu.ffs_assign_step_scratch_bytes(N, ld), dtype=torch.uint8, device="cuda")
    nxt, nobj = torch.empty_like(pop), torch.empty_like(obj)
    for gen in range(1, 4):
        gpu.ffs_assign_cellular_step(g, prm, 0, gen, 4, 4, ld, pop, obj, nxt, nobj, scratch)
        opop, oobj, _ = orc.assign_cellular_generation(o, oprm, 0, gen, 4, 4, opop, oobj)
        pop, nxt, obj, nobj = nxt, pop, nobj, obj
    torch.cuda.synchronize()
    assert np.array_equal(pop.cpu().numpy()[:, :L], opop[:, :L])
    assert np.array_equal(obj.cpu().numpy().astype(np.int64), oobj)
    assert gpu.ffs_debug_check_error() == 0


def reported_invalid_row():
    """A row with a repeated job (every gene inside [0, n)) given with a
    makespan of 1: the cell is never replaced, and the pass after the
    generation reports it (code 1)."""
    spec = make_instance(16, 3, 2, 3, seed=9)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    isl = gpu.Islands(g, gpu.ffs_params_default(), 1, 4, 4, 1, 16)
    rows, ms = gpu.island_tensors(isl, 0)
    rows = rows.cpu().numpy().copy()
    ms = ms.cpu().numpy().copy()
    rows[5, 1] = rows[5, 0]
    ms[5] = 1
    gpu.ffs_islands_set(isl, 0, rows, spec.n, ms)
    assert gpu.ffs_debug_check_error() == 0
    gpu.ffs_island_step(isl, -1, 1)
    assert gpu.ffs_debug_check_error(reset=True) == 1
    assert gpu.ffs_debug_check_error() == 0


def main():
    torch.cuda.set_device(0)
    assert gpu.ffs_debug_checks(), "the checked library is not the one loaded"
    assert gpu.ffs_debug_check_error(reset=True) == 0
    islands("ring")
    islands("penetration")
    batch()
    screened()
    screened(screen_pseudo=1)
    assign_ga()
    reported_invalid_row()
    print("debug checks ok")


if __name__ == "__main__":
    main()
