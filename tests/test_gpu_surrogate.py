"""Surrogate-screened cellular generations against the oracle: given the
network's scores (dumped from the GPU), the oracle's screened generation must
reproduce the populations and the picks bit-exactly; the scores themselves
must match the float64 network oracle on the oracle's own candidate features."""
import numpy as np
import pytest
import torch

import oracle as orc
from ffs_workloads import make_instance
from ffs_workloads import mlp_params
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _setup(gpu, n, S, mlo, mhi, rows, cols, n_pseudo, psize, K, warmup, train_every, seed=7, variant=0,
           overlap=0):
    spec = make_instance(n, S, mlo, mhi, seed=n + S)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.seed = seed
    prm.decode_variant = variant
    prm.migration_mode, prm.migration_gap = 0, 0
    isl = gpu.Islands(g, prm, 1, rows, cols, n_pseudo, psize)
    params = mlp_params(540, 512, 256, seed=11)
    params["b1"] = np.random.default_rng(1).normal(0, 0.05, 512).astype(np.float32)
    net = gpu.MLP(540, 512, 256, max(1024, ((rows * cols * K + 127) // 128) * 128))
    net.set_params(params)
    sp = gpu.ffs_surrogate_params_default()
    sp.candidates, sp.warmup_generations, sp.train_every = K, warmup, train_every
    sp.train_batch, sp.train_steps = 256, 2
    sp.ring_capacity = max(4096, rows * cols * 4)
    sp.overlap = overlap
    gpu.ffs_islands_attach_surrogate(isl, net, sp)
    ga = orc.IslandGA(o, orc.Params(seed=seed), 1, rows, cols, n_pseudo, psize)
    return spec, o, g, isl, ga, params


def _compare(gpu, isl, ga, n, tag):
    for i in range(isl.n_islands):
        pop, ms = gpu.island_tensors(isl, i)
        torch.cuda.synchronize()
        assert np.array_equal(pop.cpu().numpy(), ga.pops[i][:, :n]), (tag, i)
        assert np.array_equal(ms.cpu().numpy().astype(np.int64), ga.mss[i]), (tag, i)


@pytest.mark.parametrize("warmup,variant,n,rows,cols,K", [(0, 0, 20, 8, 8, 8), (2, 0, 20, 8, 8, 8),
                                                         (2, 5, 20, 8, 8, 8), (2, 0, 130, 8, 8, 8),
                                                         (2, 0, 37, 5, 5, 3)])
def test_screened_generations_match_oracle_given_scores(gpu, warmup, variant, n, rows, cols, K):
    """variant 5: the picks decoded by the stage-parallel select kernel and
    the pseudo children by the stage-parallel eval kernel.  n = 130: the
    candidates built a whole warp per child (rows above 120 genes), else two
    per warp; 5 x 5 cells x 3 candidates: a last warp with an odd number of
    candidates (one half idle)."""
    spec, o, g, isl, ga, params = _setup(gpu, n, 5, 3, 3, rows, cols, 1, 32, K, warmup, 0, variant=variant)
    inst_feat = omlp.instance_features(spec.n, spec.S, spec.M, spec.p)
    cells = rows * cols
    for gen in range(1, 5):
        gpu.ffs_island_step(isl, -1, 1)
        scores = np.zeros(cells * K, np.float32)
        chosen = np.zeros(cells, np.int32)
        gpu.ffs_islands_surrogate_last(isl, scores, chosen)
        torch.cuda.synchronize()
        pop, ms, want_chosen, cands = orc.screened_cellular_generation(
            o, ga.prm, 0, gen, rows, cols, ga.pops[0], ga.mss[0], scores, K)
        assert chosen.tolist() == want_chosen.tolist(), gen
        ga.pops[0], ga.mss[0] = pop, ms
        ga.pops[1], ga.mss[1], d = orc.pseudo_generation(o, ga.prm, 1, gen, ga.pops[1], ga.mss[1])
        _compare(gpu, isl, ga, spec.n, gen)
        if gen <= warmup:
            assert not scores.any()
        else:
            X = omlp.features(cands, spec.n, 500, inst_feat)
            want, _ = omlp.forward(params, X, rounded=True)
            scale = np.mean(np.abs(want)) + 1e-3
            assert np.max(np.abs(scores - want)) <= 2e-2 * scale, gen


@pytest.mark.parametrize("warmup,always,n,train", [(0, False, 20, 0), (2, False, 37, 0), (2, True, 130, 0),
                                                   (1, False, 60, 1)])
def test_screened_pseudo_generations_match_oracle_given_scores(gpu, warmup, always, n, train):
    """screen_pseudo = 1: the pseudo island's pairs screened too.  Given the
    GPU's scores (cellular and pseudo), the oracle's screened generations
    reproduce both islands, the cellular picks and the pseudo picks (-1 for
    pairs that did not cross); the pseudo scores match the float64 network
    on the oracle's own candidate children.  n = 130: whole-warp crossover;
    train = 1: with the training round beside the screen."""
    rows, cols, K, psize = 8, 8, 4, 64
    spec = make_instance(n, 4, 2, 4, seed=n)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.seed = 7
    prm.pseudo_always = int(always)
    prm.migration_mode, prm.migration_gap = 0, 0
    isl = gpu.Islands(g, prm, 1, rows, cols, 1, psize)
    params = mlp_params(540, 512, 256, seed=11)
    params["b1"] = np.random.default_rng(1).normal(0, 0.05, 512).astype(np.float32)
    net = gpu.MLP(540, 512, 256, 1024)
    net.set_params(params)
    sp = gpu.ffs_surrogate_params_default()
    sp.candidates, sp.warmup_generations, sp.train_every = K, warmup, train
    sp.train_batch, sp.train_steps, sp.ring_capacity = 128, 2, 4096
    sp.screen_pseudo = 1
    gpu.ffs_islands_attach_surrogate(isl, net, sp)
    ga = orc.IslandGA(o, orc.Params(seed=7, pseudo_always=always), 1, rows, cols, 1, psize)
    inst_feat = omlp.instance_features(spec.n, spec.S, spec.M, spec.p)
    cells, pairs = rows * cols, psize // 2
    for gen in range(1, 6):
        before = net.get()
        gpu.ffs_island_step(isl, -1, 1)
        scores = np.zeros(cells * K, np.float32)
        chosen = np.zeros(cells, np.int32)
        gpu.ffs_islands_surrogate_last(isl, scores, chosen)
        pscores = np.zeros(pairs * K * 2, np.float32)
        pchosen = np.zeros(pairs, np.int32)
        gpu.ffs_islands_surrogate_last_pseudo(isl, pscores, pchosen)
        torch.cuda.synchronize()
        pop, ms, want_chosen, _ = orc.screened_cellular_generation(o, ga.prm, 0, gen, rows, cols, ga.pops[0],
                                                                   ga.mss[0], scores, K)
        assert chosen.tolist() == want_chosen.tolist(), gen
        ga.pops[0], ga.mss[0] = pop, ms
        pop, ms, want_p, cands, _ = orc.screened_pseudo_generation(o, ga.prm, 1, gen, ga.pops[1], ga.mss[1],
                                                                   pscores, K)
        assert pchosen.tolist() == want_p.tolist(), gen
        ga.pops[1], ga.mss[1] = pop, ms
        _compare(gpu, isl, ga, spec.n, gen)
        if gen <= warmup:
            assert not pscores.any()
        else:
            # the screen scores with the weights as they stood when the generation began
            X = omlp.features(cands, spec.n, 500, inst_feat)
            want, _ = omlp.forward(before, X, rounded=True)
            scale = np.mean(np.abs(want)) + 1e-3
            assert np.max(np.abs(pscores - want)) <= 2e-2 * scale, gen
        assert (want_p >= 0).any() and (want_p < 0).any()


@pytest.mark.parametrize("overlap", [0, 1])
def test_screened_training_runs_and_keeps_parity(gpu, overlap):
    rows, cols, K = 16, 16, 8
    spec, o, g, isl, ga, params = _setup(gpu, 60, 6, 2, 4, rows, cols, 0, 0, K, 1, 1, overlap=overlap)
    cells = rows * cols
    losses = []
    for gen in range(1, 13):
        gpu.ffs_island_step(isl, -1, 1)
        scores = np.zeros(cells * K, np.float32)
        loss = np.zeros(1, np.float32)
        pairs = gpu.ffs_islands_surrogate_last(isl, scores, None, loss)
        torch.cuda.synchronize()
        pop, ms, _, _ = orc.screened_cellular_generation(o, ga.prm, 0, gen, rows, cols, ga.pops[0], ga.mss[0],
                                                         scores, K)
        ga.pops[0], ga.mss[0] = pop, ms
        _compare(gpu, isl, ga, spec.n, gen)
        assert pairs == gen * cells
        if gen >= 2:   # the first training round runs at the start of generation 2
            losses.append(float(loss[0]))
    # the targets are standardised by the latest generation's makespans, a
    # scale that moves every generation, so the loss is checked for sanity
    # only; generation G trains on the pairs of generations 1..G-1 (256 per
    # generation), so generations 2..12 each ran a round of 2 steps
    assert all(np.isfinite(losses)) and all(x > 0 for x in losses)
    assert isl.surrogate.adam_steps() == 2 * 11
    assert np.ptp(scores) > 0


@pytest.mark.parametrize("overlap", [0, 1])
def test_overlap_scores_with_the_weights_of_the_generation_start(gpu, overlap):
    """overlap = 1: the training round runs beside the whole screen, which
    scores with the network as it stood when the generation began; overlap =
    0: the round ends before the scoring, which reads its result.  A large
    learning rate makes the two networks' scores differ far beyond the
    forward pass's tolerance, so the test tells the two apart."""
    rows, cols, K, n = 16, 16, 4, 24
    spec = make_instance(n, 5, 2, 4, seed=9)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = gpu.ffs_params_default()
    prm.migration_mode, prm.migration_gap = 0, 0
    isl = gpu.Islands(g, prm, 1, rows, cols, 0, 0)
    net = gpu.MLP(540, 512, 256, rows * cols * K)
    net.init(5)
    sp = gpu.ffs_surrogate_params_default()
    sp.candidates, sp.warmup_generations, sp.train_every = K, 0, 1
    sp.train_batch, sp.train_steps, sp.lr, sp.ring_capacity = 128, 2, 0.02, 2048
    sp.overlap = overlap
    gpu.ffs_islands_attach_surrogate(isl, net, sp)
    inst_feat = omlp.instance_features(spec.n, spec.S, spec.M, spec.p)
    cells = rows * cols
    told_apart = 0
    for gen in range(1, 7):
        before = net.get()
        gpu.ffs_island_step(isl, -1, 1)
        after = net.get()
        scores = np.zeros(cells * K, np.float32)
        cands = np.zeros((cells * K, n), np.int16)
        gpu.ffs_islands_surrogate_last(isl, scores, None, None, cands, n)
        torch.cuda.synchronize()
        X = omlp.features(cands, n, 500, inst_feat)
        y_before, _ = omlp.forward(before, X, rounded=True)
        y_after, _ = omlp.forward(after, X, rounded=True)
        want = y_before if overlap else y_after
        tol = 2e-2 * (np.mean(np.abs(want)) + 1e-3)
        assert np.max(np.abs(scores - want)) <= tol, gen
        told_apart += int(np.max(np.abs(y_before - y_after)) > 10 * tol)
    assert net.adam_steps() == 2 * 5      # rounds at the start of generations 2..6
    assert told_apart >= 3


def test_overlap_needs_a_ring_of_two_generations(gpu):
    spec = make_instance(20, 4, 2, 3, seed=3)
    g = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    isl = gpu.Islands(g, gpu.ffs_params_default(), 1, 32, 32, 0, 0)
    net = gpu.MLP(540, 512, 256, 4096)
    sp = gpu.ffs_surrogate_params_default()
    sp.candidates, sp.train_batch, sp.ring_capacity, sp.overlap = 4, 128, 1024 + 128, 1
    with pytest.raises(gpu.FFSError) as e:
        gpu.ffs_islands_attach_surrogate(isl, net, sp)
    assert e.value.status == gpu.FFS_EINVAL
    sp.overlap = 2
    sp.ring_capacity = 4096
    with pytest.raises(gpu.FFSError):
        gpu.ffs_islands_attach_surrogate(isl, net, sp)
    sp.overlap = 1
    gpu.ffs_islands_attach_surrogate(isl, net, sp)


def test_trained_screen_beats_plain_ga_at_equal_exact_decodes(gpu):
    """100 x 10 instance family (64x64 cellular + pseudo 4096, ring 2% every 50):
    after 100 generations -- the same number of exact decodes per cell -- the
    screened GA with the online-trained network holds a lower best makespan
    than the plain GA (seeded run; the wall-clock comparison is reported by
    bench.py --workload surrogate_100x10)."""
    from ffs_workloads import WORKLOADS, workload_instance
    w = WORKLOADS["dual_100x10"]
    spec = workload_instance("dual_100x10")
    inst = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    best = {}
    for mode in ("plain", "screened"):
        prm = gpu.ffs_params_default()
        prm.migration_mode, prm.migration_gap = gpu.FFS_MIG_RING, w["gap"]
        isl = gpu.Islands(inst, prm, 1, w["rows"], w["cols"], 1, w["pseudo_size"])
        if mode == "screened":
            net = gpu.MLP(540, 512, 256, w["rows"] * w["cols"] * 8)
            net.init(3)
            gpu.ffs_islands_attach_surrogate(isl, net, gpu.ffs_surrogate_params_default())
        gpu.ffs_island_step(isl, -1, 100)
        best[mode] = gpu.ffs_islands_best(isl)[0]
        decoded = gpu.ffs_islands_decoded(isl)
        best[mode + "_decoded"] = decoded
        isl.close()
    print("best makespan after 100 generations:", best)
    assert best["screened"] < best["plain"]
