"""Benchmark: exact FFS makespan evaluations per second of the dual-island GA
on one GB300 (one JSON line on stdout).

Workload (default ``scale_500x20``): 500 jobs x 20 stages, machines per stage
uniform in [5, 10], processing times uniform in [1, 99] (instance seed 1);
4 cellular islands on 128 x 128 tori + 4 pseudo islands of 16384 rows
(131072 chromosomes of 500 int16 genes), GA seed 7.  A step is one
generation of every island (one breeding launch for the cellular cells and
the pseudo pairs, one decode launch for all children, the pseudo pair
replacement) followed by a ring migration of 2% (ranking + row copies),
replayed from the library's CUDA graph.  ``value`` = exact makespan evaluations
(children decoded) per second, counted by the library.

Other keys: ``roofline`` for the dominant kernel (the decode launch,
integer-ALU bound: algorithmic ops per launch / its CUDA-event duration
timed alone, against SMs x 128 lanes x max SM clock; ``group`` the same
with the breeding and pair-replacement launches around it; ``traffic`` its
DRAM bytes from an ncu capture at the launch shape in use), ``e2e`` (the
same step with the populations uploaded from and downloaded to pinned host
memory every step), ``cpu_baseline`` (the CPU oracle on a bounded sample),
``clocks`` (nvidia-smi sampled during the timed region), and two
sub-records: ``batch_256`` (256 uneven instances in one persistent launch,
with its own roofline and clocks) and ``surrogate_100x10`` (plain against
surrogate-screened GA over GA seeds 7..11: the median best-versus-time
curves, the time-to-plain-best ratio, rank quality and the per-generation
cost split); ``--no-subrecords`` leaves both out.

``--impl reference`` times the CPU oracle on this workload instead.  N > 1
(torchrun) runs independent replicas, one per GPU (the islands of one run
are not sharded across GPUs).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_SM_MHZ = 2070.0
LANES_PER_SM = 128


def ops_per_eval(n: int, M) -> int:
    """Algorithmic integer ops of one decode: per stage n * ((M_s - 1) + 3)
    (argmin compares, max, add, store) plus n * ceil(log2 M_{s-1}) for the
    merge into stage s >= 2's order."""
    import math
    Me = [min(int(m), n) for m in M]
    ops = sum(n * ((m - 1) + 3) for m in Me)
    ops += sum(n * math.ceil(math.log2(Me[s - 1])) if Me[s - 1] > 1 else 0 for s in range(1, len(Me)))
    return ops


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, dist, device: str = "cuda"):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank's times); identity without a process group."""
    if not dist:
        return list(values)
    import torch
    t = torch.tensor(list(values), device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(units_per_rank: float, world_size: int, max_time_s: float) -> float:
    """Units processed by all ranks (each processes units_per_rank) / the slowest rank's time."""
    return units_per_rank * world_size / max_time_s


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def _peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {}, "fallback"


def cpu_oracle_rate(workload: str, budget_s: float = 12.0, threads: int = 1):
    """CPU oracle: cellular generations on 16 x 16 tori of the same instance
    until ~budget_s, one independent island per thread (the oracle's C calls
    release the GIL, so threads run in parallel); returns (evals/s, sample
    description, threads)."""
    import concurrent.futures as cf

    import numpy as np

    import oracle as orc
    from ffs_workloads import workload_instance
    spec = workload_instance(workload)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = orc.Params(seed=7)
    rows = cols = 16
    ld = (spec.n + 7) // 8 * 8

    def island(t):
        pop = np.zeros((rows * cols, ld), dtype=np.int16)
        for c in range(rows * cols):
            pop[c, :spec.n] = orc.init_chromosome(7, t, c, spec.n)
        ms = orc.eval_population(o, pop)
        t0 = time.perf_counter()
        evals = gens = 0
        while time.perf_counter() - t0 < budget_s:
            gens += 1
            pop, ms, d = orc.cellular_generation(o, prm, t, gens, rows, cols, pop, ms)
            evals += d
        return evals, gens, time.perf_counter() - t0

    if threads == 1:
        results = [island(0)]
    else:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            results = list(ex.map(island, range(threads)))
    evals = sum(r[0] for r in results)
    gens = sum(r[1] for r in results)
    dt = max(r[2] for r in results)
    sample = (f"{gens} cellular generations of 16x16 tori ({evals} exact decodes) on the "
              f"{spec.n}x{spec.S} instance, {threads} thread(s), one island each, {dt:.1f} s")
    return evals / dt, sample, threads


def _shard_eval(args):
    """One process's shard of the sharded oracle figure: load the oracle,
    wait for the start time, evaluate rows [a, b) of the seeded batch."""
    import numpy as np

    import oracle as orc
    from ffs_workloads import random_population, workload_instance
    a, b, start_at = args
    spec = workload_instance("scale_500x20")
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    pop = random_population(spec.n, 4096, seed=11)[a:b]
    orc.eval_population(o, pop[:1])           # library loaded before the clock
    while time.time() < start_at:
        time.sleep(0.001)
    t0 = time.perf_counter()
    ms = orc.eval_population(o, pop)
    return float(time.perf_counter() - t0), int(np.asarray(ms).sum())


def run_oracle_full(args):
    """The oracle's full GA on the two small configurations, and the batch
    decoder on every host core as chromosome-sharded processes; one JSON line.

      * tiny (20 x 5, one 8 x 8 torus, 100 generations): the oracle on one
        core;
      * dual_100x10 (64 x 64 torus + pseudo 4096, ring 2 % every 50, 1000
        generations): the oracle with each island's cells / pairs split over
        one thread per core, and a 20-generation sample on one core;
      * 4096 random job orders of the 500 x 20 instance decoded by `nproc`
        processes (spawned; each takes a contiguous shard).
    With a GPU, the same two GA runs through the library (one
    ffs_island_step call each, CUDA-event time, graph capture before the
    clock) and their final best makespans and decode counts against the
    oracle's."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import oracle as orc
    from ffs_workloads import WORKLOADS, workload_instance

    cores = host_cores()
    out = {"metric": "oracle wall-clock of the full GA (configs tiny and dual_100x10) and sharded decoding",
           "workload": "oracle_full", "cores": cores}
    gpu = None
    try:
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(0)
            import paper_1903_10722_gb300 as gpu
    except ImportError:
        gpu = None

    def gpu_run(name):
        w = WORKLOADS[name]
        spec = workload_instance(name)
        inst = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
        prm = gpu.ffs_params_default()
        if w.get("migration") == "ring":
            prm.migration_mode, prm.migration_gap = gpu.FFS_MIG_RING, w["gap"]
            prm.ring_num, prm.ring_den = w["mig_num"], w["mig_den"]
        isl = gpu.Islands(inst, prm, w["n_cellular"], w["rows"], w["cols"], w["n_pseudo"], w["pseudo_size"])
        gpu.ffs_island_step(isl, -1, 1)               # generation 1 captures the graph, before the clock
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        gpu.ffs_island_step(isl, -1, w["generations"] - 1)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0
        return {"seconds_generations_2_on": t, "full_run_estimate_s": t * w["generations"] / (w["generations"] - 1),
                "best": int(gpu.ffs_islands_best(isl)[0]), "decoded": int(gpu.ffs_islands_decoded(isl))}

    # config tiny: one core
    w = WORKLOADS["tiny"]
    spec = workload_instance("tiny")
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    ga = orc.IslandGA(o, orc.Params(seed=7), 1, w["rows"], w["cols"], 0, 0)
    d0 = ga.decoded
    t0 = time.perf_counter()
    for _ in range(w["generations"]):
        ga.step()
    dt = time.perf_counter() - t0
    tiny = {"generations": w["generations"], "oracle_seconds": dt, "oracle_cores": 1,
            "oracle_evals_per_s": (ga.decoded - d0) / dt, "best": ga.best(), "decoded": ga.decoded}
    if gpu is not None:
        g = gpu_run("tiny")
        tiny["gpu"] = g
        tiny["gpu_matches_oracle"] = g["best"] == ga.best() and g["decoded"] == ga.decoded
    out["tiny"] = tiny

    # config dual_100x10: every core (threads over each island's cells / pairs), then a one-core sample
    w = WORKLOADS["dual_100x10"]
    spec = workload_instance("dual_100x10")
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    with cf.ThreadPoolExecutor(cores) as pool:
        ga = orc.IslandGA(o, orc.Params(seed=7), 1, w["rows"], w["cols"], 1, w["pseudo_size"], pool=pool,
                          parts=cores)
        d0 = ga.decoded
        t0 = time.perf_counter()
        for g in range(1, w["generations"] + 1):
            ga.step_threads(pool, cores)
            if g % w["gap"] == 0:
                ga.migrate_ring(w["mig_num"], w["mig_den"])
        dt = time.perf_counter() - t0
    dual = {"generations": w["generations"], "oracle_seconds": dt, "oracle_cores": cores,
            "oracle_evals_per_s": (ga.decoded - d0) / dt, "best": ga.best(), "decoded": ga.decoded}
    one = orc.IslandGA(o, orc.Params(seed=7), 1, w["rows"], w["cols"], 1, w["pseudo_size"])
    d0 = one.decoded
    t0 = time.perf_counter()
    for _ in range(20):
        one.step()
    dt1 = time.perf_counter() - t0
    dual["one_core_sample"] = {"generations": 20, "seconds": dt1, "evals_per_s": (one.decoded - d0) / dt1,
                               "full_run_estimate_s": dt1 / 20 * w["generations"]}
    if gpu is not None:
        g = gpu_run("dual_100x10")
        dual["gpu"] = g
        dual["gpu_matches_oracle"] = g["best"] == ga.best() and g["decoded"] == ga.decoded
    out["dual_100x10"] = dual

    # 4096 rows of the 500 x 20 instance over `cores` spawned processes
    N = 4096
    bounds = [(N * k // cores, N * (k + 1) // cores) for k in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_shard_eval, [(0, 1, 0.0)] * cores)   # workers up, oracle built
        start_at = time.time() + 1.0
        t0 = time.perf_counter()
        res = pool.map(_shard_eval, [(a, b, start_at) for a, b in bounds])
        wall = time.perf_counter() - t0 - 1.0
    slowest = max(r[0] for r in res)
    out["sharded_decode_500x20"] = {"rows": N, "processes": cores, "slowest_process_s": slowest,
                                    "evals_per_s": N / slowest, "wall_s_after_start": wall,
                                    "checksum": sum(r[1] for r in res)}
    print(json.dumps(out), flush=True)
    return 0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from ffs_workloads import WORKLOADS
    per_step = []
    total_evals = 0
    budget = max(0.5, min(20.0, 100.0 / max(1, args.steps + args.warmup)))   # whole run ~100 s
    cores = host_cores()
    for i in range(args.warmup + args.steps):
        rate, sample, _ = cpu_oracle_rate(args.workload, budget_s=budget, threads=cores)
        if i >= args.warmup:
            per_step.append(rate)
    value = statistics.mean(per_step)
    line = {
        "impl": "reference", "metric": "exact FFS makespan evals/sec", "value": value, "unit": "evals/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": budget * 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": _config(args.workload, ws),
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    del WORKLOADS
    print(json.dumps(line), flush=True)
    return 0


def _apply_shape(prm, args):
    """--shape THREADS,CHUNK,VARIANT pins the launch shape (no autotuning)."""
    if args.shape:
        prm.block_threads, prm.decode_chunk, prm.decode_variant = (int(x) for x in args.shape.split(","))


def _config(workload: str, ws: int) -> dict:
    from ffs_workloads import WORKLOADS
    w = WORKLOADS[workload]
    cfg = {"workload": workload, "n_jobs": w["n"], "n_stages": w["S"], "machines_per_stage": list(w["m"]),
           "cellular_islands": w["n_cellular"], "torus": [w["rows"], w["cols"]],
           "pseudo_islands": w["n_pseudo"], "pseudo_size": w["pseudo_size"],
           "chromosomes": w["n_cellular"] * w["rows"] * w["cols"] + w["n_pseudo"] * w["pseudo_size"],
           "migration": f"{w.get('migration', 'none')} {w.get('mig_num', 0)}/{w.get('mig_den', 1)} every "
                        f"{w.get('gap', 0)} generation(s)",
           "ga_seed": 7, "instance_seed": w["seed"], "parallelism": f"replicas x{ws}",
           "l2": "inputs larger than L2 (populations 2 x 131072 x 504 x 2 B = 264 MB)"}
    return cfg


def run_ours(args):
    import numpy as np
    import torch

    import paper_1903_10722_gb300 as ffs
    from ffs_workloads import WORKLOADS, workload_instance

    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    ffs.load()
    w = WORKLOADS[args.workload]
    spec = workload_instance(args.workload)
    inst = ffs.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = ffs.ffs_params_default()
    prm.seed = 7
    prm.migration_mode = ffs.FFS_MIG_RING if w.get("migration", "ring") == "ring" else ffs.FFS_MIG_PENETRATION
    prm.migration_gap = int(w.get("gap", 1))
    prm.ring_num, prm.ring_den = w.get("mig_num", 2), w.get("mig_den", 100)
    _apply_shape(prm, args)
    stream = torch.cuda.current_stream()
    isl = ffs.Islands(inst, prm, w["n_cellular"], w["rows"], w["cols"], w["n_pseudo"], w["pseudo_size"])
    tuned = None if args.no_autotune else ffs.ffs_islands_autotune(isl, repeats=8)
    if tuned:
        used = ffs.ffs_islands_params(isl)
        prm.decode_chunk, prm.block_threads, prm.decode_variant = used.decode_chunk, used.block_threads, used.decode_variant
        tuned["variant"] = used.decode_variant
    torch.cuda.synchronize()

    # ---- warm-up (also builds the CUDA graph) ----
    ffs.ffs_island_step(isl, -1, args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K generations replayed from the graph ----
    clocks = ClockSampler(dev_index)
    clocks.start()
    d0 = ffs.ffs_islands_decoded(isl)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ffs.ffs_island_step(isl, -1, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1000.0

    # ---- dominant kernel: the decode launch (all cellular and pseudo
    # children) timed alone with CUDA events on its stream: a dry run of the
    # breeding and replacement (untimed; the state does not advance), then
    # the decode launch by itself over the children it bred; the group of
    # breeding, decode and replacement launches is timed as well ----
    kernel_ms, group_ms = [], []
    for r in range(max(3, min(args.steps, 10))):
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        ffs.ffs_islands_dry_run(isl, 2)
        g1.record(stream)
        k0.record(stream)
        ffs.ffs_islands_dry_run(isl, 3)
        k1.record(stream)
        torch.cuda.synchronize()
        group_ms.append(g0.elapsed_time(g1))
        kernel_ms.append(k0.elapsed_time(k1))
    clock_info = clocks.stop()
    d1 = ffs.ffs_islands_decoded(isl)
    evals = d1 - d0
    # per-pipe integer rates (probe kernels, outside the timed regions; opt-in so
    # that the launch list of a plain run holds the generation's kernels only)
    int_rates = None
    # the measured issue rate of 32-bit min/max (the decoder's dominant
    # instruction), beside the nominal 128-lane peak
    minmax_rate = ffs.ffs_measure_int_rate(0)["lane_ops_per_s"]
    if args.int_rates:
        int_rates = {name: round(ffs.ffs_measure_int_rate(k)["lane_ops_per_s"] / 1e12, 2)
                     for k, name in enumerate(("min_max", "lop3", "iadd3", "imad", "fmnmx", "vminmax_u16x2",
                                               "min3_max3", "add_max", "min_max+imad", "min_max+fmnmx"))}

    # ---- e2e: the same steps with populations from / to pinned host memory ----
    # all islands' rows in one host buffer with the library's row stride.
    # Every step uploads every island's rows (ffs_islands_set), runs the
    # generation and downloads every island's rows and makespans
    # (ffs_islands_get); each island's upload for step k + 1 reads what its
    # download of step k wrote (ordered by events), so the round trip through
    # host memory is kept, while island i's upload overlaps island i + 1's
    # download on the other copy stream (the host link carries both
    # directions at once)
    total_rows = sum(isl.sizes)
    host_pop = torch.empty((total_rows, isl.ld), dtype=torch.int16).pin_memory()
    host_ms = torch.empty(total_rows, dtype=torch.int32).pin_memory()
    ffs.ffs_islands_get_all(isl, host_pop, isl.ld, host_ms)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 10))
    h2d = host_pop.numel() * 2
    d2h = h2d + host_ms.numel() * 4
    offs = [0]
    for size in isl.sizes:
        offs.append(offs[-1] + size)
    hp = [host_pop[offs[i]:offs[i + 1]] for i in range(isl.n_islands)]
    hm = [host_ms[offs[i]:offs[i + 1]] for i in range(isl.n_islands)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    down_done = [None] * isl.n_islands
    e_d0 = ffs.ffs_islands_decoded(isl)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for i in range(isl.n_islands):
            if down_done[i] is not None:
                up.wait_event(down_done[i])
            ffs.ffs_islands_set(isl, i, hp[i], isl.ld, None, stream=up)
        uploaded = torch.cuda.Event()
        uploaded.record(up)
        stream.wait_event(uploaded)
        ffs.ffs_island_step(isl, -1, 1, stream=stream)
        stepped = torch.cuda.Event()
        stepped.record(stream)
        down.wait_event(stepped)
        for i in range(isl.n_islands):
            ffs.ffs_islands_get(isl, i, hp[i], isl.ld, hm[i], stream=down)
            down_done[i] = torch.cuda.Event()
            down_done[i].record(down)
    torch.cuda.synchronize()
    e2e_time = time.perf_counter() - t0
    e2e_evals = ffs.ffs_islands_decoded(isl) - e_d0

    # ---- reduce over ranks (max time) ----
    value_time, e2e_time = max_over_ranks([elapsed, e2e_time], dist)
    value = whole_job_rate(evals, ws, value_time)

    peaks, peak_kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", FALLBACK_SM_MHZ))
    num_sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    peak_ops = num_sms * LANES_PER_SM * sm_max * 1e6
    ops_eval = ops_per_eval(spec.n, spec.M)
    kern_s = statistics.mean(kernel_ms) / 1000.0
    group_s = statistics.mean(group_ms) / 1000.0
    decodes_per_launch = evals / args.steps          # cellular cells + pseudo children per generation
    achieved = decodes_per_launch * ops_eval / kern_s
    achieved_group = decodes_per_launch * ops_eval / group_s

    line = {
        "metric": "exact FFS makespan evals/sec", "value": value, "unit": "evals/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value_time / args.steps * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded instance and Philox GA)",
        "config": _config(args.workload, ws),
        "e2e": {"value": e2e_evals * ws / e2e_time, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * launches_per_generation(w),
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s (int32 lane ops)", "frac": achieved / peak_ops,
                     "traffic": K_STEP_DECODE_DRAM_BYTES.get(
                         (prm.block_threads, prm.decode_chunk, prm.decode_variant)),
                     "kernel": "k_step_decode (all cellular children: decode + replace-if-better; all pseudo "
                               "children: decode), its launch timed alone",
                     "kernel_ms": statistics.mean(kernel_ms), "ops_per_launch": decodes_per_launch * ops_eval,
                     "frac_of_measured_minmax_rate": achieved / minmax_rate,
                     "measured_minmax_tops": minmax_rate / 1e12,
                     "group": {"what": "breeding (k_breed_dual) + decode (k_step_decode) + pseudo pair replacement "
                                       "launches of one generation", "ms": statistics.mean(group_ms),
                               "achieved": achieved_group / 1e12, "frac": achieved_group / peak_ops},
                     "peak_basis": f"{num_sms} SMs x {LANES_PER_SM} lanes x {sm_max:.0f} MHz ({peak_kind} max clock)",
                     "launch_shape": ffs.ffs_decode_plan(inst, 2, prm.decode_chunk, prm.block_threads,
                                                         prm.decode_variant),
                     "autotuned": tuned,
                     "measured_int_rate_tops": int_rates},
        "clocks": clock_info,
    }
    if ws == 1 and not args.no_subrecords:
        # the other measured configuration: 256 uneven instances in one
        # persistent launch per generation (its own timed region and clocks)
        sub = batch_measure("batch_256", steps=20, warmup=3, autotune=True, shape=None)
        sub["workload"] = ("batch_256: 256 instances, n ~ U[20,500], S ~ U[5,20], M_s ~ U[2,10], "
                           "p ~ U[1,99], one 32x32 cellular island each")
        line["batch_256"] = sub
        # the surrogate comparison (GA seeds 7..11)
        sur = surrogate_measure(list(range(7, 12)), plain_gens=1000, screened_gens=500)
        sur.pop("median_curves", None)
        line["surrogate_100x10"] = sur
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # all host cores, one island each (~8 s), and one thread alone (~8 s)
        cores = host_cores()
        rate, sample, used = cpu_oracle_rate(args.workload, budget_s=8.0, threads=cores)
        rate1, sample1, _ = cpu_oracle_rate(args.workload, budget_s=8.0, threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": "evals/s", "cores": used, "kind": "oracle", "sample": sample,
                                "single_thread": {"value": rate1, "sample": sample1}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    isl.close()
    inst.close()
    return 0


def batch_measure(workload: str, steps: int, warmup: int, autotune: bool, shape, dist=None, ws: int = 1) -> dict:
    """The batch of uneven instances (one cellular island each): creation,
    launch-shape autotuning, `warmup` generations, then `steps` generations
    timed with CUDA events on the launching stream (one persistent launch per
    generation, replayed from the CUDA graph).  Returns the measured fields."""
    import torch

    import paper_1903_10722_gb300 as ffs
    from ffs_workloads import WORKLOADS, make_batch

    dev_index = torch.cuda.current_device()
    w = WORKLOADS[workload]
    specs = make_batch(w["count"], seed=w["seed"])
    prm = ffs.ffs_params_default()
    if shape is not None:
        prm.block_threads, prm.decode_chunk, prm.decode_variant = shape
    b = ffs.Batch(specs, prm, w["rows"], w["cols"])
    tuned = ffs.ffs_batch_autotune(b, repeats=4) if autotune else b.info()
    tuned["variant"] = b.info()["variant"]
    stream = torch.cuda.current_stream()
    ffs.ffs_batch_step(b, warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev_index)
    clocks.start()
    d0 = ffs.ffs_batch_decoded(b)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ffs.ffs_batch_step(b, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = e0.elapsed_time(e1) / 1000.0
    clock_info = clocks.stop()
    evals = ffs.ffs_batch_decoded(b) - d0
    ffs.ffs_batch_check(b)
    elapsed = max_over_ranks([elapsed], dist)[0]
    # the dominant kernel alone: the decode launch on one breeding launch's
    # children (a generation that does not advance, then the decode launch
    # repeated), CUDA events on the launching stream
    ffs.ffs_batch_dry_run(b, 0)
    kts = []
    for _ in range(max(5, min(steps, 20))):
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        ffs.ffs_batch_dry_run(b, 1)
        k1.record(stream)
        torch.cuda.synchronize()
        kts.append(k0.elapsed_time(k1))
    ffs.ffs_batch_check(b)
    kernel_s = statistics.median(kts) / 1000.0
    minmax_rate = ffs.ffs_measure_int_rate(0)["lane_ops_per_s"]
    cells = w["rows"] * w["cols"]
    ops_gen = sum(cells * ops_per_eval(s.n, s.M) for s in specs)
    peaks, peak_kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", FALLBACK_SM_MHZ))
    num_sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    peak_ops = num_sms * LANES_PER_SM * sm_max * 1e6
    step_s = elapsed / steps
    b.close()
    shape_key = (tuned["threads"], tuned["chunk"], tuned["variant"])
    return {
        "value": evals * ws / elapsed, "unit": "evals/s", "steps": steps, "warmup": warmup,
        "ms_per_step": step_s * 1000.0, "launch_shape": tuned, "chromosomes": w["count"] * cells,
        "gpu_launches": 3 * steps,
        "roofline": {"bound": "alu", "achieved": ops_gen / kernel_s / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s (int32 lane ops)", "frac": ops_gen / kernel_s / peak_ops,
                     "traffic": K_BATCH_CELLULAR_DRAM_BYTES.get(shape_key),
                     "kernel": "k_batch_cellular (the persistent decode launch of one generation), timed alone",
                     "kernel_ms": kernel_s * 1000.0, "ops_per_launch": ops_gen,
                     "frac_of_measured_minmax_rate": ops_gen / kernel_s / minmax_rate,
                     "measured_minmax_tops": minmax_rate / 1e12,
                     "group": {"what": "one generation: breeding (k_batch_breed), counter reset, decode "
                                       "(k_batch_cellular) and generation advance",
                               "ms": step_s * 1000.0, "achieved": ops_gen / step_s / 1e12,
                               "frac": ops_gen / step_s / peak_ops},
                     "peak_basis": f"{num_sms} SMs x {LANES_PER_SM} lanes x {sm_max:.0f} MHz ({peak_kind} max clock)"},
        "clocks": clock_info,
    }


def run_batch(args):
    """256 uneven instances, one 32x32 cellular island each; a step is one
    generation of every instance (one persistent launch from the graph)."""
    import torch

    from ffs_workloads import WORKLOADS

    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    w = WORKLOADS[args.workload]
    shape = tuple(int(x) for x in args.shape.split(",")) if args.shape else None
    m = batch_measure(args.workload, args.steps, args.warmup, not args.no_autotune, shape, dist, ws)
    cells = w["rows"] * w["cols"]
    line = {
        "metric": "exact FFS makespan evals/sec", "value": m["value"], "unit": "evals/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded instances and Philox GA)",
        "config": {"workload": args.workload, "instances": w["count"], "n_jobs": list(w["n"]),
                   "n_stages": list(w["S"]), "machines_per_stage": list(w["m"]), "torus": [w["rows"], w["cols"]],
                   "chromosomes": w["count"] * cells, "launch_shape": m["launch_shape"],
                   "parallelism": f"replicas x{ws}"},
        "gpu_launches": m["gpu_launches"],
        "roofline": m["roofline"],
        "clocks": m["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _spearman(a, b) -> float:
    import numpy as np
    ra = np.argsort(np.argsort(a, kind="stable"), kind="stable").astype(np.float64)
    rb = np.argsort(np.argsort(b, kind="stable"), kind="stable").astype(np.float64)
    ra -= ra.mean()
    rb -= rb.mean()
    return float((ra * rb).sum() / np.sqrt((ra * ra).sum() * (rb * rb).sum()))


def _median_curve(curves, grid):
    """Median over seeds of best-so-far at each time of `grid` (a curve is
    [(seconds, best)] with the best at time 0 first)."""
    import numpy as np
    out = []
    for t in grid:
        vals = []
        for c in curves:
            b = c[0][1]
            for ts, bs in c:
                if ts <= t:
                    b = bs
            vals.append(b)
        out.append(float(np.median(vals)))
    return out


def surrogate_measure(seeds, plain_gens: int = 1000, screened_gens: int = 500, schedule: dict | None = None) -> dict:
    """Plain vs surrogate-screened dual-island GA on the 100 x 10 instance
    family (64x64 cellular + 4096 pseudo, ring 2% every 50): for every GA seed
    best makespan against wall-clock (host time around synchronised
    ffs_island_step calls of 10 generations, CUDA graph capture done before
    the clock starts), the median curves over the seeds, and the time the
    screened GA takes to reach the plain GA's final best, as a fraction of
    the plain GA's time.  The screen: 8 candidates per cell, the 540-512-256-1
    BF16 network (tcgen05 GEMMs) seeded by ffs_mlp_init, trained online with
    the library's default schedule; the exact decoder remains the source of
    every makespan."""
    import numpy as np
    import torch

    import paper_1903_10722_gb300 as ffs
    from ffs_workloads import WORKLOADS, workload_instance

    w = WORKLOADS["dual_100x10"]
    spec = workload_instance("dual_100x10")
    inst = ffs.Instance(spec.n, spec.S, spec.M, spec.p)
    sp0 = ffs.ffs_surrogate_params_default()
    for key, val in (schedule or {}).items():      # e.g. train_every, train_steps, candidates
        setattr(sp0, key, type(getattr(sp0, key))(val))
    cells, K = w["rows"] * w["cols"], sp0.candidates

    def make(seed, screened, train=True):
        prm = ffs.ffs_params_default()
        prm.seed = seed
        prm.migration_mode, prm.migration_gap = ffs.FFS_MIG_RING, w["gap"]
        isl = ffs.Islands(inst, prm, 1, w["rows"], w["cols"], 1, w["pseudo_size"])
        if screened:
            net = ffs.MLP(540, 512, 256, (cells * K + 127) // 128 * 128)
            net.init(3)
            sp = ffs.ffs_surrogate_params()
            ctypes.memmove(ctypes.addressof(sp), ctypes.addressof(sp0), ctypes.sizeof(sp))
            if not train:
                sp.train_every = 0
            ffs.ffs_islands_attach_surrogate(isl, net, sp)
        return isl

    def run(isl, gens):
        # the first generation (and the graph captures it triggers) before the clock
        ffs.ffs_island_step(isl, -1, 1)
        torch.cuda.synchronize()
        curve, t, done = [(0.0, ffs.ffs_islands_best(isl)[0])], 0.0, 1
        while done < gens:
            k = min(10, gens - done)
            t0 = time.perf_counter()
            ffs.ffs_island_step(isl, -1, k)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            done += k
            curve.append((t, ffs.ffs_islands_best(isl)[0]))
        return curve

    def spearman_cells(scores, exact):
        rs = []
        for c in range(cells):
            a, b = scores[c * K:(c + 1) * K], exact[c * K:(c + 1) * K]
            if np.ptp(b) > 0:
                rs.append(_spearman(a, b))
        return float(np.mean(rs)) if rs else None

    per_seed, plain_curves, scr_curves = {}, [], []
    rho_cell, rho_all, pick_best, pairs = [], [], [], 0
    for seed in seeds:
        isl = make(seed, False)
        pc = run(isl, plain_gens)
        isl.close()
        isl = make(seed, True)
        sc = run(isl, screened_gens)
        # rank quality of the last generation's scores against its candidates' exact makespans
        scores = np.zeros(cells * K, np.float32)
        cands = np.zeros((cells * K, spec.n), np.int16)
        pairs = ffs.ffs_islands_surrogate_last(isl, scores, None, None, cands, spec.n)
        exact = np.zeros(cells * K, np.int32)
        ffs.ffs_population_eval_host(inst, np.ascontiguousarray(np.pad(cands, ((0, 0), (0, inst.ld - spec.n)))),
                                     cells * K, inst.ld, exact)
        rho_cell.append(spearman_cells(scores, exact))
        rho_all.append(_spearman(scores, exact))
        picks = [int(np.argmin(scores[c * K:(c + 1) * K])) for c in range(cells)]
        pick_best.append(float(np.mean([exact[c * K + picks[c]] == exact[c * K:(c + 1) * K].min()
                                        for c in range(cells)])))
        isl.close()
        target, tp = pc[-1][1], pc[-1][0]
        reach = next((t for t, b in sc if b <= target), None)
        per_seed[str(seed)] = {"plain_best": target, "plain_s": tp, "screened_best": sc[-1][1],
                               "screened_s": sc[-1][0], "time_to_plain_best_ratio": (reach / tp) if reach else None}
        plain_curves.append(pc)
        scr_curves.append(sc)
    # median curves over the seeds on a common time grid
    t_end = max(max(c[-1][0] for c in plain_curves), max(c[-1][0] for c in scr_curves))
    grid = [t_end * i / 200 for i in range(201)]
    mp, ms = _median_curve(plain_curves, grid), _median_curve(scr_curves, grid)
    tp_end = float(np.median([c[-1][0] for c in plain_curves]))
    plain_final = _median_curve(plain_curves, [tp_end])[0]
    reach = next((t for t, b in zip(grid, ms) if b <= plain_final), None)
    # cost split: a screened generation alone (no training), a training round
    isl = make(seeds[0], True, train=False)
    g_no_train = run(isl, 101)
    isl.close()
    gen_ms = g_no_train[-1][0] / 100 * 1e3
    scr_ms = float(np.median([c[-1][0] for c in scr_curves])) / (screened_gens - 1) * 1e3
    plain_ms = tp_end / (plain_gens - 1) * 1e3
    te = max(sp0.train_every, 1)
    return {
        "metric": "best makespan vs wall-clock, plain vs surrogate-screened GA", "workload": "dual_100x10",
        "seeds": list(seeds), "plain_generations": plain_gens, "screened_generations": screened_gens,
        "exact_pairs_per_seed": pairs,
        "median": {"plain_final_best": plain_final, "plain_seconds": tp_end,
                   "screened_final_best": ms[-1], "time_to_plain_best_s": reach,
                   "time_to_plain_best_ratio": (reach / tp_end) if reach is not None else None,
                   "target_ratio": 0.5},
        "per_seed": per_seed,
        "rank_quality_last_generation": {"spearman_within_cell_mean": float(np.mean(rho_cell)),
                                         "spearman_all_candidates_mean": float(np.mean(rho_all)),
                                         "pick_is_best_fraction": float(np.mean(pick_best))},
        "ms_per_generation": {"plain": plain_ms, "screened_with_training": scr_ms,
                              "screened_without_training": gen_ms,
                              "training_round": (scr_ms - gen_ms) * te,
                              "schedule": {"candidates": sp0.candidates, "train_every": sp0.train_every,
                                           "train_steps": sp0.train_steps, "train_batch": sp0.train_batch,
                                           "lr": sp0.lr, "warmup_generations": sp0.warmup_generations}},
        "median_curves": {"t": [round(x, 5) for x in grid[::10]], "plain": mp[::10], "screened": ms[::10]},
    }


def run_surrogate(args):
    """Plain vs surrogate-screened GA over GA seeds 7..11 (1000 plain, 500
    screened generations each; --seeds, --plain-gens and --screened-gens give
    shorter runs, e.g. for a profiler); prints one JSON line."""
    import torch
    torch.cuda.set_device(0)
    seeds = [int(x) for x in args.seeds.split(",")] if args.seeds else list(range(7, 12))
    schedule = dict(kv.split("=") for kv in args.surrogate_schedule.split(",")) if args.surrogate_schedule else None
    line = surrogate_measure(seeds, plain_gens=args.plain_gens or 1000, screened_gens=args.screened_gens or 500,
                             schedule=schedule)
    print(json.dumps(line), flush=True)
    return 0


def run_mlp_forward(args):
    """The surrogate's scoring forward alone: the 540-512-256-1 BF16 network
    on 32768 rows (8 candidates for each cell of a 64 x 64 torus), one
    ffs_mlp_forward per step (two tcgen05 GEMM launches, the second with the
    output layer in its epilogue), L2 flushed between steps; one JSON line.
    Algorithmic FLOPs per row: 2 (540 * 512 + 512 * 256 + 256)."""
    import torch

    import paper_1903_10722_gb300 as ffs

    torch.cuda.set_device(0)
    B, in_dim, h1, h2 = 32768, 540, 512, 256
    net = ffs.MLP(in_dim, h1, h2, B)
    net.init(3)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    X = torch.zeros((B, net.width), dtype=torch.bfloat16, device="cuda")
    X[:, :in_dim] = torch.rand((B, in_dim), generator=g, device="cuda").to(torch.bfloat16)
    y = torch.empty(B, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        ffs.ffs_mlp_forward(net, X, net.width, B, y)
    ffs.ffs_mlp_check(net)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ffs.ffs_mlp_forward(net, X, net.width, B, y)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ffs.ffs_mlp_check(net)
    ms = statistics.median(ts)
    flops = 2.0 * B * (in_dim * h1 + h1 * h2 + h2)
    peaks, peak_kind = _peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    tf = flops / (ms / 1000.0) / 1e12
    line = {"metric": "surrogate scoring forward rows/sec", "workload": "surrogate_forward_32768",
            "value": B / (ms / 1000.0), "unit": "rows/s", "ms_per_step": ms, "steps": args.steps,
            "rows": B, "layers": [in_dim, h1, h2, 1], "dtype": "bf16 (fp32 accumulate)",
            "config": {"l2": "flushed between steps (256 MB write)"},
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": tf / peak, "kernel": "k_gemm_bf16 (both layers)",
                         "peak_basis": f"cuBLAS bf16 burst ({peak_kind})"}}
    print(json.dumps(line), flush=True)
    return 0


def run_decode(args):
    """The batched decoder alone: makespans of 131072 random job orders of the
    500 x 20 instance per step (ffs_population_eval_tuned), for each decoder
    variant at its best launch shape; one JSON line."""
    import torch

    import paper_1903_10722_gb300 as ffs
    from ffs_workloads import random_population, workload_instance

    torch.cuda.set_device(0)
    spec = workload_instance("scale_500x20")
    inst = ffs.Instance(spec.n, spec.S, spec.M, spec.p)
    N = 131072
    pop = torch.from_numpy(random_population(spec.n, N, seed=11)).cuda()
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    ops = N * ops_per_eval(spec.n, spec.M)
    peaks, peak_kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", FALLBACK_SM_MHZ))
    num_sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = num_sms * LANES_PER_SM * sm_max * 1e6
    results = {}
    shapes = [(0, 0)] if args.no_autotune else [(c, t) for c in (8, 16, 32, 48, 64, 96, 104, 112, 128) for t in (64, 128, 256, 320, 384, 448, 512)]
    variants = (1, 2, 3, 4)
    if args.shape:
        t, c, v = (int(x) for x in args.shape.split(","))
        shapes, variants = [(c, t)], (v,)
    names = {1: "single_stage", 2: "stage_pairs", 3: "single_stage_tmem", 4: "stage_pairs_tmem"}
    for variant in variants:
        best = None
        for chunk, threads in shapes:
            try:
                ffs.ffs_population_eval_tuned(inst, pop, N, inst.ld, out, chunk, threads, variant)
            except ffs.FFSError:
                continue
            ts = []
            for _ in range(max(3, args.warmup)):
                ffs.ffs_population_eval_tuned(inst, pop, N, inst.ld, out, chunk, threads, variant)
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ffs.ffs_population_eval_tuned(inst, pop, N, inst.ld, out, chunk, threads, variant)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            if best is None or ms < best["ms"]:
                best = {"chunk": chunk, "threads": threads, "ms": ms,
                        "plan": ffs.ffs_decode_plan(inst, 0, chunk, threads, variant)}
        best["evals_per_s"] = N / (best["ms"] / 1000.0)
        best["frac"] = ops / (best["ms"] / 1000.0) / peak_ops
        results[names[variant]] = best
    line = {"metric": "exact FFS makespan evals/sec (decoder alone)", "workload": "decode_500x20",
            "chromosomes": N, "ops_per_eval": ops_per_eval(spec.n, spec.M), "peak_tops": peak_ops / 1e12,
            "peak_basis": peak_kind, "variants": results}
    print(json.dumps(line), flush=True)
    return 0


def run_decode_small(args):
    """Decode launches too small to fill the GPU one chromosome per lane:
    the one-lane decoder (variant 3), the stage-parallel decoder (variant 5)
    and the library's choice (variant 0) on the small configurations' shapes.
    Per case and variant: 20 back-to-back calls between CUDA events (so that
    the host's launch work overlaps the previous decode), median over
    `steps` repetitions, L2 flushed between repetitions; one JSON line."""
    import torch

    import paper_1903_10722_gb300 as ffs
    from ffs_workloads import random_population, workload_instance

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    cases = [("dual_100x10", 4096), ("dual_100x10", 8192), ("paper_300x4", 512), ("tiny", 64),
             ("scale_500x20", 4096)]
    out = {"metric": "us per decode launch (small launches)", "workload": "decode_small", "calls_per_timing": 20,
           "cases": []}
    for name, N in cases:
        spec = workload_instance(name)
        g = ffs.Instance(spec.n, spec.S, spec.M, spec.p)
        pop = torch.from_numpy(random_population(spec.n, N, seed=1)).cuda()
        res = torch.empty(N, dtype=torch.int32, device="cuda")
        row = {"case": name, "rows": N, "n_jobs": spec.n, "n_stages": spec.S}
        ref = None
        for v in (3, 5, 0):
            for _ in range(max(3, args.warmup)):
                ffs.ffs_population_eval_tuned(g, pop, N, pop.shape[1], res, 0, 0, v)
            torch.cuda.synchronize()
            ts = []
            for _ in range(max(1, args.steps)):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(20):
                    ffs.ffs_population_eval_tuned(g, pop, N, pop.shape[1], res, 0, 0, v)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 20 * 1000.0)
            row[{3: "one_lane_us", 5: "stage_parallel_us", 0: "library_choice_us"}[v]] = statistics.median(ts)
            if ref is None:
                ref = res.clone()
            elif not torch.equal(ref, res):
                raise RuntimeError(f"decoders disagree on {name} N={N}")
        out["cases"].append(row)
    print(json.dumps(out), flush=True)
    return 0


def run_assign(args):
    """The paper's genotype: objectives of N random machine-assignment strings
    (500 jobs x 20 stages = 10000 genes per row) on unrelated machines
    (M_s ~ U[5,10], P_jsm ~ U[1,99]); one ffs_assign_eval per step; one JSON
    line.  Algorithmic bytes per row: its 2 n S bytes of genes, read once."""
    import torch

    import paper_1903_10722_gb300 as ffs
    from ffs_workloads import make_assign_instance, random_assignments

    torch.cuda.set_device(0)
    spec = make_assign_instance(500, 20, 5, 10, seed=1)
    inst = ffs.AssignInstance(spec.n, spec.S, spec.M, spec.p_u)
    N = 65536
    pop = torch.from_numpy(random_assignments(spec.n, spec.S, spec.M, N, seed=11)).cuda()
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        ffs.ffs_assign_eval(inst, pop, N, inst.ld, out)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ffs.ffs_assign_eval(inst, pop, N, inst.ld, out)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    peaks, peak_kind = _peaks()
    gbs = float(peaks.get("hbm_gbs", 6800.0))
    bytes_per_launch = N * spec.n * spec.S * 2
    line = {"metric": "exact FFS objective evals/sec (machine-assignment genotype)", "workload": "assign_500x20",
            "value": N / (ms / 1000.0), "unit": "evals/s", "ms_per_step": ms, "steps": args.steps,
            "rows": N, "genes_per_row": spec.n * spec.S, "machines_per_stage": [int(spec.M.min()), int(spec.M.max())],
            "roofline": {"bound": "latency", "achieved": bytes_per_launch / (ms / 1000.0) / 1e9,
                         "peak": gbs, "unit": "GB/s", "frac": bytes_per_launch / (ms / 1000.0) / 1e9 / gbs,
                         "kernel": "k_eval_assign", "peak_basis": f"HBM copy ({peak_kind})"}}
    print(json.dumps(line), flush=True)
    return 0


def run_paper(args):
    """The paper's Section 5 experiments on a synthetic Table 1 instance
    (300 jobs x 4 stages x 2 machines, p ~ U[1,5], release and due times,
    objective 100 * total tardiness + C_max): population 512, 2000
    generations, 50 GA seeds.  Table 2 setup: the dual GA (16 x 16 cellular
    island + 256-row pseudo island, penetration migration with theta = 1.00
    every 500 generations) against a cellular GA (16 x 32 torus) and a pseudo
    GA (512 rows) alone; Fig. 4 setup: the dual GA's final best for migration
    gaps 10 .. 800.  One JSON line; the paper's own values come from an
    unpublished instance and another genotype, so only the comparisons carry
    over."""
    import numpy as np
    import torch

    import paper_1903_10722_gb300 as ffs
    from ffs_workloads import make_paper_instance

    torch.cuda.set_device(0)
    gens, runs = 2000, (args.runs or 50)
    seeds = list(range(7, 7 + runs))
    per_instance = []
    for iseed in range(1, (args.instances or 1) + 1):
        spec = make_paper_instance(300, 4, 2, seed=iseed)
        inst = ffs.Instance(spec.n, spec.S, spec.M, spec.p, release=spec.release, due=spec.due, wt=spec.wt)
        per_instance.append(_paper_instance(ffs, inst, iseed, gens, seeds, sweep=iseed == 1))
    first = per_instance[0]
    line = {"metric": "best objective (100 x total tardiness + C_max) after 2000 generations",
            "workload": "paper_obj_300x4", "lower_is_better": True,
            "instance": "300 x 4 x 2, p ~ U[1,5], Table 1 release / due times, instance seeds 1.."
                        f"{len(per_instance)}",
            "population": 512, "generations": gens, "seeds": f"{seeds[0]}..{seeds[-1]}",
            "table2": first["table2"], "time": first["time"],
            "migration_gap_sweep_average": first["sweep"],
            "instances": [{"instance_seed": r["instance_seed"], "table2": r["table2"]} for r in per_instance]}
    print(json.dumps(line), flush=True)
    return 0


def _paper_instance(ffs, inst, iseed, gens, seeds, sweep):
    """Table 2 (dual, cellular, pseudo GA over the GA seeds) on one Table 1
    instance, and with sweep the Fig. 4 migration-gap sweep of the dual GA."""
    import numpy as np
    import torch
    runs = len(seeds)

    def run(kind, seed, gap=500):
        prm = ffs.ffs_params_default()
        prm.seed = seed
        prm.migration_mode = ffs.FFS_MIG_PENETRATION
        prm.theta_num, prm.theta_den = 1, 1
        prm.migration_gap = gap
        if kind == "dual":
            isl = ffs.Islands(inst, prm, 1, 16, 16, 1, 256)
        elif kind == "cellular":
            prm.migration_gap = 0
            isl = ffs.Islands(inst, prm, 1, 16, 32, 0, 0)
        else:
            prm.migration_gap = 0
            isl = ffs.Islands(inst, prm, 0, 0, 0, 1, 512)
        ffs.ffs_island_step(isl, -1, gens)
        best = ffs.ffs_islands_best(isl)[0]
        decoded = ffs.ffs_islands_decoded(isl)
        isl.close()
        return int(best), int(decoded)

    def summary(vals):
        a = np.array(vals, dtype=np.float64)
        return {"best": float(a.min()), "average": float(a.mean()), "variance": float(a.var(ddof=1)),
                "runs": len(vals)}

    table2, times = {}, {}
    for kind in ("dual", "cellular", "pseudo"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = [run(kind, sd) for sd in seeds]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        table2[kind] = summary([r[0] for r in res])
        times[kind] = {"s_per_run": dt / runs, "evals_per_s": sum(r[1] for r in res) / dt}
    gap_sweep = {}
    if sweep:
        for gap in (10, 50, 100, 200, 500, 800):
            gap_sweep[str(gap)] = summary([run("dual", sd, gap)[0] for sd in seeds])["average"]
    return {"instance_seed": iseed, "table2": table2, "time": times, "sweep": gap_sweep}


# DRAM bytes (read + write) of one k_step_decode launch of scale_500x20 at
# the launch shapes the autotuner picks, (threads, chunk, variant) -> bytes,
# from ncu captures of the current kernel (--metrics dram__bytes_read.sum,
# dram__bytes_write.sum); other shapes report null.
K_STEP_DECODE_DRAM_BYTES = {(384, 104, 3): 116_588_544 + 7_509_248, (384, 128, 3): 117_054_976 + 6_821_376}


# DRAM bytes of one k_batch_cellular (decode) launch of batch_256, per
# launch shape (threads, chunk, variant), from ncu captures of the current
# kernel (dram__bytes_read.sum + dram__bytes_write.sum); other shapes null.
K_BATCH_CELLULAR_DRAM_BYTES = {(384, 128, 3): 142_953_728 + 31_060_992}


def launches_per_generation(w) -> int:
    """Kernels of one generation: the breeding launch (cellular cells and
    pseudo pairs), the fused decode launch of all children, the pseudo pair
    replacement, the generation advance, and when migrating the two ranking
    launches plus the copy kernel."""
    n = 4
    if w.get("gap", 0) == 1 and w["n_cellular"] + w["n_pseudo"] > 1:
        n += 3
    return n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="scale_500x20")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="default workload: skip the surrogate sub-record")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--int-rates", action="store_true",
                    help="also measure per-pipe integer issue rates with the probe kernels")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shape")
    ap.add_argument("--seeds", default=None, help="surrogate_100x10: comma-separated GA seeds (default 7..11)")
    ap.add_argument("--plain-gens", type=int, default=0, help="surrogate_100x10: plain generations (default 1000)")
    ap.add_argument("--screened-gens", type=int, default=0,
                    help="surrogate_100x10: screened generations (default 500)")
    ap.add_argument("--surrogate-schedule", default=None,
                    help="surrogate_100x10: overrides of the screen's schedule, e.g. train_every=2,train_steps=1")
    ap.add_argument("--instances", type=int, default=0,
                    help="paper_obj_300x4: synthetic Table 1 instances (seeds 1..K; default 1)")
    ap.add_argument("--runs", type=int, default=0, help="paper_obj_300x4: GA seeds per setup (default 50)")
    ap.add_argument("--shape", default=None,
                    help="fixed launch shape THREADS,CHUNK,VARIANT instead of the autotuner (profiling)")
    args = ap.parse_args()
    if args.shape:
        args.no_autotune = True
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch_256":
        return run_batch(args)
    if args.workload == "surrogate_100x10":
        return run_surrogate(args)
    if args.workload == "oracle_full":
        return run_oracle_full(args)
    if args.workload == "surrogate_forward_32768":
        return run_mlp_forward(args)
    if args.workload == "decode_small":
        return run_decode_small(args)
    if args.workload == "decode_500x20":
        return run_decode(args)
    if args.workload == "assign_500x20":
        return run_assign(args)
    if args.workload == "paper_obj_300x4":
        return run_paper(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
