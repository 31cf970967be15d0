"""The benchmark's bookkeeping, on the CPU: the algorithmic op count of a
decode, the kernels counted per generation, the whole-job rate, and the DRAM
traffic table keyed by launch shape."""
import bench


def test_ops_per_eval_hand_counts():
    # one stage of 3 machines, 4 jobs: 4 * ((3 - 1) + 3) = 20
    assert bench.ops_per_eval(4, [3]) == 20
    # two stages (2, 4 machines), 5 jobs: 5 * 4 + 5 * 6 + 5 * ceil(log2 2) = 55
    assert bench.ops_per_eval(5, [2, 4]) == 55
    # machines beyond the job count are clamped to n
    assert bench.ops_per_eval(2, [8]) == bench.ops_per_eval(2, [2])
    # one machine per stage: no merge term
    assert bench.ops_per_eval(10, [1, 1, 1]) == 3 * 10 * 3


def test_ops_per_eval_bench_instance():
    from ffs_workloads import workload_instance
    spec = workload_instance("scale_500x20")
    assert bench.ops_per_eval(spec.n, spec.M) == 124500


def test_launches_per_generation():
    from ffs_workloads import WORKLOADS
    # breeding, decode, pair replacement, advance; + ranking (2 launches) and the copy
    assert bench.launches_per_generation(WORKLOADS["scale_500x20"]) == 7
    assert bench.launches_per_generation(dict(WORKLOADS["dual_100x10"])) == 4   # migration every 50


def test_whole_job_rate_and_traffic_table():
    assert bench.whole_job_rate(1000, 4, 2.0) == 2000.0
    for (threads, chunk, variant), v in bench.K_STEP_DECODE_DRAM_BYTES.items():
        assert threads % 32 == 0 and chunk % 8 == 0 and 1 <= variant <= 4
        # at least the algorithmic bytes of a launch: 114,688 rows of 2n + 4 bytes
        assert v >= 114688 * (2 * 500 + 4)
