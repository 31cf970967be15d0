"""The CPU oracle built with AddressSanitizer and UndefinedBehaviorSanitizer
and run once over every entry point on small seeded cases (edge shapes
included: one job, M_s >= n, 32 machines, invalid genes, release and due
times): any out-of-bounds access, leak or undefined behaviour aborts the run
with a non-zero status."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as orc
from ffs_workloads import make_instance

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def _sanitizers_available(tmp_path) -> bool:
    src = tmp_path / "probe.c"
    src.write_text("int main(void){return 0;}\n")
    r = subprocess.run(["gcc", "-fsanitize=address,undefined", str(src), "-o", str(tmp_path / "probe")],
                       capture_output=True)
    return r.returncode == 0 and subprocess.run([str(tmp_path / "probe")]).returncode == 0


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_oracle_under_asan_and_ubsan(tmp_path):
    if not _sanitizers_available(tmp_path):
        pytest.skip("gcc sanitizer runtimes not available")
    exe = tmp_path / "oracle_sanitize"
    subprocess.check_call(["gcc", "-O1", "-g", "-std=c11", "-Wall", "-Werror", "-fsanitize=address,undefined",
                           "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-I", ORACLE_DIR,
                           os.path.join(ORACLE_DIR, "sanitize_check.c"), "-o", str(exe)])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "oracle sanitizer run ok" in r.stdout


def test_invalid_gene_gives_minus_one():
    """A job order with a gene outside [0, n) has no schedule: objective -1
    (the reading shared with the machine-assignment decoder)."""
    spec = make_instance(6, 3, 2, 3, seed=2)
    o = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    for bad in ([0, 1, 2, 3, 4, 6], [-1, 1, 2, 3, 4, 5], [5, 4, 3, 2, 1, 32767]):
        assert orc.decode(o, np.array(bad, dtype=np.int16)) == -1
    assert orc.decode(o, np.arange(6, dtype=np.int16)) > 0
