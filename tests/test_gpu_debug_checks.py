"""The FFS_DEBUG_CHECKS build: the checked library gives the oracle's
results with every device check passing, and reports a row that is not a
permutation (tests/debug_checks_run.py, run in a child process that loads
the checked library).  With FFS_EAGER=1 the same run takes the generations
launch by launch instead of from the captured graphs."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("eager", ["0", "1"])
def test_checked_build_passes_and_reports(gpu, eager):
    from paper_1903_10722_gb300 import _build
    _build.build(debug=True)
    env = dict(os.environ, FFS_DEBUG_CHECKS="1", FFS_EAGER=eager)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_checks_run.py")], capture_output=True, text=True,
                       env=env, timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "debug checks ok" in r.stdout
