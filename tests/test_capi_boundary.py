"""The C-ABI boundary without a GPU: the library builds for sm_103a, loads,
exports every entry point declared in include/ffs.h, and rejects invalid
instances before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1903_10722_gb300 as ffs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "ffs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ffs_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound():
    lib = ffs.load()
    names = _declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(ffs.exported_names()) | set(), set(names) - set(ffs.exported_names())


def test_params_defaults_follow_section5():
    p = ffs.ffs_params_default()
    assert p.seed == 7
    assert p.cell_pc == 2**32 and p.cell_pm == 214748364 and p.pseudo_pc == 3221225472
    assert p.migration_mode == ffs.FFS_MIG_RING and p.migration_gap == 50
    assert (p.ring_num, p.ring_den, p.theta_num, p.theta_den) == (2, 100, 1, 1)


def _create(n, S, M, p):
    h = ctypes.c_void_p()
    M = np.ascontiguousarray(M, dtype=np.int32)
    p = np.ascontiguousarray(p, dtype=np.int32)
    rc = ffs.load().ffs_instance_create(n, S, M.ctypes.data, p.ctypes.data, ctypes.byref(h))
    return rc, ffs.load().ffs_last_error().decode()


def test_instance_validation_before_device():
    assert _create(0, 2, [1, 1], np.ones((0, 2)))[0] == ffs.FFS_EINVAL
    assert _create(40000, 1, [1], np.ones((40000, 1)))[0] == ffs.FFS_EINVAL
    assert _create(3, 0, [], np.ones((3, 0)))[0] == ffs.FFS_EINVAL
    assert _create(3, 2, [1, 0], np.ones((3, 2)))[0] == ffs.FFS_EINVAL
    rc, msg = _create(3, 2, [1, 1], [[1, 1], [0, 1], [1, 1]])
    assert rc == ffs.FFS_EINVAL and "proc_time[1][0]" in msg
    assert _create(40, 1, [33], np.ones((40, 1)))[0] == ffs.FFS_EUNSUPPORTED
    # 500 jobs: keys hold 22 bits of time; 500 * 21 * 500 > 2^22
    assert _create(500, 21, [2] * 21, np.full((500, 21), 500))[0] == ffs.FFS_EOVERFLOW
    assert _create(5, 1, [1], np.full((5, 1), 70000))[0] == ffs.FFS_EUNSUPPORTED
    assert ffs.load().ffs_instance_create(3, 1, None, None, None) == ffs.FFS_EINVAL


def test_null_handles_are_rejected():
    lib = ffs.load()
    assert lib.ffs_population_eval(None, None, 1, 8, None, None) == ffs.FFS_EINVAL
    assert lib.ffs_island_step(None, -1, 1, None) == ffs.FFS_EINVAL
    assert lib.ffs_migrate(None, 1, None) == ffs.FFS_EINVAL
    assert lib.ffs_pseudo_scratch_bytes(-1, 8) == -1
    assert lib.ffs_pseudo_scratch_bytes(4096, 104) >= 4096 * 104 * 2 + 4096 * 4


def test_normal_build_reports_no_checks():
    """The library loaded by default is the unchecked one; its check word is
    always 0 (no device access)."""
    import paper_1903_10722_gb300 as ffs
    if ffs.debug_checks_requested():
        pytest.skip("the checked build is selected in this environment")
    assert ffs.ffs_debug_checks() is False
    assert ffs.ffs_debug_check_error(stream=0) == 0
