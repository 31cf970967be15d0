"""ffs_pseudo_step_noalloc: the pseudo-island generation for callers that
cannot allocate device memory.  It must give exactly what ffs_pseudo_step
gives with caller-provided scratch, and what the CPU oracle's pseudo
generation gives, call after call (the fixed scratch array is shared and
reused), and refuse islands too large for the array.

Collected last on purpose (file name), so a stop-at-first-failure run has
run every other test before this one."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
import paper_1903_10722_gb300 as ffs
from ffs_workloads import make_instance

pytestmark = pytest.mark.gpu


def _step_noalloc_cabi(lib, inst, prm, island, gen, size, ld, a, ma, b, mb):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.ffs_pseudo_step_noalloc(inst.handle, ctypes.byref(prm), island, gen, size, ld, a.data_ptr(),
                                       ma.data_ptr(), b.data_ptr(), mb.data_ptr(), stream)


def test_noalloc_pseudo_step_matches_caller_scratch_twice():
    assert torch.cuda.is_available()
    lib = ffs.load()
    spec = make_instance(100, 10, 2, 5, seed=21)
    inst = ffs.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = ffs.ffs_params_default()
    size, ld = 2048, inst.ld
    pop0 = torch.empty((size, ld), dtype=torch.int16, device="cuda")
    ms0 = torch.empty(size, dtype=torch.int32, device="cuda")
    ffs.ffs_population_init(inst, 7, 1, 1, size, ld, pop0)
    ffs.ffs_population_eval(inst, pop0, size, ld, ms0)
    scratch = torch.empty(ffs.ffs_pseudo_scratch_bytes(size, ld), dtype=torch.uint8, device="cuda")

    ref_a, ref_ma = pop0.clone(), ms0.clone()
    new_a, new_ma = pop0.clone(), ms0.clone()
    ref_b, ref_mb = torch.empty_like(pop0), torch.empty_like(ms0)
    new_b, new_mb = torch.full_like(pop0, -1), torch.full_like(ms0, -1)
    oinst = orc.Instance(spec.n, spec.S, spec.M, spec.p)
    opop = pop0.cpu().numpy()
    oms = ms0.cpu().numpy().astype(np.int64)
    for gen in (1, 2):
        ffs.ffs_pseudo_step(inst, prm, 1, gen, size, ld, ref_a, ref_ma, ref_b, ref_mb, scratch)
        rc = _step_noalloc_cabi(lib, inst, prm, 1, gen, size, ld, new_a, new_ma, new_b, new_mb)
        assert rc == ffs.FFS_OK, lib.ffs_last_error()
        torch.cuda.synchronize()
        # integer results: the tolerance is exact equality
        assert torch.equal(new_b[:, :spec.n], ref_b[:, :spec.n]), gen
        assert torch.equal(new_mb, ref_mb), gen
        opop, oms, _ = orc.pseudo_generation(oinst, orc.Params(seed=prm.seed), 1, gen, opop, oms)
        assert np.array_equal(new_b[:, :spec.n].cpu().numpy(), opop[:, :spec.n]), gen
        assert np.array_equal(new_mb.cpu().numpy().astype(np.int64), oms), gen
        ref_a, ref_b, ref_ma, ref_mb = ref_b, ref_a, ref_mb, ref_ma
        new_a, new_b, new_ma, new_mb = new_b, new_a, new_mb, new_ma


def test_noalloc_rejects_islands_beyond_the_fixed_scratch():
    lib = ffs.load()
    spec = make_instance(500, 4, 2, 3, seed=2)
    inst = ffs.Instance(spec.n, spec.S, spec.M, spec.p)
    prm = ffs.ffs_params_default()
    size, ld = 16384, inst.ld
    assert ffs.ffs_pseudo_scratch_bytes(size, ld) > ffs.FFS_NOALLOC_SCRATCH_BYTES
    # buffers of the full island size (about 33 MB), so that even a call that
    # failed to refuse the size would stay inside them
    a = torch.zeros((size, ld), dtype=torch.int16, device="cuda")
    m = torch.zeros(size, dtype=torch.int32, device="cuda")
    b = torch.full((size, ld), -1, dtype=torch.int16, device="cuda")
    mb = torch.full((size,), -1, dtype=torch.int32, device="cuda")
    ffs.ffs_population_init(inst, 7, 0, 1, size, ld, a)
    rc = _step_noalloc_cabi(lib, inst, prm, 0, 1, size, ld, a, m, b, mb)
    assert rc == ffs.FFS_EUNSUPPORTED
    assert b"fixed array" in lib.ffs_last_error()
    torch.cuda.synchronize()
    assert bool((b == -1).all()) and bool((mb == -1).all())     # nothing was launched
