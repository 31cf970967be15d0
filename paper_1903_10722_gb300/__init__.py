"""GB300 (sm_103a) library for the dual heterogeneous island GA on the
flexible flow shop (Luo & El Baz, arXiv:1903.10722).

This package is a thin ctypes binding over the C ABI declared in
``include/ffs.h``; every function keeps the C name and only marshals
arguments (tensor pointers, the current torch CUDA stream, host arrays).
All computation happens in the CUDA kernels of ``libffs_gb300.so``.  There is
no CPU fallback: if the library cannot be loaded, every call raises.

Device memory and streams come from PyTorch: pass CUDA tensors (int16 rows
of ``ld`` genes, int32 makespans) and calls run on the current stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import _build

_lib = None

FFS_OK, FFS_EINVAL, FFS_ENOMEM, FFS_ECUDA, FFS_EOVERFLOW, FFS_ETIMEOUT, FFS_EDEVICE, FFS_EUNSUPPORTED = range(8)
FFS_PURPOSE_INIT, FFS_PURPOSE_CELLULAR, FFS_PURPOSE_PSEUDO, FFS_PURPOSE_SURROGATE = 1, 2, 3, 16
FFS_PURPOSE_MLP_INIT = 14
FFS_MIG_NONE, FFS_MIG_RING, FFS_MIG_PENETRATION = 0, 1, 2

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64


class FFSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ffs status {status}: {msg}")
        self.status = status


class ffs_params(ctypes.Structure):
    _fields_ = [
        ("seed", _u64), ("cell_pc", _u64), ("cell_pm", _u64), ("pseudo_pc", _u64),
        ("cell_replace_le", _i32), ("pseudo_always", _i32),
        ("migration_mode", _i32), ("migration_gap", _i32),
        ("ring_num", _i64), ("ring_den", _i64), ("theta_num", _i64), ("theta_den", _i64),
        ("decode_chunk", _i32), ("block_threads", _i32), ("decode_variant", _i32),
    ]


# (name, restype, argtypes) of every exported call; the names follow include/ffs.h
_SIGS = [
    ("ffs_last_error", ctypes.c_char_p, []),
    ("ffs_debug_checks", _i32, [ctypes.POINTER(_i32)]),
    ("ffs_debug_check_error", _i32, [ctypes.POINTER(_i32), _i32, _vp]),
    ("ffs_instance_create", _i32, [_i32, _i32, _vp, _vp, ctypes.POINTER(_vp)]),
    ("ffs_instance_create_objective", _i32, [_i32, _i32, _vp, _vp, _vp, _vp, _i32, ctypes.POINTER(_vp)]),
    ("ffs_instance_destroy", _i32, [_vp]),
    ("ffs_assign_instance_create", _i32, [_i32, _i32, _vp, _vp, _vp, _vp, _i32, ctypes.POINTER(_vp)]),
    ("ffs_assign_instance_destroy", _i32, [_vp]),
    ("ffs_assign_eval", _i32, [_vp, _vp, _i64, _i32, _vp, _vp]),
    ("ffs_population_eval", _i32, [_vp, _vp, _i64, _i32, _vp, _vp]),
    ("ffs_population_eval_tuned", _i32, [_vp, _vp, _i64, _i32, _vp, _i32, _i32, _i32, _vp]),
    ("ffs_population_eval_host", _i32, [_vp, _vp, _i64, _i32, _vp, _vp]),
    ("ffs_decode_plan", _i32, [_vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
    ("ffs_philox_draws", _i32, [_u64, _u32, _u32, _u32, _u32, _i32, _i32, _vp, _vp]),
    ("ffs_params_default", None, [ctypes.POINTER(ffs_params)]),
    ("ffs_population_init", _i32, [_vp, _u64, _u32, _i32, _i64, _i32, _vp, _vp]),
    ("ffs_cellular_step", _i32, [_vp, ctypes.POINTER(ffs_params), _u32, _u32, _i32, _i32, _i32,
                                 _vp, _vp, _vp, _vp, _vp]),
    ("ffs_pseudo_scratch_bytes", _i64, [_i32, _i32]),
    ("ffs_pseudo_step", _i32, [_vp, ctypes.POINTER(ffs_params), _u32, _u32, _i32, _i32,
                               _vp, _vp, _vp, _vp, _vp, _vp]),
    ("ffs_pseudo_step_noalloc", _i32, [_vp, ctypes.POINTER(ffs_params), _u32, _u32, _i32, _i32,
                                       _vp, _vp, _vp, _vp, _vp]),
    ("ffs_islands_create", _i32, [_vp, ctypes.POINTER(ffs_params), _i32, _i32, _i32, _i32, _i32,
                                  _vp, ctypes.POINTER(_vp)]),
    ("ffs_islands_destroy", _i32, [_vp]),
    ("ffs_islands_info", _i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("ffs_island_step", _i32, [_vp, _i32, _i32, _vp]),
    ("ffs_migrate", _i32, [_vp, _i32, _vp]),
    ("ffs_islands_get", _i32, [_vp, _i32, _vp, _i32, _vp, _vp]),
    ("ffs_islands_set", _i32, [_vp, _i32, _vp, _i32, _vp, _vp]),
    ("ffs_islands_get_all", _i32, [_vp, _vp, _i32, _vp, _vp]),
    ("ffs_islands_set_all", _i32, [_vp, _vp, _i32, _vp, _vp]),
    ("ffs_islands_best", _i32, [_vp, _vp, _vp, _vp, _vp]),
    ("ffs_islands_decoded", _i32, [_vp, _vp, _vp]),
    ("ffs_islands_stats", _i32, [_vp, _vp, _vp]),
    ("ffs_islands_record_stats", _i32, [_vp, _i32, _vp]),
    ("ffs_islands_stats_history", _i32, [_vp, _vp, _i32, _vp, _vp]),
    ("ffs_batch_create", _i32, [_i32, _vp, _vp, _vp, _vp, ctypes.POINTER(ffs_params), _i32, _i32, _vp,
                                ctypes.POINTER(_vp)]),
    ("ffs_batch_destroy", _i32, [_vp]),
    ("ffs_batch_step", _i32, [_vp, _i32, _vp]),
    ("ffs_batch_autotune", _i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    ("ffs_batch_info", _i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("ffs_batch_get", _i32, [_vp, _i32, _vp, _i32, _vp, _vp]),
    ("ffs_batch_best", _i32, [_vp, _vp, _vp]),
    ("ffs_batch_decoded", _i32, [_vp, _vp, _vp]),
    ("ffs_batch_check", _i32, [_vp, _vp]),
    ("ffs_batch_dry_run", _i32, [_vp, _i32, _vp]),
    ("ffs_gemm_bf16", _i32, [_vp, _i32, _vp, _i32, _vp, _i32, _i32, _i32, _i32, _vp, _vp]),
    ("ffs_mlp_create", _i32, [_i32, _i32, _i32, _i32, ctypes.POINTER(_vp)]),
    ("ffs_mlp_destroy", _i32, [_vp]),
    ("ffs_mlp_input_width", _i32, [_vp]),
    ("ffs_mlp_set_params", _i32, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_float]),
    ("ffs_mlp_get", _i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("ffs_mlp_forward", _i32, [_vp, _vp, _i32, _i32, _vp, _vp]),
    ("ffs_mlp_train_step", _i32, [_vp, _vp, _i32, _vp, _i32, ctypes.c_float, _vp, _vp]),
    ("ffs_mlp_check", _i32, [_vp, _vp]),
    ("ffs_surrogate_params_default", None, [_vp]),
    ("ffs_islands_attach_surrogate", _i32, [_vp, _vp, _vp, _vp]),
    ("ffs_islands_surrogate_last", _i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp]),
    ("ffs_islands_surrogate_last_pseudo", _i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    ("ffs_measure_int_rate", _i32, [_i32, _vp, _vp, _vp]),
    ("ffs_selftest_wait_timeout", _i32, [_i64, _vp, _vp]),
    ("ffs_islands_set_generation", _i32, [_vp, _i64]),
    ("ffs_islands_autotune", _i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    ("ffs_islands_dry_run", _i32, [_vp, _i32, _vp]),
    ("ffs_islands_params", _i32, [_vp, ctypes.POINTER(ffs_params)]),
    ("ffs_assign_population_init", _i32, [_vp, _u64, _u32, _i32, _i64, _i32, _vp, _vp]),
    ("ffs_assign_step_scratch_bytes", _i64, [_i64, _i32]),
    ("ffs_assign_cellular_step", _i32, [_vp, ctypes.POINTER(ffs_params), _u32, _u32, _i32, _i32, _i32,
                                        _vp, _vp, _vp, _vp, _vp, _vp]),
    ("ffs_assign_pseudo_step", _i32, [_vp, ctypes.POINTER(ffs_params), _u32, _u32, _i32, _i32,
                                      _vp, _vp, _vp, _vp, _vp, _vp]),
    ("ffs_mlp_init", _i32, [_vp, _u64, _vp]),
    ("ffs_mlp_adam_steps", _i32, [_vp, _vp]),
    ("ffs_mlp_state_bytes", _i64, [_vp]),
    ("ffs_mlp_save", _i32, [_vp, _vp, _i64, _vp]),
    ("ffs_mlp_load", _i32, [_vp, _vp, _i64, _vp]),
    ("ffs_checkpoint_bytes", _i64, [_vp]),
    ("ffs_checkpoint_save", _i32, [_vp, _vp, _i64, _vp]),
    ("ffs_checkpoint_load", _i32, [_vp, _vp, _i64, _vp]),
    ("ffs_batch_set", _i32, [_vp, _i32, _vp, _i32, _vp, _vp]),
    ("ffs_batch_checkpoint_bytes", _i64, [_vp]),
    ("ffs_batch_checkpoint_save", _i32, [_vp, _vp, _i64, _vp]),
    ("ffs_batch_checkpoint_load", _i32, [_vp, _vp, _i64, _vp]),
]


def library_path() -> str:
    return _build.LIB


def debug_checks_requested() -> bool:
    """FFS_DEBUG_CHECKS=1 in the environment selects the checked library."""
    return os.environ.get("FFS_DEBUG_CHECKS", "0") not in ("", "0")


def load(build_if_missing: bool = True):
    """Load libffs_gb300.so, or libffs_gb300_debug.so when FFS_DEBUG_CHECKS=1
    (building it with nvcc if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    debug = debug_checks_requested()
    path = _build.LIB_DEBUG if debug else _build.LIB
    if build_if_missing and not _build.up_to_date(debug):
        _build.build(debug=debug)
    if not os.path.exists(path):
        raise FFSError(FFS_EUNSUPPORTED, f"CUDA library not built: {path}")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def ffs_debug_checks() -> bool:
    """True when the loaded library is the checked build."""
    v = _i32()
    _check(load().ffs_debug_checks(ctypes.byref(v)))
    return bool(v.value)


def ffs_debug_check_error(reset: bool = False, stream=None) -> int:
    """The checked build's device error word (0: no check failed)."""
    v = _i32()
    _check(load().ffs_debug_check_error(ctypes.byref(v), int(reset), _stream(stream)))
    return v.value


def exported_names() -> list[str]:
    return [s[0] for s in _SIGS]


def _check(rc: int):
    if rc != FFS_OK:
        raise FFSError(rc, load().ffs_last_error().decode(errors="replace"))


def _ptr(x):
    """Device/host address of a torch tensor, numpy array or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def ffs_params_default() -> ffs_params:
    p = ffs_params()
    load().ffs_params_default(ctypes.byref(p))
    return p


def threshold(prob: float) -> int:
    """Bernoulli threshold floor(prob * 2^32) of a probability."""
    return int(prob * 4294967296.0) if prob < 1.0 else 4294967296


# ---------------------------------------------------------------------------
# Instances
# ---------------------------------------------------------------------------
class Instance:
    """Owner of an ffs_instance handle (Section 3 problem tables; with release
    and/or due times the objective WT * total tardiness + C_max)."""

    def __init__(self, n: int, S: int, M, p, release=None, due=None, wt: int = 0):
        import numpy as np
        self.n, self.S = int(n), int(S)
        self.M = np.ascontiguousarray(M, dtype=np.int32)
        self.p = np.ascontiguousarray(p, dtype=np.int32).reshape(self.n, self.S)
        self.release = None if release is None else np.ascontiguousarray(release, dtype=np.int32).reshape(self.n)
        self.due = None if due is None else np.ascontiguousarray(due, dtype=np.int32).reshape(self.n)
        self.wt = int(wt)
        h = _vp()
        _check(load().ffs_instance_create_objective(
            self.n, self.S, self.M.ctypes.data, self.p.ctypes.data,
            None if self.release is None else self.release.ctypes.data,
            None if self.due is None else self.due.ctypes.data, self.wt, ctypes.byref(h)))
        self.handle = h

    @property
    def ld(self) -> int:
        return (self.n + 7) // 8 * 8

    def close(self):
        if getattr(self, "handle", None):
            load().ffs_instance_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ffs_instance_create(n, S, M, p) -> Instance:
    return Instance(n, S, M, p)


def ffs_instance_create_objective(n, S, M, p, release, due, wt) -> Instance:
    return Instance(n, S, M, p, release=release, due=due, wt=wt)


class AssignInstance:
    """Owner of an ffs_assign_instance handle: the paper's genotype (n*S
    machine-assignment genes per row) on unrelated machines, p_u[j][off_s + m]
    (Section 3, P_jsm; Section 4.1)."""

    def __init__(self, n: int, S: int, M, p_u, release=None, due=None, wt: int = 0):
        import numpy as np
        self.n, self.S = int(n), int(S)
        self.M = np.ascontiguousarray(M, dtype=np.int32)
        self.W = int(self.M.sum())
        self.p_u = np.ascontiguousarray(p_u, dtype=np.int32).reshape(self.n, self.W)
        self.release = None if release is None else np.ascontiguousarray(release, dtype=np.int32).reshape(self.n)
        self.due = None if due is None else np.ascontiguousarray(due, dtype=np.int32).reshape(self.n)
        self.wt = int(wt)
        h = _vp()
        _check(load().ffs_assign_instance_create(
            self.n, self.S, self.M.ctypes.data, self.p_u.ctypes.data,
            None if self.release is None else self.release.ctypes.data,
            None if self.due is None else self.due.ctypes.data, self.wt, ctypes.byref(h)))
        self.handle = h

    @property
    def ld(self) -> int:
        return (self.n * self.S + 7) // 8 * 8

    def close(self):
        if getattr(self, "handle", None):
            load().ffs_assign_instance_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ffs_assign_eval(inst: AssignInstance, pop, N: int, ld: int, objective, stream=None):
    _check(load().ffs_assign_eval(inst.handle, _ptr(pop), N, ld, _ptr(objective), _stream(stream)))


def ffs_assign_population_init(inst: AssignInstance, seed, island, kind, N, ld, pop, stream=None):
    _check(load().ffs_assign_population_init(inst.handle, seed, island, kind, N, ld, _ptr(pop), _stream(stream)))


def ffs_assign_step_scratch_bytes(N: int, ld: int) -> int:
    return int(load().ffs_assign_step_scratch_bytes(N, ld))


def ffs_assign_cellular_step(inst: AssignInstance, prm: ffs_params, island, generation, rows, cols, ld, pop_in,
                             obj_in, pop_out, obj_out, scratch, stream=None):
    _check(load().ffs_assign_cellular_step(inst.handle, ctypes.byref(prm), island, generation, rows, cols, ld,
                                           _ptr(pop_in), _ptr(obj_in), _ptr(pop_out), _ptr(obj_out), _ptr(scratch),
                                           _stream(stream)))


def ffs_assign_pseudo_step(inst: AssignInstance, prm: ffs_params, island, generation, size, ld, pop_in, obj_in,
                           pop_out, obj_out, scratch, stream=None):
    _check(load().ffs_assign_pseudo_step(inst.handle, ctypes.byref(prm), island, generation, size, ld,
                                         _ptr(pop_in), _ptr(obj_in), _ptr(pop_out), _ptr(obj_out), _ptr(scratch),
                                         _stream(stream)))


def ffs_population_eval(inst: Instance, pop, N: int, ld: int, makespan, stream=None):
    _check(load().ffs_population_eval(inst.handle, _ptr(pop), N, ld, _ptr(makespan), _stream(stream)))


def ffs_population_eval_tuned(inst: Instance, pop, N, ld, makespan, decode_chunk=0, block_threads=0, variant=0,
                              stream=None):
    _check(load().ffs_population_eval_tuned(inst.handle, _ptr(pop), N, ld, _ptr(makespan),
                                            decode_chunk, block_threads, variant, _stream(stream)))


def ffs_decode_plan(inst: Instance, kernel: int = 0, decode_chunk: int = 0, block_threads: int = 0,
                    variant: int = 0) -> dict:
    """Launch shape of the decoder (kernel 0), the fused cellular kernel (1) or
    the fused decode launch of a dual-island generation (2)."""
    B, T, bps, tm = _i32(), _i32(), _i32(), _i32()
    sm = _i64()
    _check(load().ffs_decode_plan(inst.handle, kernel, decode_chunk, block_threads, variant, ctypes.byref(B),
                                  ctypes.byref(T), ctypes.byref(bps), ctypes.byref(sm), ctypes.byref(tm)))
    return {"chunk": B.value, "threads": T.value, "blocks_per_sm": bps.value, "smem_bytes": sm.value,
            "tmem_cols": tm.value}


def ffs_population_eval_host(inst: Instance, pop, N, ld, makespan, stream=None):
    _check(load().ffs_population_eval_host(inst.handle, _ptr(pop), N, ld, _ptr(makespan), _stream(stream)))


def ffs_philox_draws(seed, purpose, island, generation, cell0, n_cells, n_draws, out, stream=None):
    _check(load().ffs_philox_draws(seed, purpose, island, generation, cell0, n_cells, n_draws, _ptr(out),
                                   _stream(stream)))


def ffs_population_init(inst: Instance, seed, island, kind, N, ld, pop, stream=None):
    _check(load().ffs_population_init(inst.handle, seed, island, kind, N, ld, _ptr(pop), _stream(stream)))


def ffs_cellular_step(inst: Instance, prm: ffs_params, island, generation, rows, cols, ld,
                      pop_in, ms_in, pop_out, ms_out, stream=None):
    _check(load().ffs_cellular_step(inst.handle, ctypes.byref(prm), island, generation, rows, cols, ld,
                                    _ptr(pop_in), _ptr(ms_in), _ptr(pop_out), _ptr(ms_out), _stream(stream)))


def ffs_pseudo_scratch_bytes(size: int, ld: int) -> int:
    return int(load().ffs_pseudo_scratch_bytes(size, ld))


def ffs_pseudo_step(inst: Instance, prm: ffs_params, island, generation, size, ld, pop_in, ms_in,
                    pop_out, ms_out, scratch, stream=None):
    _check(load().ffs_pseudo_step(inst.handle, ctypes.byref(prm), island, generation, size, ld,
                                  _ptr(pop_in), _ptr(ms_in), _ptr(pop_out), _ptr(ms_out), _ptr(scratch),
                                  _stream(stream)))


FFS_NOALLOC_SCRATCH_BYTES = 4 << 20


def ffs_pseudo_step_noalloc(inst: Instance, prm: ffs_params, island, generation, size, ld, pop_in, ms_in,
                            pop_out, ms_out, stream=None):
    """ffs_pseudo_step with the library's fixed scratch array (no allocation)."""
    _check(load().ffs_pseudo_step_noalloc(inst.handle, ctypes.byref(prm), island, generation, size, ld,
                                          _ptr(pop_in), _ptr(ms_in), _ptr(pop_out), _ptr(ms_out),
                                          _stream(stream)))


# ---------------------------------------------------------------------------
# Islands
# ---------------------------------------------------------------------------
class Islands:
    """Owner of an ffs_islands handle (ring order [cell 0, pseudo 0, cell 1, ...])."""

    def __init__(self, inst: Instance, prm: ffs_params, n_cellular: int, rows: int, cols: int,
                 n_pseudo: int, pseudo_size: int, stream=None):
        self.inst = inst
        h = _vp()
        _check(load().ffs_islands_create(inst.handle, ctypes.byref(prm), n_cellular, rows, cols, n_pseudo,
                                         pseudo_size, _stream(stream), ctypes.byref(h)))
        self.handle = h
        n = _i32()
        ld = _i32()
        gen = _i64()
        _check(load().ffs_islands_info(h, ctypes.byref(n), ctypes.byref(ld), ctypes.byref(gen), None, None))
        self.n_islands, self.ld = n.value, ld.value
        sizes = (_i32 * self.n_islands)()
        kinds = (_i32 * self.n_islands)()
        _check(load().ffs_islands_info(h, None, None, None, sizes, kinds))
        self.sizes = list(sizes)
        self.kinds = ["cellular" if k == 0 else "pseudo" for k in kinds]

    def generation(self) -> int:
        g = _i64()
        _check(load().ffs_islands_info(self.handle, None, None, ctypes.byref(g), None, None))
        return g.value

    def close(self):
        if getattr(self, "handle", None):
            load().ffs_islands_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ffs_islands_create(inst, prm, n_cellular, rows, cols, n_pseudo, pseudo_size, stream=None) -> Islands:
    return Islands(inst, prm, n_cellular, rows, cols, n_pseudo, pseudo_size, stream)


def ffs_island_step(isl: Islands, island: int, n_generations: int, stream=None):
    _check(load().ffs_island_step(isl.handle, island, n_generations, _stream(stream)))


def ffs_migrate(isl: Islands, mode: int, stream=None):
    _check(load().ffs_migrate(isl.handle, mode, _stream(stream)))


def ffs_islands_get(isl: Islands, island: int, pop, ld_out: int, makespan, stream=None):
    _check(load().ffs_islands_get(isl.handle, island, _ptr(pop), ld_out, _ptr(makespan), _stream(stream)))


def ffs_islands_set(isl: Islands, island: int, pop, ld_in: int, makespan, stream=None):
    _check(load().ffs_islands_set(isl.handle, island, _ptr(pop), ld_in, _ptr(makespan), _stream(stream)))


def ffs_islands_get_all(isl: Islands, pop, ld_out: int, makespan, stream=None):
    _check(load().ffs_islands_get_all(isl.handle, _ptr(pop), ld_out, _ptr(makespan), _stream(stream)))


def ffs_islands_set_all(isl: Islands, pop, ld_in: int, makespan, stream=None):
    _check(load().ffs_islands_set_all(isl.handle, _ptr(pop), ld_in, _ptr(makespan), _stream(stream)))


def ffs_islands_best(isl: Islands, stream=None):
    m, i, r = _i32(), _i32(), _i32()
    _check(load().ffs_islands_best(isl.handle, ctypes.byref(m), ctypes.byref(i), ctypes.byref(r),
                                   _stream(stream)))
    return m.value, i.value, r.value


FFS_STAT_WORDS = 8
STAT_FIELDS = ("generation", "best", "worst", "sum", "valid", "best_so_far", "migrations", "migrated_rows")


def ffs_islands_stats(isl: Islands, stream=None):
    """The current generation's metrics of every island: int64 [n_islands][8]
    (fields in STAT_FIELDS order)."""
    import numpy as np
    out = np.zeros((isl.n_islands, FFS_STAT_WORDS), dtype=np.int64)
    _check(load().ffs_islands_stats(isl.handle, out.ctypes.data, _stream(stream)))
    return out


def ffs_islands_record_stats(isl: Islands, capacity: int, stream=None):
    _check(load().ffs_islands_record_stats(isl.handle, capacity, _stream(stream)))


def ffs_islands_stats_history(isl: Islands, stream=None):
    """The recorded metrics, oldest generation first: int64
    [records][n_islands][8]."""
    import numpy as np
    n = _i32()
    _check(load().ffs_islands_stats_history(isl.handle, None, 0, ctypes.byref(n), _stream(stream)))
    out = np.zeros((n.value, isl.n_islands, FFS_STAT_WORDS), dtype=np.int64)
    if n.value:
        _check(load().ffs_islands_stats_history(isl.handle, out.ctypes.data, n.value, ctypes.byref(n),
                                                _stream(stream)))
    return out


def ffs_islands_decoded(isl: Islands, stream=None) -> int:
    c = _i64()
    _check(load().ffs_islands_decoded(isl.handle, ctypes.byref(c), _stream(stream)))
    return c.value


def ffs_checkpoint_save(isl: Islands, stream=None):
    """The islands' whole state as a host byte array (numpy uint8)."""
    import numpy as np
    n = int(load().ffs_checkpoint_bytes(isl.handle))
    if n < 0:
        _check(FFS_EINVAL)
    buf = np.zeros(n, dtype=np.uint8)
    _check(load().ffs_checkpoint_save(isl.handle, buf.ctypes.data, n, _stream(stream)))
    return buf


def ffs_checkpoint_load(isl: Islands, blob, stream=None):
    import numpy as np
    b = np.ascontiguousarray(blob, dtype=np.uint8)
    _check(load().ffs_checkpoint_load(isl.handle, b.ctypes.data, b.size, _stream(stream)))


def island_tensors(isl: Islands, island: int):
    """(pop int16 [N][n], makespans int32 [N]) of one island, as CUDA tensors."""
    import torch
    N = isl.sizes[island]
    pop = torch.empty((N, isl.inst.n), dtype=torch.int16, device="cuda")
    ms = torch.empty(N, dtype=torch.int32, device="cuda")
    ffs_islands_get(isl, island, pop, isl.inst.n, ms)
    return pop, ms


# ---------------------------------------------------------------------------
# Batch of uneven instances
# ---------------------------------------------------------------------------
class Batch:
    """Owner of an ffs_batch handle: one cellular island per instance."""

    def __init__(self, specs, prm: ffs_params, rows: int, cols: int, stream=None):
        import numpy as np
        self.specs = specs
        self.count = len(specs)
        self.rows, self.cols = rows, cols
        n = np.array([s.n for s in specs], dtype=np.int32)
        S = np.array([s.S for s in specs], dtype=np.int32)
        M = np.ascontiguousarray(np.concatenate([np.asarray(s.M, dtype=np.int32) for s in specs]))
        p = np.ascontiguousarray(np.concatenate([np.asarray(s.p, dtype=np.int32).ravel() for s in specs]))
        h = _vp()
        _check(load().ffs_batch_create(self.count, n.ctypes.data, S.ctypes.data, M.ctypes.data, p.ctypes.data,
                                       ctypes.byref(prm), rows, cols, _stream(stream), ctypes.byref(h)))
        self.handle = h

    def info(self) -> dict:
        c, t, b, bps, v = _i32(), _i32(), _i32(), _i32(), _i32()
        g = _i64()
        _check(load().ffs_batch_info(self.handle, ctypes.byref(c), ctypes.byref(g), ctypes.byref(t),
                                     ctypes.byref(b), ctypes.byref(bps), ctypes.byref(v)))
        return {"count": c.value, "generation": g.value, "threads": t.value, "chunk": b.value,
                "blocks_per_sm": bps.value, "variant": v.value}

    def close(self):
        if getattr(self, "handle", None):
            load().ffs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ffs_batch_step(b: Batch, n_generations: int, stream=None):
    _check(load().ffs_batch_step(b.handle, n_generations, _stream(stream)))


def ffs_batch_autotune(b: Batch, repeats: int = 2, stream=None) -> dict:
    t, c = _i32(), _i32()
    ms = ctypes.c_float()
    _check(load().ffs_batch_autotune(b.handle, repeats, _stream(stream), ctypes.byref(t), ctypes.byref(c),
                                     ctypes.byref(ms)))
    return {"threads": t.value, "chunk": c.value, "ms": ms.value}


def ffs_batch_get(b: Batch, instance: int, pop, ld_out: int, makespan, stream=None):
    _check(load().ffs_batch_get(b.handle, instance, _ptr(pop), ld_out, _ptr(makespan), _stream(stream)))


def ffs_batch_set(b: Batch, instance: int, pop, ld_in: int, makespan, stream=None):
    _check(load().ffs_batch_set(b.handle, instance, _ptr(pop), ld_in, _ptr(makespan), _stream(stream)))


def ffs_batch_checkpoint_save(b: Batch, stream=None):
    """The batch's whole state as a host byte array (numpy uint8)."""
    import numpy as np
    n = int(load().ffs_batch_checkpoint_bytes(b.handle))
    if n < 0:
        _check(FFS_EINVAL)
    buf = np.zeros(n, dtype=np.uint8)
    _check(load().ffs_batch_checkpoint_save(b.handle, buf.ctypes.data, n, _stream(stream)))
    return buf


def ffs_batch_checkpoint_load(b: Batch, blob, stream=None):
    import numpy as np
    buf = np.ascontiguousarray(blob, dtype=np.uint8)
    _check(load().ffs_batch_checkpoint_load(b.handle, buf.ctypes.data, buf.size, _stream(stream)))


def ffs_batch_best(b: Batch, stream=None):
    import numpy as np
    out = np.zeros(b.count, dtype=np.int32)
    _check(load().ffs_batch_best(b.handle, out.ctypes.data, _stream(stream)))
    return out


def ffs_batch_decoded(b: Batch, stream=None) -> int:
    c = _i64()
    _check(load().ffs_batch_decoded(b.handle, ctypes.byref(c), _stream(stream)))
    return c.value


def ffs_batch_check(b: Batch, stream=None):
    _check(load().ffs_batch_check(b.handle, _stream(stream)))


def ffs_batch_dry_run(b: Batch, kind: int, stream=None):
    _check(load().ffs_batch_dry_run(b.handle, kind, _stream(stream)))


def batch_tensors(b: Batch, instance: int):
    """(pop int16 [cells][n], makespans int32 [cells]) of one instance, as CUDA tensors."""
    import torch
    n = b.specs[instance].n
    cells = b.rows * b.cols
    pop = torch.empty((cells, n), dtype=torch.int16, device="cuda")
    ms = torch.empty(cells, dtype=torch.int32, device="cuda")
    ffs_batch_get(b, instance, pop, n, ms)
    return pop, ms


# ---------------------------------------------------------------------------
# Surrogate network (tensor-core GEMM and MLP)
# ---------------------------------------------------------------------------
def ffs_gemm_bf16(A, lda: int, B, ldb: int, D, ldd: int, M: int, N: int, K: int, err, stream=None):
    """D = A B^T on the tensor cores (A, B bf16 tensors, D fp32, err int32 device scalar)."""
    _check(load().ffs_gemm_bf16(_ptr(A), lda, _ptr(B), ldb, _ptr(D), ldd, M, N, K, _ptr(err), _stream(stream)))


class MLP:
    """Owner of an ffs_mlp handle."""

    def __init__(self, in_dim: int, h1: int, h2: int, max_batch: int):
        h = _vp()
        _check(load().ffs_mlp_create(in_dim, h1, h2, max_batch, ctypes.byref(h)))
        self.handle = h
        self.in_dim, self.h1, self.h2, self.max_batch = in_dim, h1, h2, max_batch
        self.width = int(load().ffs_mlp_input_width(h))

    def set_params(self, p: dict):
        import numpy as np
        arrs = [np.ascontiguousarray(p[k], dtype=np.float32) for k in ("W1", "b1", "W2", "b2", "w3")]
        _check(load().ffs_mlp_set_params(self.handle, *[a.ctypes.data for a in arrs], float(p["b3"])))

    def get(self, grads: bool = False, which: int | None = None) -> dict:
        """Parameters (which 0), last gradients (1, or grads=True), Adam's
        first (2) or second (3) moments, as host float32 arrays."""
        import numpy as np
        w = int(grads) if which is None else int(which)
        out = {"W1": np.zeros((self.h1, self.in_dim), np.float32), "b1": np.zeros(self.h1, np.float32),
               "W2": np.zeros((self.h2, self.h1), np.float32), "b2": np.zeros(self.h2, np.float32),
               "w3": np.zeros(self.h2, np.float32)}
        b3 = ctypes.c_float()
        _check(load().ffs_mlp_get(self.handle, w, *[out[k].ctypes.data for k in ("W1", "b1", "W2", "b2", "w3")],
                                  ctypes.byref(b3)))
        out["b3"] = np.float32(b3.value)
        return out

    def init(self, seed: int, stream=None):
        """He-uniform weights drawn from Philox (ffs_mlp_init), biases 0."""
        _check(load().ffs_mlp_init(self.handle, seed, _stream(stream)))

    def adam_steps(self) -> int:
        t = _i64()
        _check(load().ffs_mlp_adam_steps(self.handle, ctypes.byref(t)))
        return t.value

    def save(self, stream=None):
        import numpy as np
        n = int(load().ffs_mlp_state_bytes(self.handle))
        buf = np.zeros(n, dtype=np.uint8)
        _check(load().ffs_mlp_save(self.handle, buf.ctypes.data, n, _stream(stream)))
        return buf

    def load_state(self, blob, stream=None):
        import numpy as np
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(load().ffs_mlp_load(self.handle, b.ctypes.data, b.size, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().ffs_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ffs_mlp_forward(m: MLP, x, ldx: int, B: int, y, stream=None):
    _check(load().ffs_mlp_forward(m.handle, _ptr(x), ldx, B, _ptr(y), _stream(stream)))


def ffs_mlp_train_step(m: MLP, x, ldx: int, target, B: int, lr: float, loss=None, stream=None):
    _check(load().ffs_mlp_train_step(m.handle, _ptr(x), ldx, _ptr(target), B, lr, _ptr(loss), _stream(stream)))


def ffs_mlp_check(m: MLP, stream=None):
    _check(load().ffs_mlp_check(m.handle, _stream(stream)))


class ffs_surrogate_params(ctypes.Structure):
    _fields_ = [("candidates", _i32), ("train_every", _i32), ("train_steps", _i32), ("train_batch", _i32),
                ("ring_capacity", _i32), ("warmup_generations", _i32), ("lr", ctypes.c_float),
                ("overlap", _i32), ("screen_pseudo", _i32)]


def ffs_surrogate_params_default() -> ffs_surrogate_params:
    p = ffs_surrogate_params()
    load().ffs_surrogate_params_default(ctypes.byref(p))
    return p


def ffs_islands_attach_surrogate(isl: Islands, m: MLP, sp: ffs_surrogate_params, stream=None):
    _check(load().ffs_islands_attach_surrogate(isl.handle, m.handle, ctypes.byref(sp), _stream(stream)))
    isl.surrogate = m


def ffs_islands_surrogate_last(isl: Islands, scores=None, chosen=None, loss=None, candidates=None, ld_out: int = 0,
                               stream=None) -> int:
    pairs = _i64()
    _check(load().ffs_islands_surrogate_last(isl.handle, _ptr(scores), _ptr(chosen), _ptr(loss), ctypes.byref(pairs),
                                             _ptr(candidates), ld_out, _stream(stream)))
    return pairs.value


def ffs_islands_surrogate_last_pseudo(isl: Islands, scores=None, chosen=None, candidates=None, ld_out: int = 0,
                                      stream=None):
    _check(load().ffs_islands_surrogate_last_pseudo(isl.handle, _ptr(scores), _ptr(chosen), _ptr(candidates), ld_out,
                                                    _stream(stream)))


def ffs_measure_int_rate(kind: int, stream=None) -> dict:
    rate = ctypes.c_double()
    ms = ctypes.c_float()
    _check(load().ffs_measure_int_rate(kind, ctypes.byref(rate), ctypes.byref(ms), _stream(stream)))
    return {"lane_ops_per_s": rate.value, "ms": ms.value}


def ffs_selftest_wait_timeout(limit_ns: int, stream=None):
    """(status code of the call, device status word)."""
    st = _i32()
    rc = load().ffs_selftest_wait_timeout(limit_ns, ctypes.byref(st), _stream(stream))
    return rc, st.value


def ffs_islands_set_generation(isl: Islands, generation: int):
    _check(load().ffs_islands_set_generation(isl.handle, generation))


def ffs_islands_autotune(isl: Islands, repeats: int = 2, stream=None) -> dict:
    t, c = _i32(), _i32()
    ms = ctypes.c_float()
    _check(load().ffs_islands_autotune(isl.handle, repeats, _stream(stream), ctypes.byref(t), ctypes.byref(c),
                                       ctypes.byref(ms)))
    return {"threads": t.value, "chunk": c.value, "ms": ms.value}


def ffs_islands_dry_run(isl: Islands, kind: int, stream=None):
    _check(load().ffs_islands_dry_run(isl.handle, kind, _stream(stream)))


def ffs_islands_params(isl: Islands) -> ffs_params:
    p = ffs_params()
    _check(load().ffs_islands_params(isl.handle, ctypes.byref(p)))
    return p
