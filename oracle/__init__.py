"""CPU oracle for the FFS island GA hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline arm of
``bench.py`` may import this package.  It is the independent, slow,
single-threaded statement of what the GPU library computes (Luo & El Baz,
arXiv:1903.10722, Sections 3, 4.1-4.3 and 5), written in plain C
(``ffs_oracle.c``) plus plain numpy, and it shares no code with the CUDA path.

The C part is compiled with gcc on first use (or by ``build()``) into
``oracle/_build/libffs_oracle.so`` and driven through ctypes; everything here
is argument marshalling around it, except the surrogate network
(``oracle.mlp``), which is plain numpy in float64.

Parity status: see the header of ``ffs_oracle.c``.  The decoder, operators,
Philox and migration formulas are pinned by ``tests/test_oracle_*.py``; the
multi-generation GA trajectory itself is "parity unpinned" (the paper prints
none).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffs_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libffs_oracle.so")
_lock = threading.Lock()
_lib = None

PURPOSE_INIT = 1
PURPOSE_CELLULAR = 2
PURPOSE_PSEUDO = 3
PURPOSE_SURROGATE = 16   # + candidate index

_i16p = ctypes.POINTER(ctypes.c_int16)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("cell_pc", ctypes.c_uint64),
        ("cell_pm", ctypes.c_uint64),
        ("pseudo_pc", ctypes.c_uint64),
        ("cell_replace_le", ctypes.c_int32),
        ("pseudo_always", ctypes.c_int32),
        ("obj", ctypes.c_void_p),
    ]


class _Objective(ctypes.Structure):
    _fields_ = [
        ("release", ctypes.POINTER(ctypes.c_int32)),
        ("due", ctypes.POINTER(ctypes.c_int32)),
        ("wt", ctypes.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile ffs_oracle.c with gcc (plain -O2, no vectorisation flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.orc_philox4x32_10.restype = None
        lib.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.orc_draw.restype = ctypes.c_uint32
        lib.orc_uniform.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.orc_uniform.restype = ctypes.c_uint32
        lib.orc_bernoulli.argtypes = [ctypes.c_uint32, ctypes.c_uint64]
        lib.orc_bernoulli.restype = ctypes.c_int
        lib.orc_decode.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i16p, _i64p]
        lib.orc_decode.restype = ctypes.c_int64
        lib.orc_decode_obj.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, ctypes.c_void_p, _i16p,
                                       _i64p]
        lib.orc_decode_obj.restype = ctypes.c_int64
        lib.orc_eval_population_obj.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, ctypes.c_void_p,
                                                _i16p, ctypes.c_int64, ctypes.c_int64, _i64p]
        lib.orc_eval_population_obj.restype = None
        lib.orc_bruteforce_obj.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, ctypes.c_void_p, _i64p,
                                           _i16p]
        lib.orc_bruteforce_obj.restype = ctypes.c_int64
        lib.orc_decode_assign.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, ctypes.c_void_p, _i16p,
                                          _i64p]
        lib.orc_decode_assign.restype = ctypes.c_int64
        lib.orc_eval_population_assign.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, ctypes.c_void_p,
                                                   _i16p, ctypes.c_int64, ctypes.c_int64, _i64p]
        lib.orc_eval_population_assign.restype = None
        lib.orc_assign_init_row.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32,
                                            ctypes.c_int32, _i32p, _i16p]
        lib.orc_assign_init_row.restype = None
        lib.orc_assign_init_pair.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, _i32p, _i16p, _i16p]
        lib.orc_assign_init_pair.restype = None
        lib.orc_assign_complement.argtypes = [ctypes.c_int32, ctypes.c_int32]
        lib.orc_assign_complement.restype = ctypes.c_int32
        lib.orc_two_point.argtypes = [ctypes.c_int32, _i16p, _i16p, ctypes.c_int32, ctypes.c_int32, _i16p]
        lib.orc_two_point.restype = None
        lib.orc_assign_reassign.argtypes = [_i16p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32]
        lib.orc_assign_reassign.restype = None
        lib.orc_assign_cellular_child.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, ctypes.c_int32,
                                                  ctypes.c_int32, ctypes.c_int32, _u32p, ctypes.POINTER(_Params),
                                                  _i16p, ctypes.c_int64, _i64p, _i16p]
        lib.orc_assign_cellular_child.restype = None
        agen = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, ctypes.POINTER(_Params), ctypes.c_uint32,
                ctypes.c_uint32]
        lib.orc_assign_cellular_generation.argtypes = agen + [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _i16p,
                                                              _i64p, _i16p, _i64p]
        lib.orc_assign_cellular_generation.restype = ctypes.c_int64
        lib.orc_assign_pseudo_generation.argtypes = agen + [ctypes.c_int32, ctypes.c_int64, _i16p, _i64p, _i16p,
                                                            _i64p]
        lib.orc_assign_pseudo_generation.restype = ctypes.c_int64
        lib.orc_eval_population.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                            _i16p, ctypes.c_int64, ctypes.c_int64, _i64p]
        lib.orc_eval_population.restype = None
        lib.orc_bruteforce.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i64p, _i16p]
        lib.orc_bruteforce.restype = ctypes.c_int64
        lib.orc_init_chromosome.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_int32, _i16p]
        lib.orc_init_chromosome.restype = None
        lib.orc_order_crossover.argtypes = [ctypes.c_int32, _i16p, _i16p, ctypes.c_int32,
                                            ctypes.c_int32, _i16p]
        lib.orc_order_crossover.restype = None
        lib.orc_neighbours.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p]
        lib.orc_neighbours.restype = None
        lib.orc_cellular_child.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, _u32p, ctypes.POINTER(_Params),
                                           _i16p, ctypes.c_int64, _i64p, _i16p, _i32p]
        lib.orc_cellular_child.restype = None
        gen_args = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, ctypes.POINTER(_Params),
                    ctypes.c_uint32, ctypes.c_uint32]
        lib.orc_cellular_generation.argtypes = gen_args + [ctypes.c_int32, ctypes.c_int32,
                                                           ctypes.c_int64, _i16p, _i64p, _i16p, _i64p]
        lib.orc_cellular_generation.restype = ctypes.c_int64
        lib.orc_pseudo_generation.argtypes = gen_args + [ctypes.c_int32, ctypes.c_int64,
                                                         _i16p, _i64p, _i16p, _i64p]
        lib.orc_pseudo_generation.restype = ctypes.c_int64
        lib.orc_cellular_generation_range.argtypes = lib.orc_cellular_generation.argtypes + [ctypes.c_int32,
                                                                                             ctypes.c_int32]
        lib.orc_cellular_generation_range.restype = ctypes.c_int64
        lib.orc_pseudo_generation_range.argtypes = lib.orc_pseudo_generation.argtypes + [ctypes.c_int32,
                                                                                         ctypes.c_int32]
        lib.orc_pseudo_generation_range.restype = ctypes.c_int64
        lib.orc_screened_cellular_generation.argtypes = gen_args + [
            ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _i16p, _i64p, _i16p, _i64p,
            ctypes.POINTER(ctypes.c_float), ctypes.c_int32, _i32p, _i16p]
        lib.orc_screened_cellular_generation.restype = ctypes.c_int64
        lib.orc_screened_pseudo_generation.argtypes = gen_args + [
            ctypes.c_int32, ctypes.c_int64, _i16p, _i64p, _i16p, _i64p,
            ctypes.POINTER(ctypes.c_float), ctypes.c_int32, _i32p, _i16p]
        lib.orc_screened_pseudo_generation.restype = ctypes.c_int64
        lib.orc_family_best2.argtypes = [_i64p, _i32p]
        lib.orc_family_best2.restype = None
        lib.orc_init_pseudo_pair.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                             ctypes.c_int32, _i16p, _i16p]
        lib.orc_init_pseudo_pair.restype = None
        lib.orc_rank_island.argtypes = [ctypes.c_int32, _i64p, _i32p]
        lib.orc_rank_island.restype = None
        lib.orc_migrate_ring.argtypes = [ctypes.c_int32, _i32p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.POINTER(_i16p), ctypes.POINTER(_i64p),
                                         ctypes.c_int64, ctypes.c_int64]
        lib.orc_migrate_ring.restype = None
        lib.orc_penetration_count.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int64, ctypes.c_int64]
        lib.orc_penetration_count.restype = ctypes.c_int64
        lib.orc_migrate_penetration.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                                ctypes.c_int32, _i16p, _i64p, _i16p, _i64p,
                                                ctypes.c_int64, ctypes.c_int64]
        lib.orc_migrate_penetration.restype = ctypes.c_int64
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ---------------------------------------------------------------------------
# Problem instance (Section 3): n jobs, S stages, M_s identical machines,
# processing times p[j][s]; optionally release times R_j, due times D_j and
# the tardiness weight WT (objective WT * sum_j max(0, C_j - D_j) + C_max).
# ---------------------------------------------------------------------------
@dataclass
class Instance:
    n: int
    S: int
    M: np.ndarray   # int32 [S]
    p: np.ndarray   # int32 [n][S], job-major
    release: np.ndarray | None = None   # int32 [n]
    due: np.ndarray | None = None       # int32 [n]
    wt: int = 0

    def __post_init__(self):
        self.M = np.ascontiguousarray(self.M, dtype=np.int32)
        self.p = np.ascontiguousarray(self.p, dtype=np.int32).reshape(self.n, self.S)
        self._obj = None
        if self.release is not None or self.due is not None:
            if self.release is not None:
                self.release = np.ascontiguousarray(self.release, dtype=np.int32).reshape(self.n)
            if self.due is not None:
                self.due = np.ascontiguousarray(self.due, dtype=np.int32).reshape(self.n)
            self._obj = _Objective(
                _ptr(self.release, ctypes.c_int32) if self.release is not None else None,
                _ptr(self.due, ctypes.c_int32) if self.due is not None else None, int(self.wt))

    def obj_addr(self):
        """Address of the C objective record (None: the makespan alone)."""
        return ctypes.addressof(self._obj) if self._obj is not None else None


def lower_bound(inst: Instance) -> int:
    """max(largest job total, largest per-stage ceil(load / M_s))."""
    job = int(inst.p.sum(axis=1).max())
    stage = max(-(-int(inst.p[:, s].sum()) // int(inst.M[s])) for s in range(inst.S))
    return max(job, stage)


# ---------------------------------------------------------------------------
# Philox4x32-10 and the draw conventions
# ---------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                          _ptr(out, ctypes.c_uint32))
    return out


def draw(seed, purpose, island, generation, cell, d) -> int:
    return int(_load().orc_draw(seed, purpose, island, generation, cell, d))


def uniform(x: int, k: int) -> int:
    return int(_load().orc_uniform(x, k))


def bernoulli(x: int, threshold: int) -> bool:
    return bool(_load().orc_bernoulli(x, threshold))


def threshold(prob: float) -> int:
    """floor(prob * 2^32), the Bernoulli threshold of a probability."""
    return int(np.floor(prob * 4294967296.0))


# ---------------------------------------------------------------------------
# Decoder
# ---------------------------------------------------------------------------
def decode(inst: Instance, perm, gantt: bool = False):
    """The instance's objective (the makespan without due times) of one job
    order; with gantt, also its (stage, job, machine, start, end) records."""
    lib = _load()
    perm = np.ascontiguousarray(perm, dtype=np.int16)
    g = np.zeros((inst.n * inst.S, 5), dtype=np.int64) if gantt else None
    v = lib.orc_decode_obj(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32), _ptr(inst.p, ctypes.c_int32),
                           inst.obj_addr(), _ptr(perm, ctypes.c_int16), _ptr(g, ctypes.c_int64) if gantt else None)
    return (int(v), g) if gantt else int(v)


def eval_population(inst: Instance, pop: np.ndarray) -> np.ndarray:
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    N, ld = pop.shape
    out = np.zeros(N, dtype=np.int64)
    lib.orc_eval_population_obj(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32), _ptr(inst.p, ctypes.c_int32),
                                inst.obj_addr(), _ptr(pop, ctypes.c_int16), N, ld, _ptr(out, ctypes.c_int64))
    return out


def eval_population_threads(inst: Instance, pop: np.ndarray, pool, parts: int) -> np.ndarray:
    """eval_population with the rows split into `parts` ranges on a thread pool."""
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    chunks = [(a, b) for a, b in _split(pop.shape[0], parts) if b > a]
    return np.concatenate([r for r in pool.map(lambda ab: eval_population(inst, pop[ab[0]:ab[1]]), chunks)])


class AssignInstance:
    """An instance with unrelated machines for the paper's genotype (Section
    3, P_jsm; Section 4.1): p_u[j][off_s + m] = time of job j at stage s on
    machine m, off_s = M_0 + ... + M_{s-1}; optional release / due times and
    WT as in Instance."""

    def __init__(self, n, S, M, p_u, release=None, due=None, wt=0):
        self.n, self.S, self.wt = int(n), int(S), int(wt)
        self.M = np.ascontiguousarray(M, dtype=np.int32)
        self.W = int(self.M.sum())
        self.p_u = np.ascontiguousarray(p_u, dtype=np.int32).reshape(self.n, self.W)
        self.release = None if release is None else np.ascontiguousarray(release, dtype=np.int32).reshape(self.n)
        self.due = None if due is None else np.ascontiguousarray(due, dtype=np.int32).reshape(self.n)
        self._obj = None
        if self.release is not None or self.due is not None:
            self._obj = _Objective(
                _ptr(self.release, ctypes.c_int32) if self.release is not None else None,
                _ptr(self.due, ctypes.c_int32) if self.due is not None else None, self.wt)

    def obj_addr(self):
        return ctypes.addressof(self._obj) if self._obj is not None else None


def decode_assign(inst: AssignInstance, genes, gantt: bool = False):
    """Objective of one machine-assignment string (n*S genes, gene j*S + s =
    machine of job j at stage s; -1 if a gene is out of range); with gantt,
    also the (stage, job, machine, start, end) records."""
    lib = _load()
    genes = np.ascontiguousarray(genes, dtype=np.int16)
    g = np.zeros((inst.n * inst.S, 5), dtype=np.int64) if gantt else None
    v = lib.orc_decode_assign(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32), _ptr(inst.p_u, ctypes.c_int32),
                              inst.obj_addr(), _ptr(genes, ctypes.c_int16),
                              _ptr(g, ctypes.c_int64) if gantt else None)
    return (int(v), g) if gantt else int(v)


def eval_population_assign(inst: AssignInstance, pop: np.ndarray) -> np.ndarray:
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    N, ld = pop.shape
    out = np.zeros(N, dtype=np.int64)
    lib.orc_eval_population_assign(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32), _ptr(inst.p_u, ctypes.c_int32),
                                   inst.obj_addr(), _ptr(pop, ctypes.c_int16), N, ld, _ptr(out, ctypes.c_int64))
    return out


def bruteforce(inst: Instance):
    """(optimum, worst, an optimal order) over all n! orders, n <= 10."""
    assert inst.n <= 10
    lib = _load()
    worst = ctypes.c_int64(0)
    bp = np.zeros(inst.n, dtype=np.int16)
    best = lib.orc_bruteforce_obj(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32), _ptr(inst.p, ctypes.c_int32),
                                  inst.obj_addr(), ctypes.byref(worst), _ptr(bp, ctypes.c_int16))
    return int(best), int(worst.value), bp


# ---------------------------------------------------------------------------
# Operators
# ---------------------------------------------------------------------------
def init_chromosome(seed: int, island: int, cell: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int16)
    _load().orc_init_chromosome(seed, island, cell, n, _ptr(out, ctypes.c_int16))
    return out


def init_pseudo_pair(seed: int, island: int, k: int, n: int):
    a = np.zeros(n, dtype=np.int16)
    b = np.zeros(n, dtype=np.int16)
    _load().orc_init_pseudo_pair(seed, island, k, n, _ptr(a, ctypes.c_int16), _ptr(b, ctypes.c_int16))
    return a, b


def order_crossover(p1, p2, l: int, r: int) -> np.ndarray:
    p1 = np.ascontiguousarray(p1, dtype=np.int16)
    p2 = np.ascontiguousarray(p2, dtype=np.int16)
    out = np.zeros_like(p1)
    _load().orc_order_crossover(len(p1), _ptr(p1, ctypes.c_int16), _ptr(p2, ctypes.c_int16), l, r,
                                _ptr(out, ctypes.c_int16))
    return out


def neighbours(rows: int, cols: int, c: int) -> list:
    out = np.zeros(5, dtype=np.int32)
    _load().orc_neighbours(rows, cols, c, _ptr(out, ctypes.c_int32))
    return out.tolist()


@dataclass
class Params:
    """GA parameters; defaults are the paper's Section 5 values."""
    seed: int = 7
    cell_pc: float = 1.00
    cell_pm: float = 0.05
    pseudo_pc: float = 0.75
    cell_replace_le: bool = False
    pseudo_always: bool = False

    def _c(self, inst: Instance | None = None) -> _Params:
        return _Params(self.seed, threshold(self.cell_pc), threshold(self.cell_pm),
                       threshold(self.pseudo_pc), int(self.cell_replace_le), int(self.pseudo_always),
                       inst.obj_addr() if inst is not None else None)


def cellular_child(inst: Instance, prm: Params, rows: int, cols: int, c: int, x,
                   pop: np.ndarray, ms: np.ndarray):
    """The child of cell c given its ten draws x (no evaluation)."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    child = np.zeros(inst.n, dtype=np.int16)
    parents = np.zeros(2, dtype=np.int32)
    cp = prm._c(inst)
    _load().orc_cellular_child(inst.n, rows, cols, c, _ptr(x, ctypes.c_uint32), ctypes.byref(cp),
                               _ptr(pop, ctypes.c_int16), pop.shape[1], _ptr(ms, ctypes.c_int64),
                               _ptr(child, ctypes.c_int16), _ptr(parents, ctypes.c_int32))
    return child, parents.tolist()


def cellular_generation(inst: Instance, prm: Params, island: int, generation: int,
                        rows: int, cols: int, pop: np.ndarray, ms: np.ndarray):
    """One synchronous cellular generation; returns (new pop, new makespans, #decoded)."""
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    out = np.zeros_like(pop)
    out_ms = np.zeros_like(ms)
    cp = prm._c(inst)
    k = lib.orc_cellular_generation(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32),
                                    _ptr(inst.p, ctypes.c_int32), ctypes.byref(cp), island, generation,
                                    rows, cols, pop.shape[1], _ptr(pop, ctypes.c_int16),
                                    _ptr(ms, ctypes.c_int64), _ptr(out, ctypes.c_int16),
                                    _ptr(out_ms, ctypes.c_int64))
    return out, out_ms, int(k)


def _split(total: int, parts: int):
    parts = max(1, min(parts, total))
    edges = [total * i // parts for i in range(parts + 1)]
    return [(edges[i], edges[i + 1]) for i in range(parts)]


def cellular_generation_threads(inst: Instance, prm: Params, island: int, generation: int, rows: int, cols: int,
                                pop: np.ndarray, ms: np.ndarray, pool, parts: int):
    """cellular_generation with the cells split into `parts` ranges run on a
    thread pool (the C calls release the GIL); the same result."""
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    out = np.zeros_like(pop)
    out_ms = np.zeros_like(ms)
    cp = prm._c(inst)

    def run(r):
        return lib.orc_cellular_generation_range(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32),
                                                 _ptr(inst.p, ctypes.c_int32), ctypes.byref(cp), island, generation,
                                                 rows, cols, pop.shape[1], _ptr(pop, ctypes.c_int16),
                                                 _ptr(ms, ctypes.c_int64), _ptr(out, ctypes.c_int16),
                                                 _ptr(out_ms, ctypes.c_int64), r[0], r[1])
    k = sum(pool.map(run, _split(rows * cols, parts)))
    return out, out_ms, int(k)


def pseudo_generation_threads(inst: Instance, prm: Params, island: int, generation: int, pop: np.ndarray,
                              ms: np.ndarray, pool, parts: int):
    """pseudo_generation with the pairs split into `parts` ranges on a thread pool."""
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    out = np.zeros_like(pop)
    out_ms = np.zeros_like(ms)
    cp = prm._c(inst)

    def run(r):
        return lib.orc_pseudo_generation_range(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32),
                                               _ptr(inst.p, ctypes.c_int32), ctypes.byref(cp), island, generation,
                                               pop.shape[0], pop.shape[1], _ptr(pop, ctypes.c_int16),
                                               _ptr(ms, ctypes.c_int64), _ptr(out, ctypes.c_int16),
                                               _ptr(out_ms, ctypes.c_int64), r[0], r[1])
    k = sum(pool.map(run, _split(pop.shape[0] // 2, parts)))
    return out, out_ms, int(k)


def screened_cellular_generation(inst: Instance, prm: Params, island: int, generation: int, rows: int,
                                 cols: int, pop: np.ndarray, ms: np.ndarray, scores: np.ndarray, K: int):
    """One surrogate-screened cellular generation given the candidates' scores;
    returns (new pop, new makespans, chosen candidate per cell, candidates [cells*K][n])."""
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    sc = np.ascontiguousarray(scores, dtype=np.float32)
    out = np.zeros_like(pop)
    out_ms = np.zeros_like(ms)
    cells = rows * cols
    chosen = np.zeros(cells, dtype=np.int32)
    cands = np.zeros((cells * K, inst.n), dtype=np.int16)
    cp = prm._c(inst)
    lib.orc_screened_cellular_generation(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32), _ptr(inst.p, ctypes.c_int32),
                                         ctypes.byref(cp), island, generation, rows, cols, pop.shape[1],
                                         _ptr(pop, ctypes.c_int16), _ptr(ms, ctypes.c_int64),
                                         _ptr(out, ctypes.c_int16), _ptr(out_ms, ctypes.c_int64),
                                         _ptr(sc, ctypes.c_float), K, _ptr(chosen, ctypes.c_int32),
                                         _ptr(cands, ctypes.c_int16))
    return out, out_ms, chosen, cands


def screened_pseudo_generation(inst: Instance, prm: Params, island: int, generation: int, pop: np.ndarray,
                               ms: np.ndarray, scores: np.ndarray, K: int):
    """One surrogate-screened pseudo generation given the candidate children's
    scores ([pairs][K][2], flattened); returns (new pop, new makespans, chosen
    candidate per pair (-1: the pair did not cross), candidates
    [pairs*K*2][n], #decoded)."""
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    sc = np.ascontiguousarray(scores, dtype=np.float32)
    out = np.zeros_like(pop)
    out_ms = np.zeros_like(ms)
    pairs = pop.shape[0] // 2
    chosen = np.zeros(pairs, dtype=np.int32)
    cands = np.zeros((pairs * K * 2, inst.n), dtype=np.int16)
    cp = prm._c(inst)
    k = lib.orc_screened_pseudo_generation(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32),
                                           _ptr(inst.p, ctypes.c_int32), ctypes.byref(cp), island, generation,
                                           pop.shape[0], pop.shape[1], _ptr(pop, ctypes.c_int16),
                                           _ptr(ms, ctypes.c_int64), _ptr(out, ctypes.c_int16),
                                           _ptr(out_ms, ctypes.c_int64), _ptr(sc, ctypes.c_float), K,
                                           _ptr(chosen, ctypes.c_int32), _ptr(cands, ctypes.c_int16))
    return out, out_ms, chosen, cands, int(k)


def family_best2(fms) -> list:
    """Indices (role order c1, c2, a, b) of the two best family members."""
    f = np.ascontiguousarray(fms, dtype=np.int64)
    out = np.zeros(2, dtype=np.int32)
    _load().orc_family_best2(_ptr(f, ctypes.c_int64), _ptr(out, ctypes.c_int32))
    return out.tolist()


def pseudo_generation(inst: Instance, prm: Params, island: int, generation: int,
                      pop: np.ndarray, ms: np.ndarray):
    """One pseudo-island generation; returns (new pop, new makespans, #decoded)."""
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    out = np.zeros_like(pop)
    out_ms = np.zeros_like(ms)
    cp = prm._c(inst)
    k = lib.orc_pseudo_generation(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32),
                                  _ptr(inst.p, ctypes.c_int32), ctypes.byref(cp), island, generation,
                                  pop.shape[0], pop.shape[1], _ptr(pop, ctypes.c_int16),
                                  _ptr(ms, ctypes.c_int64), _ptr(out, ctypes.c_int16),
                                  _ptr(out_ms, ctypes.c_int64))
    return out, out_ms, int(k)


# ---------------------------------------------------------------------------
# Migration
# ---------------------------------------------------------------------------
def rank_island(ms: np.ndarray) -> np.ndarray:
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    out = np.zeros(len(ms), dtype=np.int32)
    _load().orc_rank_island(len(ms), _ptr(ms, ctypes.c_int64), _ptr(out, ctypes.c_int32))
    return out


def migrate_ring(pops: list, mss: list, n: int, num: int = 2, den: int = 100):
    """In place on lists of C-contiguous int16 [N_i][ld] and int64 [N_i] arrays."""
    lib = _load()
    I = len(pops)
    ld = pops[0].shape[1]
    sizes = np.array([p.shape[0] for p in pops], dtype=np.int32)
    parr = (_i16p * I)(*[_ptr(p, ctypes.c_int16) for p in pops])
    marr = (_i64p * I)(*[_ptr(m, ctypes.c_int64) for m in mss])
    lib.orc_migrate_ring(I, _ptr(sizes, ctypes.c_int32), ld, n, parr, marr, num, den)


def penetration_count(cA: int, cB: int, N: int, theta_num: int = 1, theta_den: int = 1) -> int:
    return int(_load().orc_penetration_count(cA, cB, N, theta_num, theta_den))


def migrate_penetration(popA, msA, popB, msB, n: int, theta_num: int = 1, theta_den: int = 1) -> int:
    """In place; returns the signed count (> 0: A -> B)."""
    return int(_load().orc_migrate_penetration(
        popA.shape[0], popB.shape[0], popA.shape[1], n, _ptr(popA, ctypes.c_int16),
        _ptr(msA, ctypes.c_int64), _ptr(popB, ctypes.c_int16), _ptr(msB, ctypes.c_int64),
        theta_num, theta_den))


# ---------------------------------------------------------------------------
# Whole dual-island GA driver (Section 4.1, Fig. 2): islands in ring order
# [cellular 0, pseudo 0, cellular 1, pseudo 1, ...], synchronous generations,
# migration every `gap` generations.
# ---------------------------------------------------------------------------
class IslandGA:
    def __init__(self, inst: Instance, prm: Params, n_cellular: int, rows: int, cols: int,
                 n_pseudo: int, pseudo_size: int, ld: int | None = None, pool=None, parts: int = 1):
        self.inst, self.prm = inst, prm
        self.rows, self.cols = rows, cols
        self.ld = ld if ld is not None else ((inst.n + 7) // 8) * 8
        self.kinds = []
        for q in range(max(n_cellular, n_pseudo)):
            if q < n_cellular:
                self.kinds.append("cellular")
            if q < n_pseudo:
                self.kinds.append("pseudo")
        self.sizes = [rows * cols if k == "cellular" else pseudo_size for k in self.kinds]
        self.pops, self.mss = [], []
        self.generation = 0
        for i, k in enumerate(self.kinds):
            N = self.sizes[i]
            pop = np.zeros((N, self.ld), dtype=np.int16)
            if k == "cellular":
                for c in range(N):
                    pop[c, :inst.n] = init_chromosome(prm.seed, i, c, inst.n)
            else:
                for q in range(N // 2):
                    a, b = init_pseudo_pair(prm.seed, i, q, inst.n)
                    pop[2 * q, :inst.n] = a
                    pop[2 * q + 1, :inst.n] = b
            self.pops.append(pop)
            self.mss.append(eval_population_threads(inst, pop, pool, parts) if pool else eval_population(inst, pop))
        self.decoded = 0

    def step(self):
        self.generation += 1
        g = self.generation
        for i, k in enumerate(self.kinds):
            if k == "cellular":
                p, m, d = cellular_generation(self.inst, self.prm, i, g, self.rows, self.cols,
                                              self.pops[i], self.mss[i])
            else:
                p, m, d = pseudo_generation(self.inst, self.prm, i, g, self.pops[i], self.mss[i])
            self.pops[i], self.mss[i] = p, m
            self.decoded += d

    def step_threads(self, pool, parts: int):
        """step() with every island's cells or pairs split over a thread pool."""
        self.generation += 1
        g = self.generation
        for i, k in enumerate(self.kinds):
            if k == "cellular":
                p, m, d = cellular_generation_threads(self.inst, self.prm, i, g, self.rows, self.cols,
                                                      self.pops[i], self.mss[i], pool, parts)
            else:
                p, m, d = pseudo_generation_threads(self.inst, self.prm, i, g, self.pops[i], self.mss[i], pool,
                                                    parts)
            self.pops[i], self.mss[i] = p, m
            self.decoded += d

    def migrate_ring(self, num: int = 2, den: int = 100):
        migrate_ring(self.pops, self.mss, self.inst.n, num, den)

    def migrate_penetration(self, theta_num: int = 1, theta_den: int = 1):
        counts = []
        for q in range(0, len(self.kinds) - 1, 2):
            counts.append(migrate_penetration(self.pops[q], self.mss[q], self.pops[q + 1],
                                              self.mss[q + 1], self.inst.n, theta_num, theta_den))
        return counts

    def best(self) -> int:
        return int(min(m.min() for m in self.mss))


# ---------------------------------------------------------------------------
# GA on the paper's genotype (machine-assignment strings of L = n * S genes)
# ---------------------------------------------------------------------------
def assign_init_row(seed: int, island: int, cell: int, n: int, S: int, M) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.int32)
    out = np.zeros(n * S, dtype=np.int16)
    _load().orc_assign_init_row(seed, island, cell, n, S, _ptr(M, ctypes.c_int32), _ptr(out, ctypes.c_int16))
    return out


def assign_init_pair(seed: int, island: int, k: int, n: int, S: int, M):
    M = np.ascontiguousarray(M, dtype=np.int32)
    a, b = np.zeros(n * S, dtype=np.int16), np.zeros(n * S, dtype=np.int16)
    _load().orc_assign_init_pair(seed, island, k, n, S, _ptr(M, ctypes.c_int32), _ptr(a, ctypes.c_int16),
                                 _ptr(b, ctypes.c_int16))
    return a, b


def assign_complement(m: int, M_s: int) -> int:
    return int(_load().orc_assign_complement(m, M_s))


def two_point(p1, p2, l: int, r: int) -> np.ndarray:
    p1 = np.ascontiguousarray(p1, dtype=np.int16)
    p2 = np.ascontiguousarray(p2, dtype=np.int16)
    out = np.zeros_like(p1)
    _load().orc_two_point(len(p1), _ptr(p1, ctypes.c_int16), _ptr(p2, ctypes.c_int16), l, r, _ptr(out, ctypes.c_int16))
    return out


def assign_reassign(genes, i: int, M_s: int, x: int) -> np.ndarray:
    g = np.array(genes, dtype=np.int16)
    _load().orc_assign_reassign(_ptr(g, ctypes.c_int16), i, M_s, x)
    return g


def assign_cellular_child(inst: AssignInstance, prm: Params, rows: int, cols: int, c: int, x, pop: np.ndarray,
                          obj: np.ndarray) -> np.ndarray:
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    obj = np.ascontiguousarray(obj, dtype=np.int64)
    xs = np.ascontiguousarray(x, dtype=np.uint32)
    child = np.zeros(inst.n * inst.S, dtype=np.int16)
    cp = prm._c(inst)
    _load().orc_assign_cellular_child(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32), rows, cols, c,
                                      _ptr(xs, ctypes.c_uint32), ctypes.byref(cp), _ptr(pop, ctypes.c_int16),
                                      pop.shape[1], _ptr(obj, ctypes.c_int64), _ptr(child, ctypes.c_int16))
    return child


def assign_cellular_generation(inst: AssignInstance, prm: Params, island: int, generation: int, rows: int,
                               cols: int, pop: np.ndarray, obj: np.ndarray):
    """One cellular generation of assignment strings; returns (pop, objectives, #evaluated)."""
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    obj = np.ascontiguousarray(obj, dtype=np.int64)
    out, out_obj = np.zeros_like(pop), np.zeros_like(obj)
    cp = prm._c(inst)
    k = lib.orc_assign_cellular_generation(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32),
                                           _ptr(inst.p_u, ctypes.c_int32), ctypes.byref(cp), island, generation, rows,
                                           cols, pop.shape[1], _ptr(pop, ctypes.c_int16), _ptr(obj, ctypes.c_int64),
                                           _ptr(out, ctypes.c_int16), _ptr(out_obj, ctypes.c_int64))
    return out, out_obj, int(k)


def assign_pseudo_generation(inst: AssignInstance, prm: Params, island: int, generation: int, pop: np.ndarray,
                             obj: np.ndarray):
    """One pseudo generation of assignment strings; returns (pop, objectives, #evaluated)."""
    lib = _load()
    pop = np.ascontiguousarray(pop, dtype=np.int16)
    obj = np.ascontiguousarray(obj, dtype=np.int64)
    out, out_obj = np.zeros_like(pop), np.zeros_like(obj)
    cp = prm._c(inst)
    k = lib.orc_assign_pseudo_generation(inst.n, inst.S, _ptr(inst.M, ctypes.c_int32),
                                         _ptr(inst.p_u, ctypes.c_int32), ctypes.byref(cp), island, generation,
                                         pop.shape[0], pop.shape[1], _ptr(pop, ctypes.c_int16),
                                         _ptr(obj, ctypes.c_int64), _ptr(out, ctypes.c_int16),
                                         _ptr(out_obj, ctypes.c_int64))
    return out, out_obj, int(k)
