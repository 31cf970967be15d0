"""Seeded synthetic inputs for the FFS island GA (tests, smoke check and bench).

This module holds no arithmetic of the method: it only draws instances and
random job orders with numpy's PCG64 generator, so both the CUDA path and
the CPU oracle can be fed identical inputs.  The GA's own randomness
(Philox4x32-10) is not here; each side implements it on its own.

Instance shapes follow the workloads the library is measured on (the paper's
own 300x4x2 instances, Section 5 and Table 1, are unpublished; these stand
in for them):

  tiny         20 jobs x 5 stages, 3 machines per stage, p ~ U[1,99]; 8x8 torus
  dual_100x10  100 jobs x 10 stages, M_s ~ U[2,5]; 64x64 torus + pseudo 4096
  scale_500x20 500 jobs x 20 stages, M_s ~ U[5,10]; 4 x 128x128 torus +
               4 pseudo islands of 16384 (131072 chromosomes)
  batch_256    256 instances, n ~ U[20,500], S ~ U[5,20], M_s ~ U[2,10];
               32x32 torus each
  paper_300x4  the paper's shape: 300 jobs x 4 stages x 2 machines,
               p ~ U[1,5] (Section 5, Table 1), for context runs
  paper_obj_300x4  the same shape with Table 1's release and due times
               and WT = 100 (objective WT * total tardiness + C_max)
  assign_500x20  the paper's genotype (machine-assignment strings of 500 x 20
               genes) on unrelated machines: M_s ~ U[5,10], P_jsm ~ U[1,99]
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class InstanceSpec:
    n: int
    S: int
    M: np.ndarray   # int32 [S]
    p: np.ndarray   # int32 [n][S]
    release: np.ndarray | None = None   # int32 [n]
    due: np.ndarray | None = None       # int32 [n]
    wt: int = 0


def make_instance(n: int, S: int, m_lo: int, m_hi: int, p_lo: int = 1, p_hi: int = 99,
                  seed: int = 1) -> InstanceSpec:
    """M_s ~ U{m_lo..m_hi}, p[j][s] ~ U{p_lo..p_hi}, drawn in that order."""
    rng = np.random.default_rng(seed)
    M = rng.integers(m_lo, m_hi + 1, size=S, dtype=np.int64).astype(np.int32)
    p = rng.integers(p_lo, p_hi + 1, size=(n, S), dtype=np.int64).astype(np.int32)
    return InstanceSpec(n, S, M, p)


def make_paper_instance(n: int = 300, S: int = 4, m: int = 2, seed: int = 1, wt: int = 100) -> InstanceSpec:
    """The paper's experimental instances (Section 5, Table 1) on identical
    machines: p[j][s] ~ U{1..5}; Pbar_j = sum_s p[j][s] (the table's
    sum_m P_jsm / M_s with P_jsm = p_js), Pbar = sum_j Pbar_j; R_j ~ U{0..Pbar};
    sigma_j ~ U[0, 2) real, D_j = R_j + floor(Pbar_j (1 + sigma_j)); WT = 100.
    Drawn in that order from one stream."""
    rng = np.random.default_rng(seed)
    M = np.full(S, m, dtype=np.int32)
    p = rng.integers(1, 6, size=(n, S), dtype=np.int64).astype(np.int32)
    pbar_j = p.sum(axis=1).astype(np.int64)
    pbar = int(pbar_j.sum())
    release = rng.integers(0, pbar + 1, size=n, dtype=np.int64)
    sigma = rng.random(n) * 2.0
    due = release + np.floor(pbar_j * (1.0 + sigma)).astype(np.int64)
    return InstanceSpec(n, S, M, p, release.astype(np.int32), due.astype(np.int32), wt)


def make_batch(count: int = 256, seed: int = 1, n_range=(20, 500), s_range=(5, 20),
               m_range=(2, 10), p_range=(1, 99)) -> list[InstanceSpec]:
    """Uneven instances: n, S, then M_s and p per instance, one stream."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        S = int(rng.integers(s_range[0], s_range[1] + 1))
        M = rng.integers(m_range[0], m_range[1] + 1, size=S, dtype=np.int64).astype(np.int32)
        p = rng.integers(p_range[0], p_range[1] + 1, size=(n, S), dtype=np.int64).astype(np.int32)
        out.append(InstanceSpec(n, S, M, p))
    return out


def random_population(n: int, N: int, ld: int | None = None, seed: int = 0) -> np.ndarray:
    """N random job orders of n jobs as int16 rows of length ld (padding = 0)."""
    ld = ld if ld is not None else ((n + 7) // 8) * 8
    rng = np.random.default_rng(seed)
    pop = np.zeros((N, ld), dtype=np.int16)
    keys = rng.random((N, n))
    pop[:, :n] = np.argsort(keys, axis=1).astype(np.int16)
    return pop


@dataclass
class AssignSpec:
    n: int
    S: int
    M: np.ndarray     # int32 [S]
    p_u: np.ndarray   # int32 [n][sum M]: job j, stage s, machine m at [j][M_0 + ... + M_{s-1} + m]


def make_assign_instance(n: int, S: int, m_lo: int, m_hi: int, p_lo: int = 1, p_hi: int = 99,
                         seed: int = 1) -> AssignSpec:
    """Unrelated machines: M_s ~ U{m_lo..m_hi}, then every P_jsm ~ U{p_lo..p_hi}
    (job-major, stage, machine), drawn in that order."""
    rng = np.random.default_rng(seed)
    M = rng.integers(m_lo, m_hi + 1, size=S, dtype=np.int64).astype(np.int32)
    p_u = rng.integers(p_lo, p_hi + 1, size=(n, int(M.sum())), dtype=np.int64).astype(np.int32)
    return AssignSpec(n, S, M, p_u)


def random_assignments(n: int, S: int, M, N: int, ld: int | None = None, seed: int = 0) -> np.ndarray:
    """N random machine-assignment strings (gene j*S + s ~ U{0..M_s - 1}) as
    int16 rows of length ld (padding = 0)."""
    M = np.asarray(M, dtype=np.int64)
    ld = ld if ld is not None else ((n * S + 7) // 8) * 8
    rng = np.random.default_rng(seed)
    pop = np.zeros((N, ld), dtype=np.int16)
    u = rng.random((N, n, S))
    pop[:, :n * S] = np.floor(u * M[None, None, :]).astype(np.int16).reshape(N, n * S)
    return pop


WORKLOADS = {
    "tiny": dict(n=20, S=5, m=(3, 3), seed=1, n_cellular=1, rows=8, cols=8,
                 n_pseudo=0, pseudo_size=0, generations=100),
    "dual_100x10": dict(n=100, S=10, m=(2, 5), seed=1, n_cellular=1, rows=64, cols=64,
                        n_pseudo=1, pseudo_size=4096, generations=1000,
                        migration="ring", gap=50, mig_num=2, mig_den=100),
    "scale_500x20": dict(n=500, S=20, m=(5, 10), seed=1, n_cellular=4, rows=128, cols=128,
                         n_pseudo=4, pseudo_size=16384, generations=200,
                         migration="ring", gap=1, mig_num=2, mig_den=100),
    "batch_256": dict(count=256, n=(20, 500), S=(5, 20), m=(2, 10), seed=1, rows=32, cols=32,
                      generations=500),
    "paper_300x4": dict(n=300, S=4, m=(2, 2), p=(1, 5), seed=1, n_cellular=1, rows=16, cols=16,
                        n_pseudo=1, pseudo_size=256, generations=2000,
                        migration="penetration", gap=500),
}


def workload_instance(name: str) -> InstanceSpec:
    w = WORKLOADS[name]
    p = w.get("p", (1, 99))
    return make_instance(w["n"], w["S"], w["m"][0], w["m"][1], p[0], p[1], seed=w["seed"])


def mlp_params(in_dim: int, h1: int, h2: int, seed: int = 0) -> dict:
    """Random network parameters for tests (numpy PCG64, He-style uniform
    limits sqrt(6 / fan_in), the output weights scaled by 0.1, biases 0): an
    input, like the instances above.  The library draws its own with
    ffs_mlp_init."""
    rng = np.random.default_rng(seed)

    def u(shape, fan_in):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=shape).astype(np.float32)
    return {"W1": u((h1, in_dim), in_dim), "b1": np.zeros(h1, np.float32),
            "W2": u((h2, h1), h1), "b2": np.zeros(h2, np.float32),
            "w3": u((h2,), h2) * 0.1, "b3": np.float32(0.0)}
