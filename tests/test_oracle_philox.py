"""Pins of the oracle's Philox4x32-10 stream and its integer mappings.

Philox4x32-10: Salmon, Moraes, Dror, Shaw, SC 2011.  The oracle's block
function is checked against NVIDIA's cuRAND host generator (a library run on
the CPU): with offset 0 and seed s, cuRAND's output block b is Philox applied
to the counter (0, 0, b, 0) under the key (low, high) of s.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle as orc


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) if cand.startswith("/") else cand:
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    return None


def _curand_host_philox(lib, seed, count):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), ctypes.c_int(161)) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(0)) == 0
        out = (ctypes.c_uint32 * count)()
        assert lib.curandGenerate(gen, out, ctypes.c_size_t(count)) == 0
        return np.frombuffer(out, dtype=np.uint32).copy()
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 7, 1, 0xFFFFFFFF, 0x0123456789ABCDEF, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    ref = _curand_host_philox(lib, seed, 4 * 64)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in range(64):
        got = orc.philox([0, 0, b, 0], key)
        assert got.tolist() == ref[4 * b:4 * b + 4].tolist(), (seed, b)


def test_draw_layout():
    # draw d = word d mod 4 of the block with counter (d/4, cell, gen, island | purpose<<24)
    seed = 0xDEADBEEF12345678
    for d in range(12):
        blk = orc.philox([d // 4, 5, 9, 3 | (orc.PURPOSE_CELLULAR << 24)],
                         [seed & 0xFFFFFFFF, seed >> 32])
        assert orc.draw(seed, orc.PURPOSE_CELLULAR, 3, 9, 5, d) == int(blk[d % 4])


def test_uniform_closed_form():
    assert orc.uniform(0, 5) == 0
    assert orc.uniform(2**32 - 1, 5) == 4
    assert orc.uniform(2**31, 2) == 1 and orc.uniform(2**31 - 1, 2) == 0
    for k in (1, 3, 5, 99, 500):
        for x in (0, 1, 12345, 2**31, 2**32 - 1):
            assert orc.uniform(x, k) == (x * k) >> 32
    # slot k of [0,5) starts at ceil(k * 2^32 / 5)
    for k in range(5):
        lo = -(-k * 2**32 // 5)
        assert orc.uniform(lo, 5) == k
        if lo > 0:
            assert orc.uniform(lo - 1, 5) == k - 1


def test_bernoulli_thresholds():
    # paper's rates (Section 5): pc 1.00 and pm 0.05 cellular, pc 0.75 pseudo
    assert orc.threshold(1.0) == 2**32
    assert orc.threshold(0.75) == 3221225472
    assert orc.threshold(0.05) == 214748364
    assert orc.bernoulli(2**32 - 1, 2**32)
    assert not orc.bernoulli(0, 0)
    assert orc.bernoulli(3221225471, 3221225472) and not orc.bernoulli(3221225472, 3221225472)


def test_init_chromosome_is_uniform_permutation():
    # Fisher-Yates over n = 3: all 6 orders equally likely (chi-square, 5 dof)
    counts = {}
    N = 6000
    for c in range(N):
        perm = tuple(orc.init_chromosome(7, 0, c, 3).tolist())
        counts[perm] = counts.get(perm, 0) + 1
    assert len(counts) == 6
    chi2 = sum((v - N / 6) ** 2 / (N / 6) for v in counts.values())
    assert chi2 < 20.5  # p < 0.001 critical value for 5 dof
    for c in range(50):
        perm = orc.init_chromosome(7, 2, c, 500)
        assert sorted(perm.tolist()) == list(range(500))


def test_init_chromosome_uses_listed_draws():
    n, seed, isl, cell = 6, 99, 1, 4
    a = list(range(n))
    for i in range(n - 1, 0, -1):
        x = orc.draw(seed, orc.PURPOSE_INIT, isl, 0, cell, n - 1 - i)
        j = (x * (i + 1)) >> 32
        a[i], a[j] = a[j], a[i]
    assert orc.init_chromosome(seed, isl, cell, n).tolist() == a


def test_pseudo_pair_is_reversal():
    a, b = orc.init_pseudo_pair(7, 1, 3, 50)
    assert b.tolist() == a.tolist()[::-1]
    assert a.tolist() == orc.init_chromosome(7, 1, 6, 50).tolist()
