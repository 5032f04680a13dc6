"""Pins of the oracle's random numbers.

Philox-4x32-10 (Salmon et al., SC'11) is pinned bit-exactly against the
cuRAND host generator (a library routine that runs on the CPU).  That
generator's output block b, counted from its offset, is the Philox block
with counter (b >> 16 as a 64-bit number in words 0-1, b & 0xffff in word 2,
0 in word 3) and key (seed low, seed high): every round, multiplier and key
increment, and counter words 0, 1 and 2, are exercised.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

pytestmark = []

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             ctypes.util.find_library("curand")]
    for c in cands:
        if c:
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    pytest.skip("libcurand not found")


def _curand_host(seed, offset, n_blocks):
    lib = _curand()
    g = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out.reshape(n_blocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x190104200, 0xFFFFFFFFFFFFFFFF, 0x9E3779B97F4A7C15])
@pytest.mark.parametrize("offset_blocks", [0, 65530, 3 * 65536 + 17, (1 << 48) + (5 << 16) + 3])
def test_philox_matches_curand_host(orc, seed, offset_blocks):
    n = 12
    ref = _curand_host(seed, 4 * offset_blocks, n)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for k in range(n):
        b = offset_blocks + k
        hi = b >> 16
        ctr = (hi & 0xFFFFFFFF, hi >> 32, b & 0xFFFF, 0)
        assert orc.philox4x32_10(ctr, key) == [int(v) for v in ref[k]], (seed, b)


def test_philox_fill_layout(orc):
    """Block (call c, path p) has counter (c, 0, p low, p high)."""
    seed = 0x190104200
    key = (seed & 0xFFFFFFFF, seed >> 32)
    path0 = (1 << 32) - 3  # crosses into the high path word
    out = orc.philox_fill(seed, path0, 6, 3)
    for i in range(6):
        p = path0 + i
        for c in range(3):
            assert list(out[i, c]) == orc.philox4x32_10((c, 0, p & 0xFFFFFFFF, p >> 32), key)


def test_uniform_map_exact_and_open():
    import oracle
    oracle.build()
    lo, hi = oracle.uniform(0), oracle.uniform(0xFFFFFFFF)
    assert lo == 2.0 ** -24 and hi == 1.0 - 2.0 ** -24
    # the low 9 bits are dropped; every value is an odd multiple of 2^-24, exact in FP32
    for w in [0, 511, 512, 0x80000000, 0xDEADBEEF, 0xFFFFFFFF]:
        u = oracle.uniform(w)
        assert u == ((w >> 9) + 0.5) / 2.0 ** 23
        assert float(np.float32(u)) == u
        assert 0.0 < u < 1.0


def test_box_muller_structure(orc):
    """Each normal pair has radius^2 = -2 ln u_a and angle 2 pi u_b (Box-Muller)."""
    seed = 12345
    key = (seed & 0xFFFFFFFF, seed >> 32)
    z = orc.normals_fill(seed, 7, 3, 8)
    for i in range(3):
        p = 7 + i
        for call in range(2):
            o = orc.philox4x32_10((call, 0, p, 0), key)
            for q in range(2):
                ua, ub = orc.uniform(o[2 * q]), orc.uniform(o[2 * q + 1])
                za, zb = z[i, 4 * call + 2 * q], z[i, 4 * call + 2 * q + 1]
                assert math.isclose(za * za + zb * zb, -2.0 * math.log(ua), rel_tol=1e-13)
                ang = math.atan2(zb, za) % (2 * math.pi)
                assert abs(ang - 2 * math.pi * ub) < 1e-12


def test_normals_distribution(orc):
    """Moments and a Kolmogorov-Smirnov test against the standard normal."""
    from scipy import stats
    z = orc.normals_fill(0x190104200, 0, 4096, 256).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(z)) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(z[: 1 << 18], "norm").pvalue > 1e-4
    # consecutive normals of one path are uncorrelated
    zz = orc.normals_fill(99, 0, 8192, 64)
    c = np.corrcoef(zz[:, :-1].ravel(), zz[:, 1:].ravel())[0, 1]
    assert abs(c) < 5 / math.sqrt(zz.size)
