"""Pins of the oracle's random inputs: Philox4x32-10 against the cuRAND host
generator (an independent implementation run as a library), the uniform
grids against their exactness and symmetry, and the normal quantile against
scipy's ndtri and mpmath at high precision."""
import ctypes
import math
import os

import numpy as np
import pytest
import scipy.special as sp
from scipy import stats

import oracle

_CURAND_PATHS = ["/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"]


def _curand():
    for p in _CURAND_PATHS:
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _curand_host_philox(seed, n, offset=0):
    """n 32-bit outputs of cuRAND's host Philox4x32-10 generator."""
    cr = _curand()
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = (ctypes.c_uint32 * n)()
        assert cr.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    return np.frombuffer(buf, dtype=np.uint32).copy()


def _host_block_counter(q):
    # cuRAND's host Philox generator emits block q (4 words) from counter
    # (q >> 16 as a 64-bit value in words 0-1, q & 0xffff in word 2, 0),
    # key = seed; established by experiment against this library
    hi = q >> 16
    return (hi & 0xFFFFFFFF, hi >> 32, q & 0xFFFF, 0)


@pytest.mark.parametrize("seed", [0, 42, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    n_blocks = 4096
    out = _curand_host_philox(seed, 4 * n_blocks).reshape(-1, 4)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    ctr = np.array([_host_block_counter(q) for q in range(n_blocks)], dtype=np.uint32)
    assert np.array_equal(oracle.philox(ctr, key), out)


@pytest.mark.parametrize("q0", [65536 * 5 + 7, 65536 * (2**32 + 3) + 11, 65536 * 1000003 + 65535])
def test_philox_matches_curand_high_counter_words(q0):
    seed = 0xDEADBEEFCAFEF00D
    out = _curand_host_philox(seed, 4 * 64, offset=4 * q0).reshape(-1, 4)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    ctr = np.array([_host_block_counter(q0 + i) for i in range(64)], dtype=np.uint32)
    assert np.array_equal(oracle.philox(ctr, key), out)


def test_philox_avalanche_on_each_counter_and_key_word():
    rng = np.random.default_rng(1)
    base = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([0x01234567, 0x89ABCDEF], dtype=np.uint32)
    y0 = oracle.philox(base, key)
    for word in range(4):
        flipped = base.copy()
        flipped[:, word] ^= np.uint32(1 << (word * 7 % 32))
        y1 = oracle.philox(flipped, key)
        bits = np.unpackbits((y0 ^ y1).view(np.uint8)).mean()
        assert 0.45 < bits < 0.55
    y2 = oracle.philox(base, key ^ np.array([0, 1 << 20], dtype=np.uint32))
    assert 0.45 < np.unpackbits((y0 ^ y2).view(np.uint8)).mean() < 0.55


def test_uniform_grids_are_exact_symmetric_and_open():
    assert oracle.uniform_f64(0, 0) == 2.0**-53
    assert oracle.uniform_f64(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0**-53
    assert oracle.uniform_f32(0) == 2.0**-24
    assert oracle.uniform_f32(0xFFFFFFFF) == 1.0 - 2.0**-24
    rng = np.random.default_rng(2)
    for hi, lo in rng.integers(0, 2**32, size=(2000, 2)):
        u = oracle.uniform_f64(hi, lo)
        # complementing every bit reflects the grid: U(~w) = 1 - U(w) exactly
        assert oracle.uniform_f64(hi ^ 0xFFFFFFFF, lo ^ 0xFFFFFFFF) == 1.0 - u
        # the low 12 bits of the second word are dropped (52-bit mantissa)
        assert oracle.uniform_f64(hi, lo ^ 0xFFF) == u
        w = int(hi)
        assert oracle.uniform_f32(w ^ 0xFFFFFFFF) == 1.0 - oracle.uniform_f32(w)
        # the single-precision grid is the double grid's top 23 bits
        assert abs(oracle.uniform_f32(w) - u) <= 2.0**-23
        assert np.float32(oracle.uniform_f32(w)) == oracle.uniform_f32(w)


def _ulp(x):
    return np.spacing(np.abs(x))


def test_norm_inv_matches_ndtri_and_mpmath():
    mpmath = pytest.importorskip("mpmath")
    rng = np.random.default_rng(3)
    u = np.concatenate([
        rng.random(100000),
        np.exp(-rng.uniform(1.0, 36.7, size=20000)),        # lower tail to 2^-53
        1.0 - np.exp(-rng.uniform(1.0, 36.0, size=20000)),  # upper tail
        np.array([2.0**-53, 1.0 - 2.0**-53, 0.5 - 2.0**-40, 0.5 + 2.0**-40]),
    ])
    u = u[(u > 0) & (u < 1)]
    z = oracle.norm_inv(u)
    ref = sp.ndtri(u)
    err = np.abs(z - ref)
    tol = 8 * _ulp(ref) + 1e-300
    bad = err > tol
    # settle any disagreement with ndtri at 40 digits
    mpmath.mp.dps = 40
    for i in np.flatnonzero(bad)[:200]:
        exact = float(-mpmath.sqrt(2) * mpmath.erfinv(1 - 2 * mpmath.mpf(float(u[i]))))
        assert abs(z[i] - exact) <= 4 * _ulp(exact) + 1e-300, (u[i], z[i], exact)
    assert bad.mean() < 1e-3


def test_norm_inv_symmetry_on_the_grid():
    rng = np.random.default_rng(4)
    w = rng.integers(0, 2**32, size=(5000, 2))
    u = np.array([oracle.uniform_f64(a, b) for a, b in w])
    um = np.array([oracle.uniform_f64(a ^ 0xFFFFFFFF, b ^ 0xFFFFFFFF) for a, b in w])
    assert np.array_equal(oracle.norm_inv(u), -oracle.norm_inv(um))


def test_draws_compose_philox_grid_and_quantile():
    seed, stream = 0xABCDEF0123456789, 7
    path = np.array([0, 1, 4095, 131071, 2**32 - 1], dtype=np.uint32)
    step = np.array([0, 251, 3, 499, 2**32 - 1], dtype=np.uint32)
    d64 = oracle.draws(seed, stream, path, step, oracle.GRID_F64)
    d32 = oracle.draws(seed, stream, path, step, oracle.GRID_F32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    ctr = np.stack([path, step, np.full_like(path, stream), np.zeros_like(path)], 1)
    w = oracle.philox(ctr, key)
    for i in range(path.size):
        uV = oracle.uniform_f64(w[i, 0], w[i, 1])
        uX = oracle.uniform_f64(w[i, 2], w[i, 3])
        assert d64[i, 0] == uV
        assert d64[i, 1] == oracle.norm_inv([uV])[0]
        assert d64[i, 2] == oracle.norm_inv([uX])[0]
        assert d32[i, 0] == oracle.uniform_f32(w[i, 0])
        assert d32[i, 2] == oracle.norm_inv([oracle.uniform_f32(w[i, 2])])[0]


def test_draws_are_independent_standard_normals():
    n = 4096 * 49
    path = np.arange(n, dtype=np.uint32) % 4096
    step = (np.arange(n, dtype=np.uint32) // 4096)
    d = oracle.draws(42, 0, path, step)
    for col in (1, 2):
        assert stats.kstest(d[:, col], "norm").pvalue > 1e-3
    assert abs(np.corrcoef(d[:, 1], d[:, 2])[0, 1]) < 5.0 / math.sqrt(n)
    # consecutive steps of one path are uncorrelated too
    z = d[:, 1].reshape(-1, 4096)
    assert abs(np.corrcoef(z[:-1].ravel(), z[1:].ravel())[0, 1]) < 5.0 / math.sqrt(z[1:].size)
