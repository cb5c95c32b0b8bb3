"""Pin of the oracle's Philox4x32-10 against a library implementation: the
host-side Philox4_32_10 generator of curand (run as a library, no GPU needed).
curand's host generator with seed S and offset 4n (n < 2^16; larger offsets follow
curand's own multi-stream layout) returns the block for key
(S_lo, S_hi) and counter (0, 0, n_lo, n_hi); many keys and counters exercise
every round of the bijection and the key schedule."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from oracle import philox4x32_10


def _curand():
    cands = [ctypes.util.find_library("curand"), "/usr/local/cuda/lib64/libcurand.so",
             "libcurand.so.10"]
    for c in cands:
        if c and (os.path.exists(c) or not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                continue
    pytest.skip("libcurand not available")


def _curand_block(lib, seed, offset):
    gen = ctypes.c_void_p()
    PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10 in curand.h
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX) != 0:
        pytest.skip("curand host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(4, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 8, 0x123456789ABCDEF, 2**64 - 1, 977])
@pytest.mark.parametrize("n", [0, 1, 2, 1000, 4095, 65535])
def test_philox_matches_curand_host(seed, n):
    lib = _curand()
    ref = _curand_block(lib, seed, 4 * n)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    got = philox4x32_10(np.array([0, 0, n & 0xFFFFFFFF, n >> 32], dtype=np.uint32), key)
    np.testing.assert_array_equal(got, ref)


def test_philox_bits_uniform():
    """Counter-indexed draws look uniform: chi-square of the top 4 bits of
    8192 blocks (the generator's bijection property is what matters here)."""
    key = np.array([1, 0], dtype=np.uint32)
    words = np.concatenate([philox4x32_10(np.array([k, 3, 7, 1], np.uint32), key) for k in range(8192)])
    hist = np.bincount(words >> 28, minlength=16)
    exp = words.size / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 45.0  # 15 dof, p ~ 1e-4
