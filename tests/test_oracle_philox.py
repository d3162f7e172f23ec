"""Pins of the oracle's counter-based generator and its normal draws.

The oracle implements Philox4x32-10 from Salmon et al. (SC'11).  It is pinned
against an independent implementation: cuRAND's host-side
CURAND_RNG_PSEUDO_PHILOX4_32_10 generator, which runs on the CPU.  That
generator emits block ``i = 65536 r + t`` from counter ``(r_lo, r_hi, t, 0)``
under key ``(seed_lo, seed_hi)``; ``curandSetGeneratorOffset`` moves the start.
"""
import ctypes
import os

import numpy as np
import pytest
from scipy import stats

CURAND_PHILOX = 161


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def _curand_blocks(lib, seed, offset_blocks, nblocks):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_PHILOX) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * offset_blocks)) == 0
        buf = np.zeros(4 * nblocks, np.uint32)
        assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(buf.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return buf.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 3004])
def test_philox_matches_curand(oracle_mod, seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not present")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    # counter word 2 (the thread/subsequence index of cuRAND's host layout)
    ref = _curand_blocks(lib, seed, 0, 64)
    for t in range(64):
        assert np.array_equal(oracle_mod.philox([0, 0, t, 0], key), ref[t])
    # counter words 0 and 1 (the per-thread 64-bit counter), reached through the offset
    for r, t in [(1, 0), (2, 5), (7, 65535), ((1 << 32) + 3, 9), ((0x2FFF << 32) | 0xFFFFFFFF, 77)]:
        got = _curand_blocks(lib, seed, 65536 * r + t, 1)[0]
        want = oracle_mod.philox([r & 0xFFFFFFFF, r >> 32, t, 0], key)
        assert np.array_equal(got, want), (r, t)


def test_stream_layout(oracle_mod):
    """Block b of the (step, chain, tag) stream is Philox of counter (b, step, chain, tag)."""
    seed = 0xDEADBEEF12345678
    key = [seed & 0xFFFFFFFF, seed >> 32]
    blocks = oracle_mod.philox_blocks(seed, 17, 4242, 2, 3, 5)
    for i in range(5):
        assert np.array_equal(blocks[i], oracle_mod.philox([3 + i, 17, 4242, 2], key))


def test_uniform_open_interval_and_alpha(oracle_mod):
    seed = 77
    key = [seed, 0]
    for step in range(1, 50):
        w = oracle_mod.philox([0, step, 5, 2], key)
        want = ((int(w[0]) >> 9) + 0.5) / 2.0 ** 23
        a = oracle_mod.alpha(seed, step, 5)
        assert a == want
        assert 0.0 < a < 1.0
        # exactly representable in float32 as well as float64
        assert float(np.float32(a)) == a


def test_box_muller_pairs(oracle_mod):
    """z_{4b+2i}, z_{4b+2i+1} = sqrt(-2 ln u) (cos, sin)(2 pi v) on the block's uniforms."""
    seed, step, chain, tag = 99, 3, 11, 1
    z = oracle_mod.normals(seed, step, chain, tag, 16)
    blocks = oracle_mod.philox_blocks(seed, step, chain, tag, 0, 4)
    for b in range(4):
        u = ((blocks[b].astype(np.int64) >> 9) + 0.5) / 2.0 ** 23
        for i in range(2):
            r = np.sqrt(-2.0 * np.log(u[2 * i]))
            assert z[4 * b + 2 * i] == pytest.approx(r * np.cos(2 * np.pi * u[2 * i + 1]), rel=1e-15, abs=1e-15)
            assert z[4 * b + 2 * i + 1] == pytest.approx(r * np.sin(2 * np.pi * u[2 * i + 1]), rel=1e-15, abs=1e-15)


def test_normals_are_standard(oracle_mod):
    z = np.concatenate([oracle_mod.normals(5, s, c, 1, 1024) for s in range(4) for c in range(25)])
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # streams with different tags / chains / steps are not copies of one another
    a = oracle_mod.normals(5, 1, 0, 1, 64)
    assert not np.array_equal(a, oracle_mod.normals(5, 1, 0, 0, 64))
    assert not np.array_equal(a, oracle_mod.normals(5, 1, 1, 1, 64))
    assert not np.array_equal(a, oracle_mod.normals(5, 2, 0, 1, 64))
