"""Pins the oracle's Philox4x32-10 (written from Salmon et al., SC'11) against
NVIDIA's curand implementation of the same generator, called on the host."""
import ctypes

import numpy as np

import oracle


def _ref(lib, c, k):
    o = np.zeros(4, np.uint32)
    lib.curand_philox_ref(c.ctypes.data_as(ctypes.c_void_p), k.ctypes.data_as(ctypes.c_void_p),
                          o.ctypes.data_as(ctypes.c_void_p))
    return o


def test_philox_matches_curand_random_inputs(curand_philox):
    rng = np.random.default_rng(12345)
    for _ in range(3000):
        c = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(oracle.philox4x32_10(c, k), _ref(curand_philox, c, k))


def test_philox_matches_curand_edge_inputs(curand_philox):
    for c in ([0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 5]):
        for k in ([0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [1, 0]):
            c_ = np.array(c, np.uint32)
            k_ = np.array(k, np.uint32)
            assert np.array_equal(oracle.philox4x32_10(c_, k_), _ref(curand_philox, c_, k_))


def test_philox_output_bits_balanced():
    # 4096 draws x 128 bits: every output bit position is set about half the time
    bits = np.zeros(128)
    for t in range(4096):
        out = oracle.philox4x32_10([t, 0, 7, 0], [3, 0])
        for w in range(4):
            for b in range(32):
                bits[32 * w + b] += (int(out[w]) >> b) & 1
    frac = bits / 4096
    assert np.all(np.abs(frac - 0.5) < 0.04)
