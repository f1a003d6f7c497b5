"""Pin of the oracle's Philox4x32-10 against an independent implementation: the
Philox4_32_10 generator of NVIDIA's cuRAND library, run on the host CPU (cuRAND's host
generator needs no GPU).

cuRAND's host generator with seed s keys every block with (s mod 2^32, s div 2^32) and
writes block j of its output (j counted from the generator offset / 4) as the four words of
the counter (lo32(j div 65536), hi32(j div 65536), j mod 65536, 0): it emulates 65,536
device threads, thread t drawing from subsequence t. The tests locate that layout by its
known structure and then compare the oracle's words, bit for bit, at counters covering the
key schedule (keys with both halves set), word 0 and word 1 of the counter (carries
included) and word 2. Word 3 of the counter stays 0 on this route; the GPU test
``tests/test_gpu_philox_curand_device.py`` covers it through cuRAND's device API.

A wrong multiplier or Weyl constant, a missing round, a swapped output word or a misplaced
counter word turns these tests red.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

from oracle.philox import move_draws, philox4x32_10, seed_key, to_unit

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
THREADS = 65536


def _load_curand():
    names = [ctypes.util.find_library("curand"), "libcurand.so.10", "libcurand.so",
             "/usr/local/cuda/lib64/libcurand.so"]
    for n in names:
        if not n:
            continue
        try:
            return ctypes.CDLL(n)
        except OSError:
            continue
    return None


_LIB = _load_curand()
pytestmark = pytest.mark.skipif(_LIB is None, reason="cuRAND library not found")


def curand_host_words(seed: int, first_block: int, n_blocks: int) -> np.ndarray:
    """Blocks first_block .. first_block + n_blocks - 1 of cuRAND's host Philox4_32_10
    output for `seed`, as a [n_blocks][4] uint32 array."""
    lib = _LIB
    g = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out.reshape(n_blocks, 4)


def oracle_words(seed: int, first_block: int, n_blocks: int) -> np.ndarray:
    j = first_block + np.arange(n_blocks, dtype=np.uint64)
    step, t = j // np.uint64(THREADS), j % np.uint64(THREADS)
    ctr = (step & np.uint64(0xFFFFFFFF), step >> np.uint64(32), t, np.zeros_like(t))
    return np.stack(philox4x32_10(ctr, seed_key(seed)), -1)


SEEDS = [0, 1, 0xFFFFFFFFFFFFFFFF, 0xA4093822299F31D0, 0x243F6A8885A308D3, 0x00000001_00000000]
# first output block: zero counter; across the first thread-block wrap (word 0 of the
# counter becomes 1); word 0 at its maximum and its carry into word 1; large word 1
STARTS = [0, THREADS - 5, THREADS * 0xFFFFFFFF - 3, THREADS * ((0x1234 << 32) | 0xFFFFFFFE) + 60000]


@pytest.mark.parametrize("seed", SEEDS)
@pytest.mark.parametrize("start", STARTS)
def test_oracle_equals_curand_host_philox(seed, start):
    n = 300
    got = oracle_words(seed, start, n)
    ref = curand_host_words(seed, start, n)
    bad = np.argwhere(got != ref)
    assert bad.size == 0, f"first mismatch at block/word {bad[0]}"


def test_every_counter_word_below_three_is_exercised():
    """The compared blocks really vary words 0, 1 and 2 of the counter and both key halves
    (guards the test itself against a layout that would leave one of them constant)."""
    j = np.array([STARTS[2] + 3, STARTS[2] + 3 + THREADS, STARTS[3]], dtype=np.uint64)
    step = j // np.uint64(THREADS)
    assert (step & np.uint64(0xFFFFFFFF))[0] == 0xFFFFFFFF
    assert (step >> np.uint64(32))[1] == 1 and (step & np.uint64(0xFFFFFFFF))[1] == 0
    assert (step >> np.uint64(32))[2] == 0x1234
    assert seed_key(SEEDS[3]) == (0x299F31D0, 0xA4093822)


@pytest.mark.parametrize("seed,sweep,electron,walker", [(0, 0, 0, 0), (0, 3, 17, 255),
                                                        (0xDEADBEEF12345678, 41, 511, 65535)])
def test_move_draw_words_are_curands(seed, sweep, electron, walker):
    """The displacement words of a move (block (sweep, electron, walker, 0), Box-Muller on
    words 0-1 and 2-3) are the words cuRAND writes for that counter."""
    j = ((electron << 32) | sweep) * THREADS + walker
    w = curand_host_words(seed, j, 1)[0].astype(np.float64)
    u = (w + 0.5) * 2.0 ** -32
    xi, _ = move_draws(seed, sweep, electron, walker)
    r01 = np.sqrt(-2.0 * np.log(u[0]))
    r23 = np.sqrt(-2.0 * np.log(u[2]))
    expect = np.array([r01 * np.cos(2 * np.pi * u[1]), r01 * np.sin(2 * np.pi * u[1]),
                       r23 * np.cos(2 * np.pi * u[3])])
    assert np.array_equal(xi, expect)
    assert np.array_equal(to_unit(np.uint32(curand_host_words(seed, j, 1)[0, 0])), u[0])
