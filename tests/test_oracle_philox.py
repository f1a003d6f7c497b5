"""Statistical checks of the oracle's Philox4x32-10 generator and move draws (CPU).

The bit-exact pins against an independent implementation (cuRAND's Philox4_32_10) are in
``test_oracle_philox_curand.py`` (host generator, CPU) and
``test_gpu_philox_curand_device.py`` (device API); here: statistics, avalanche and
structure.
"""
import numpy as np

from oracle.philox import (box_muller, branch_draw, move_draws, philox4x32_10,
                           seed_key, to_unit)


def _block(n, key=(0, 0), lane=0):
    c = np.arange(n, dtype=np.uint64)
    ctr = [np.zeros(n, np.uint64)] * 4
    ctr = list(ctr)
    ctr[lane] = c
    return philox4x32_10(ctr, key)


def test_uniform_moments_and_chi2():
    w = np.concatenate(_block(1 << 18, key=(12345, 678)))
    u = to_unit(w)
    assert 0.0 < u.min() and u.max() < 1.0
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5e-3 / np.sqrt(n / 1e4)
    counts = np.bincount((u * 64).astype(int), minlength=64)
    chi2 = ((counts - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)        # ~6 sigma


def test_every_output_word_and_counter_lane_is_random():
    for lane in range(4):
        words = _block(1 << 14, key=(7, 9), lane=lane)
        for w in words:
            bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 32).mean(0)
            assert np.all(np.abs(bits - 0.5) < 0.03)


def test_avalanche_single_bit_flips():
    rng = np.random.default_rng(1)
    base = rng.integers(0, 2 ** 32, size=(4, 2048), dtype=np.uint64)
    out0 = np.stack(philox4x32_10(list(base), (0xDEADBEEF, 0x1234)))
    for lane in range(4):
        for bit in (0, 13, 31):
            flipped = base.copy()
            flipped[lane] ^= np.uint64(1 << bit)
            out1 = np.stack(philox4x32_10(list(flipped), (0xDEADBEEF, 0x1234)))
            diff = np.unpackbits((out0 ^ out1).astype(np.uint32).view(np.uint8)).mean()
            assert abs(diff - 0.5) < 0.02
    # the key matters too
    out2 = np.stack(philox4x32_10(list(base), (0xDEADBEEF, 0x1235)))
    assert abs(np.unpackbits((out0 ^ out2).astype(np.uint32).view(np.uint8)).mean() - 0.5) < 0.02


def test_vectorised_words_match_python_integers():
    """Not a pin of the definition (it restates it): checks that the vectorised uint64
    arithmetic (masking, 32x32->64 products, shifts) matches unbounded Python integers."""
    M0, M1 = 0xD2511F53, 0xCD9E8D57
    W0, W1 = 0x9E3779B9, 0xBB67AE85
    c = [0x01234567, 0x89ABCDEF, 0x0F1E2D3C, 0x4B5A6978]
    k = [0x11111111, 0x22222222]
    x = list(c)
    kk = list(k)
    for r in range(10):
        if r:
            kk = [(kk[0] + W0) & 0xFFFFFFFF, (kk[1] + W1) & 0xFFFFFFFF]
        p0, p1 = M0 * x[0], M1 * x[2]
        x = [(p1 >> 32) ^ x[1] ^ kk[0], p1 & 0xFFFFFFFF, (p0 >> 32) ^ x[3] ^ kk[1], p0 & 0xFFFFFFFF]
    got = [int(v) for v in philox4x32_10(c, k)]
    assert got == x


def test_box_muller_normal_moments():
    xi, u = move_draws(3, 5, np.arange(40000), 17)
    assert xi.shape == (40000, 3)
    for d in range(3):
        g = xi[:, d]
        assert abs(g.mean()) < 0.03
        assert abs(g.var() - 1) < 0.03
        assert abs(((g - g.mean()) ** 4).mean() / g.var() ** 2 - 3) < 0.15
    assert abs(np.corrcoef(xi[:, 0], xi[:, 2])[0, 1]) < 0.03
    assert abs(u.mean() - 0.5) < 0.01


def test_draws_depend_on_every_counter_field():
    a = move_draws(0, 1, 2, 3)
    for args in [(1, 1, 2, 3), (0, 2, 2, 3), (0, 1, 3, 3), (0, 1, 2, 4)]:
        b = move_draws(*args)
        assert not np.allclose(a[0], b[0]) and a[1] != b[1]
    assert branch_draw(0, 1, 3) != branch_draw(0, 1, 4)
    assert seed_key((5 << 32) | 7) == (7, 5)
    r, s = box_muller(np.array([np.exp(-0.5)]), np.array([0.25]))
    assert abs(r[0]) < 1e-15 and abs(s[0] - 1.0) < 1e-15
