"""Philox4x32-10 counter-based generator and the draws of one proposed move.

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4-word counter is passed
through ten rounds; each round multiplies words 0 and 2 by two fixed 32-bit constants,
takes the high and low halves of the 64-bit products and mixes them with the other two
words and the 2-word key, and the key is bumped by two Weyl constants between rounds.

The paper (Sec. "Trial Moves", Eq. trans_prob_alle and the particle-by-particle
transition density) draws the trial displacement of one electron from a 3D Gaussian
and accepts with a uniform variate. The counter layout below is an adopted reading
(the paper does not say how random numbers are drawn):

* move of electron e of walker w in sweep t: block (t, e, w, 0) gives three normals by
  Box-Muller on words (0, 1) and (2, 3) (the second pair's sine output is unused);
  block (t, e, w, 1) word 0 gives the acceptance variate u;
* DMC branching of walker w at step t: block (t, 0xB, w, 2) word 0;
* a word w maps to the open interval (0, 1) as (w + 0.5) * 2**-32.

Pins: bit-exact agreement with an independent implementation, the Philox4_32_10 generator
of NVIDIA's cuRAND library, run (never disassembled) at matching key and counter: its host
generator on the CPU covers counter words 0-2 and the key schedule
(tests/test_oracle_philox_curand.py), its device API on the GPU covers counter word 3
(tests/test_gpu_philox_curand_device.py); plus uniformity and independence statistics.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(ctr, key):
    """Ten Philox rounds. ``ctr`` is 4 broadcastable integer arrays, ``key`` 2 integers.
    Returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in ctr)
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def seed_key(seed: int):
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def to_unit(word) -> np.ndarray:
    """Map 32-bit words to (0, 1): (w + 0.5) * 2^-32 (exact in double precision)."""
    return (np.asarray(word, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(u1, u2):
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return r * np.cos(ang), r * np.sin(ang)


def move_draws(seed: int, sweep: int, electron, walker_id):
    """Gaussian displacement xi (..., 3) and acceptance variate u (...) of the moves of
    ``electron`` in walkers ``walker_id`` during sweep ``sweep``."""
    key = seed_key(seed)
    w0, w1, w2, w3 = philox4x32_10((sweep, electron, walker_id, 0), key)
    gx, gy = box_muller(to_unit(w0), to_unit(w1))
    gz, _ = box_muller(to_unit(w2), to_unit(w3))
    b0, _, _, _ = philox4x32_10((sweep, electron, walker_id, 1), key)
    return np.stack([gx, gy, gz], -1), to_unit(b0)


def comb_draw(seed: int, step: int):
    """Uniform offset of the comb of one stochastic reconfiguration step (Sec. "Diffusion
    Monte Carlo"), one per system and step: block (step, 0xC, 0, 2) word 0."""
    w0, _, _, _ = philox4x32_10((step, 0xC, 0, 2), seed_key(seed))
    return to_unit(w0)


def branch_draw(seed: int, step: int, walker_id):
    """Uniform variate of the branching decision M = floor(w + xi) (Sec. "Diffusion
    Monte Carlo")."""
    w0, _, _, _ = philox4x32_10((step, 0xB, walker_id, 2), seed_key(seed))
    return to_unit(w0)
