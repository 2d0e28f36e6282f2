"""Counter-based Gaussian sampling for the oracle (test infrastructure only).

The Gaussian test matrices Omega of Algorithms 2 and 3 are drawn from a
counter-based generator so that the oracle and the CUDA path see the same random
numbers without passing them around.  Both sides implement the same published
definition independently:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
  1, 2, 3", SC'11): a 4x32-bit counter and a 2x32-bit key; each of 10 rounds
  multiplies words 0 and 2 by the constants M0, M1 (full 64-bit products split
  into hi/lo halves) and mixes as
      (x0, x1, x2, x3) <- (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0))
  with the key bumped by the Weyl constants (W0, W1) between rounds.
* Box-Muller: g0 = sqrt(-2 ln u1) cos(2 pi u2), g1 = sqrt(-2 ln u1) sin(2 pi u2).

Stream layout (a choice of this implementation; the paper only asks for an n x w
Gaussian matrix): entry (j, col) of the block drawn in SVT iteration `it`, block
number `b`, uses counter (j, col // 2, it, b) and key (seed lo 32 bits, seed hi 32
bits); words (x0, x1) give u1 = (((x0 << 20) | (x1 >> 12)) + 0.5) * 2^-52 and
(x2, x3) give u2 the same way, so u1, u2 lie strictly inside (0, 1).  Even
columns take the cosine branch, odd columns the sine branch.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr: (..., 4) array of uint32 counters; key: pair of uint32.
    Returns the (..., 4) uint32 output words.
    """
    ctr = np.asarray(ctr, dtype=np.uint64)
    x0, x1, x2, x3 = (ctr[..., i] for i in range(4))
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    for _ in range(10):
        p0 = m0 * x0            # < 2^64: product of two 32-bit values
        p1 = m1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
        k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def _unit_open(hi, lo):
    """52 random bits from two words -> float64 strictly inside (0, 1)."""
    a = (hi.astype(np.uint64) << np.uint64(20)) | (lo.astype(np.uint64) >> np.uint64(12))
    return (a.astype(np.float64) + 0.5) * (2.0 ** -52)


def gaussian_block(seed: int, it: int, block: int, n: int, w: int) -> np.ndarray:
    """n x w block of standard normals for SVT iteration `it`, block `block`."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    key = (seed & 0xFFFFFFFF, seed >> 32)
    pairs = (w + 1) // 2
    j = np.repeat(np.arange(n, dtype=np.uint64), pairs)
    c = np.tile(np.arange(pairs, dtype=np.uint64), n)
    ctr = np.stack([j, c, np.full_like(j, it & 0xFFFFFFFF), np.full_like(j, block & 0xFFFFFFFF)],
                   axis=-1)
    x = philox4x32_10(ctr, key).reshape(n, pairs, 4)
    u1 = _unit_open(x[..., 0], x[..., 1])
    u2 = _unit_open(x[..., 2], x[..., 3])
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty((n, 2 * pairs), dtype=np.float64)
    out[:, 0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[:, 1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:, :w]
