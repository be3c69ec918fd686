"""Philox4x32-10 counter-based random numbers, vectorised over counters.

Philox is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC 2011).  A 4x32-bit counter
and a 2x32-bit key go through ten rounds; each round multiplies two counter
words by fixed odd constants, splits the 64-bit products into high and low
halves and mixes them with the other two words and the key.  The key is bumped
by two Weyl constants between rounds.

Because any output block is a pure function of (key, counter), every row of
a synthetic MDP can be regenerated on its own, in any order, on any machine.
This module holds only random-number plumbing: no MDP arithmetic.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)
_SHIFT32 = np.uint64(32)


def philox4x32(counter, key, rounds: int = 10):
    """Apply Philox4x32-R to counters.

    counter: sequence of four integer arrays (broadcastable), the words c0..c3.
    key: sequence of two integers or arrays, the words k0, k1.
    Returns a tuple of four uint32 arrays.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK32 for c in counter)
    k0 = np.asarray(key[0], dtype=np.uint64) & _MASK32
    k1 = np.asarray(key[1], dtype=np.uint64) & _MASK32
    for r in range(rounds):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _SHIFT32, p0 & _MASK32
        hi1, lo1 = p1 >> _SHIFT32, p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r + 1 < rounds:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


def uniform53(hi_word, lo_word):
    """Map two uint32 words to a double in [0, 1) with 53 random bits.

    The top 27 bits of the first word and the top 26 bits of the second form
    a 53-bit integer m; the result is m * 2**-53, exact in binary64.
    """
    a = np.asarray(hi_word, dtype=np.uint64) >> np.uint64(5)
    b = np.asarray(lo_word, dtype=np.uint64) >> np.uint64(6)
    m = a * np.uint64(1 << 26) + b
    return m.astype(np.float64) * (2.0 ** -53)


def stream(seed: int, tag: int, row, block, lane: int = 0):
    """Uniform doubles in [0, 1) for (row, block) counters of one stream.

    seed, tag: the key (generator seed and a per-purpose stream tag).
    row: integer array of row indices (up to 2**64).
    block: integer array (broadcast against row) of draw indices within a row.
    lane: 0 or 1, which pair of output words to use.
    """
    row = np.asarray(row, dtype=np.uint64)
    block = np.asarray(block, dtype=np.uint64)
    row, block = np.broadcast_arrays(row, block)
    out = philox4x32(
        (row & _MASK32, row >> _SHIFT32, block & _MASK32, block >> _SHIFT32),
        (seed, tag),
    )
    if lane == 0:
        return uniform53(out[0], out[1])
    return uniform53(out[2], out[3])
