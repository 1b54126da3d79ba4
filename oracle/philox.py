"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy
as 1, 2, 3", SC'11).  TEST INFRASTRUCTURE ONLY (see oracle/__init__).

Written from the published definition: ten rounds; each round multiplies
counter words 0 and 2 by the two round constants (full 64-bit products), and
builds the new counter from the high halves xor-ed with the other counter
words and the key, and the low halves; the key is bumped by the two Weyl
constants between rounds.  Vectorised over counters with numpy; each lane is
one independent Philox call.
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for counters (c0..c3) and key (k0, k1).

    All arguments are broadcastable integer arrays (values < 2^32); returns a
    tuple of four uint64 arrays holding 32-bit values.
    """
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3)]
    c = np.broadcast_arrays(*c)
    c = [x.copy() for x in c]
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = c[0] * np.uint64(M0)          # < 2^64: exact in uint64
        p1 = c[2] * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return tuple(c)
