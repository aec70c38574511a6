"""Philox4x32-10 counter-based generator, written from its published
definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): a 4-word counter and a 2-word key; each of the 10 rounds
multiplies words 0 and 2 by fixed 32-bit constants, keeps the high and low
halves, permutes and mixes them with the other words and the round key; the
key is bumped by two Weyl constants between rounds.

Vectorised over numpy arrays of counters.  Used by the oracle to draw the
Z(4) noise of Sec. 1 (the paper leaves the generator open).
"""
import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for counters (c0..c3) and key (k0, k1).

    Counter words may be numpy arrays (broadcast together); key words are ints.
    """
    x0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    x1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    x2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    x3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    ka, kb = int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = x0 * PHILOX_M0
        p1 = x2 * PHILOX_M1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(ka), lo1, hi0 ^ x3 ^ np.uint64(kb), lo0)
        ka = (ka + PHILOX_W0) & 0xFFFFFFFF
        kb = (kb + PHILOX_W1) & 0xFFFFFFFF
    return (x0.astype(np.uint32), x1.astype(np.uint32), x2.astype(np.uint32), x3.astype(np.uint32))
