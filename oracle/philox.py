"""Philox4x32-10 counter-based generator (oracle, numpy).

Written from the published definition (J. K. Salmon, M. A. Moraes, R. O. Dror,
D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit
counter and a 2x32-bit key; each of 10 rounds multiplies counter words 0 and 2 by
0xD2511F53 and 0xCD9E8D57 and mixes the high/low halves with the other words and
the key; the key is advanced by the Weyl constants 0x9E3779B9, 0xBB67AE85 between
rounds.

Sampling points of the integrator are drawn from it (points are not generated
by the paper's program on the device; this is the stream layout both sides of
this project implement):

    key     = (seed mod 2^32, unit key)
    counter = (point index mod 2^32, point index div 2^32, iteration, q)

The four output words of counter q give coordinates 2q and 2q+1; each coordinate
takes 52 bits m = (hi << 20) | (lo >> 12) of a word pair (lo, hi) and becomes
u = (2m + 1) 2^-53, exactly representable and strictly inside (0, 1).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  All arguments uint32 arrays (broadcastable)."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0, k1 = k0.copy(), k1.copy()
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = (k0 + W0).astype(np.uint32)
                k1 = (k1 + W1).astype(np.uint32)
            p0 = M0 * c0.astype(np.uint64)
            p1 = M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def words_to_unit(lo, hi):
    """Two 32-bit words -> u = (2m+1) 2^-53 with m the 52-bit integer (hi << 20) | (lo >> 12)."""
    m = (hi.astype(np.uint64) << np.uint64(20)) | (lo.astype(np.uint64) >> np.uint64(12))
    return (2.0 * m.astype(np.float64) + 1.0) * 2.0 ** -53


def uniforms(seed, unit_key, iteration, first, count, dim):
    """Points ``first .. first+count-1`` of the (seed, unit, iteration) stream: shape (count, dim)."""
    idx = np.arange(first, first + count, dtype=np.uint64)
    lo = (idx & MASK32).astype(np.uint32)
    hi = (idx >> np.uint64(32)).astype(np.uint32)
    out = np.empty((count, dim))
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32(unit_key & 0xFFFFFFFF)
    for q in range((dim + 1) // 2):
        r0, r1, r2, r3 = philox4x32_10(lo, hi, np.uint32(iteration), np.uint32(q), k0, k1)
        out[:, 2 * q] = words_to_unit(r0, r1)
        if 2 * q + 1 < dim:
            out[:, 2 * q + 1] = words_to_unit(r2, r3)
    return out
