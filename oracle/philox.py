"""Philox4x32-10 counter-based generator (oracle side).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

Written from the published definition of Philox4x32 with 10 rounds
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11): each round multiplies counter words 0 and 2 by two fixed 32-bit
constants, keeps the high and low halves, mixes the high halves with the other
two counter words and the key by XOR, and bumps the key by two Weyl constants
between rounds.  The synthetic inputs of this project (Sec. 8 structural
properties of H and S) draw every random value from this generator keyed by
the seed, with the counter (index_lo, index_hi, stream, 0).

Conversions (this project's definition, used identically by the library):
  uniform u in [0,1): 53 bits from the 64-bit word (w0 << 32 | w1) >> 11
  normal: sqrt(-2 ln(1 - u_a)) * cos(2 pi u_b), u_a from (w0,w1), u_b from (w2,w3)
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
SHIFT32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  All arguments are uint32-valued arrays/scalars.

    Returns four uint64 arrays holding the 32-bit output words.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0          # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> SHIFT32, p0 & MASK32
        hi1, lo1 = p1 >> SHIFT32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32)


def _u53(a, b):
    return (((a << SHIFT32) | b) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def draws(seed: int, stream: int, index):
    """(u_a, u_b) uniforms in [0,1) for draw indices `index` of `stream`."""
    idx = np.asarray(index, dtype=np.uint64)
    k0, k1 = _key(seed)
    w0, w1, w2, w3 = philox4x32_10(idx & MASK32, idx >> SHIFT32, np.uint64(stream), np.uint64(0),
                                   k0, k1)
    return _u53(w0, w1), _u53(w2, w3)


def uniform(seed: int, stream: int, index) -> np.ndarray:
    return draws(seed, stream, index)[0]


def normal(seed: int, stream: int, index) -> np.ndarray:
    ua, ub = draws(seed, stream, index)
    return np.sqrt(-2.0 * np.log(1.0 - ua)) * np.cos(2.0 * np.pi * ub)
