"""Philox4x32-10 counter-based generator, vectorised with numpy.

Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter is pushed through ten rounds;
each round multiplies counter words 0 and 2 by two fixed 32-bit constants, swaps the
high/low halves of the products with words 1 and 3 xor-ed with the round key, and the
two-word key is bumped by two Weyl constants between rounds.

This module holds no decoder arithmetic: it only turns (key, counter) into uniform
32-bit words for the seeded input generators.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(c0, c1, c2, c3, k0: int, k1: int, rounds: int = 10):
    """Return the four 32-bit output words for counters (c0..c3) under key (k0, k1).

    Counters may be numpy arrays (broadcast together) or scalars; outputs are uint32 arrays.
    """
    x0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    x1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    x2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    x3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    x0 = x0.copy(); x1 = x1.copy(); x2 = x2.copy(); x3 = x3.copy()
    key0 = int(k0) & 0xFFFFFFFF
    key1 = int(k1) & 0xFFFFFFFF
    for _ in range(rounds):
        p0 = PHILOX_M0 * x0
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        n0 = hi1 ^ x1 ^ np.uint64(key0)
        n2 = hi0 ^ x3 ^ np.uint64(key1)
        x0, x1, x2, x3 = n0, lo1, n2, lo0
        key0 = (key0 + PHILOX_W0) & 0xFFFFFFFF
        key1 = (key1 + PHILOX_W1) & 0xFFFFFFFF
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


def seed_key(seed: int) -> tuple[int, int]:
    """Split a 64-bit seed into the two Philox key words."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


class PhiloxStream:
    """Sequential draws from one Philox stream: counter (n, stream_id, 0, 0), n = 0, 1, ...

    Each counter yields four 32-bit words, consumed in order (word 0 first).  Used for the
    small, order-dependent draws of the graph generator.
    """

    def __init__(self, seed: int, stream_id: int):
        self.k0, self.k1 = seed_key(seed)
        self.stream_id = int(stream_id)
        self.block = 0
        self.buf: list[int] = []

    def next_u32(self) -> int:
        if not self.buf:
            w = philox4x32(self.block, self.stream_id, 0, 0, self.k0, self.k1)
            self.buf = [int(w[0]), int(w[1]), int(w[2]), int(w[3])]
            self.block += 1
        return self.buf.pop(0)

    def uniform_int(self, n: int) -> int:
        """Integer in [0, n): high word of the 64-bit product u32 * n (multiply-shift)."""
        return (self.next_u32() * int(n)) >> 32
