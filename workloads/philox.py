"""Counter-based normal start blocks: the host-side definition of the block
that the C ABI's solve draws when it is given no start block.

Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC 2011).  A 128-bit counter (c0, c1, c2, c3)
and a 64-bit key (k0, k1) go through ten rounds; one round multiplies c0 and
c2 by the constants M0 and M1 (full 64-bit products split into hi / lo
words) and mixes

    (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),

and the key is bumped by the Weyl constants (W0, W1) between rounds.

Normals (this library's convention): block element e (column-major, e = i +
n j) belongs to pair p = e // 2 (real) or p = e (complex).  The pair's counter
is (p mod 2^32, p // 2^32, 0, 0), the key is (seed mod 2^32, seed // 2^32).  The
four output words give two uniforms in (0, 1) with 53 random bits each,

    u1 = ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) 2^-53,   u2 from (x2, x3) likewise,

and Box-Muller gives z0 = r cos(2 pi u2), z1 = r sin(2 pi u2) with
r = sqrt(-2 ln u1).  A real element takes z0 (even e) or z1 (odd e); a complex
element is (z0 s, z1 s) with s the double nearest 1 / sqrt(2).

This module holds no arithmetic of the eigensolver.  It is only the
definition of an input.
"""
from __future__ import annotations

import math

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
INV_SQRT2 = 0.70710678118654752440   # 1 / sqrt(2), the nearest double


def philox4x32(ctr, key, rounds: int = 10):
    """Philox4x32 of counters ``ctr`` (uint32 array [..., 4]) under ``key``
    (two ints); returns uint32 [..., 4]."""
    c = [np.asarray(ctr, dtype=np.uint64)[..., i] for i in range(4)]
    k0, k1 = np.uint64(key[0] & 0xFFFFFFFF), np.uint64(key[1] & 0xFFFFFFFF)
    for r in range(rounds):
        if r:
            k0 = (k0 + np.uint64(W0)) & _MASK
            k1 = (k1 + np.uint64(W1)) & _MASK
        p0 = c[0] * np.uint64(M0)          # < 2^64: exact in uint64
        p1 = c[2] * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1).astype(np.uint32)


def normal_pairs(count: int, seed: int):
    """z0, z1 (float64 arrays of length ``count``) of pairs 0 .. count-1."""
    p = np.arange(count, dtype=np.uint64)
    ctr = np.zeros((count, 4), dtype=np.uint64)
    ctr[:, 0] = p & _MASK
    ctr[:, 1] = p >> np.uint64(32)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    x = philox4x32(ctr, (seed & 0xFFFFFFFF, seed >> 32)).astype(np.float64)
    u1 = (np.floor(x[:, 0] / 32.0) * 67108864.0 + np.floor(x[:, 1] / 64.0) + 0.5) * 2.0 ** -53
    u2 = (np.floor(x[:, 2] / 32.0) * 67108864.0 + np.floor(x[:, 3] / 64.0) + 0.5) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    return r * np.cos(t), r * np.sin(t)


def start_block_seeded(n: int, m: int, seed: int, complex_: bool = False) -> np.ndarray:
    """The n x m start block (returned as the C-contiguous m x n array, the
    column-major storage the C ABI uses) drawn for ``seed``."""
    ne = n * m
    if complex_:
        z0, z1 = normal_pairs(ne, seed)
        X = np.empty(ne, dtype=np.complex128)
        X.real = z0 * INV_SQRT2
        X.imag = z1 * INV_SQRT2
    else:
        z0, z1 = normal_pairs((ne + 1) // 2, seed)
        X = np.empty(ne)
        X[0::2] = z0[: (ne + 1) // 2]
        X[1::2] = z1[: ne // 2]
    return X.reshape(m, n)
