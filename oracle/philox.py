"""Oracle: the counter-based generator that defines the Gaussian test matrix Omega.

Algorithm 1 (step 1) draws an n x l matrix of independent N(0, 1) entries.  So that
the CUDA path and this oracle see the same Omega without passing it around, both
sides implement Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC 2011) from its published definition, each in its
own code, and turn its output into normals with the Box-Muller transform.

Definition of Omega[g, j] (global vertex row g, column j), seed s (64-bit):
    x = Philox4x32-10(counter = (g, j >> 1, 0x4F6D6567, 0), key = (s mod 2^32, s >> 32))
    u1 = ((x0 >> 5) * 2^26 + (x1 >> 6) + 1/2) * 2^-53          in (0, 1)
    u2 = ((x2 >> 5) * 2^26 + (x3 >> 6) + 1/2) * 2^-53
    Omega[g, j] = sqrt(-2 ln u1) * (cos(2 pi u2) if j even else sin(2 pi u2))
A tessellation block b uses rows block_ptr[b] .. block_ptr[b+1]-1 of the same Omega,
so the matrix does not depend on how the vertices are tessellated.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
OMEGA_STREAM = 0x4F6D6567


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit counters with a 64-bit key.

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (full 64-bit products);
    new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0).  Between rounds the key
    is bumped by the Weyl constants (k0 += W0, k1 += W1, mod 2^32).
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
    return c0, c1, c2, c3


def _unit53(a, b):
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    v = (a >> np.uint64(5)).astype(np.float64) * 67108864.0 + (b >> np.uint64(6)).astype(np.float64)
    return (v + 0.5) * (2.0 ** -53)


def omega(rows: np.ndarray, l: int, seed: int) -> np.ndarray:
    """Omega[g, j] for the given global rows g and columns 0..l-1 (float64)."""
    rows = np.asarray(rows, dtype=np.uint64)
    g = np.repeat(rows, l)
    j = np.tile(np.arange(l, dtype=np.uint64), rows.size)
    x0, x1, x2, x3 = philox4x32_10(g, j >> np.uint64(1), np.uint64(OMEGA_STREAM), 0,
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1 = _unit53(x0, x1)
    u2 = _unit53(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    z = np.where((j & np.uint64(1)) == 0, r * np.cos(ang), r * np.sin(ang))
    return z.reshape(rows.size, l)
