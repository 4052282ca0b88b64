"""Philox4x32-10 counter-based generator and the Rademacher sketch matrix
(oracle side; test infrastructure only).

Written from the published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.3): a 4x32-bit
counter is put through 10 rounds; each round multiplies words 0 and 2 by the
constants 0xD2511F53 and 0xCD9E8D57 into 64-bit products, and forms the next
counter as (hi(c2*M1) ^ c1 ^ k0, lo(c2*M1), hi(c0*M0) ^ c3 ^ k1, lo(c0*M0));
between rounds the 2x32-bit key is bumped by the Weyl constants
(0x9E3779B9, 0xBB67AE85).

The sketch matrix the randomized range finder draws (the paper's randUTV
reference, Sec. 2.2 and 3.3) is defined here as: key = (seed lo, seed hi),
counter = (row i, column block j // 128, sweep step k, purpose); the 128 output
bits give the signs of columns 128*(j//128) .. +127 of row i, bit b of word w
for column 32*w + b, and Omega(i, j) = +1 if that bit is 0 else -1.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 over arrays of counters (uint32); returns 4 uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint32).copy() for x in (c0, c1, c2, c3)]
    c = np.broadcast_arrays(*c)
    c = [x.astype(np.uint32) for x in c]
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint32((int(k0) + int(W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(W1)) & 0xFFFFFFFF)
        p0 = c[0].astype(np.uint64) * M0
        p1 = c[2].astype(np.uint64) * M1
        hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
        lo0 = (p0 & MASK32).astype(np.uint32)
        hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
        lo1 = (p1 & MASK32).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


SKETCH_PURPOSE = 0


def rademacher(rows, cols, seed, step, purpose=SKETCH_PURPOSE):
    """Omega (rows x cols, FP64, entries +-1) as defined in the module docstring."""
    seed = int(seed)
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    nblk = (cols + 127) // 128
    i = np.arange(rows, dtype=np.uint64)[:, None]
    jb = np.arange(nblk, dtype=np.uint64)[None, :]
    ii = np.broadcast_to(i, (rows, nblk))
    jj = np.broadcast_to(jb, (rows, nblk))
    words = philox4x32_10(ii & MASK32, jj & MASK32, np.full((rows, nblk), step & 0xFFFFFFFF),
                          np.full((rows, nblk), purpose & 0xFFFFFFFF), k0, k1)
    out = np.empty((rows, nblk * 128))
    for w in range(4):
        for b in range(32):
            bit = (words[w] >> np.uint32(b)) & np.uint32(1)
            out[:, np.arange(nblk) * 128 + 32 * w + b] = 1.0 - 2.0 * bit
    return out[:, :cols]
