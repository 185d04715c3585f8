"""Philox4x32-10 counter-based generator, written from its published
definition (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11), with Box-Muller normals.  Test infrastructure only.

Stream layout used by the sampler (both implementations follow it):
  key     = (seed & 0xffffffff, seed >> 32)
  counter = (j, walker, step & 0xffffffff, step >> 32)
  uniform = (word + 0.5) * 2^-32, in (0, 1)
Each counter value j yields four words = two Box-Muller pairs = four normals:
normal m of a (walker, step) comes from block j = m // 4, words
(2*((m%4)//2), 2*((m%4)//2)+1), cosine branch for even m, sine for odd m.
The acceptance uniform of a step is word 0 of block j = ceil(3N/4).
Walker initialisation uses step = 2^64 - 1.
"""

from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF
INIT_STEP = (1 << 64) - 1


def philox4x32(c0, c1, c2, c3, k0, k1, rounds=10):
    """Vectorised over numpy uint64 arrays holding 32-bit values."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
        p0 = np.uint64(M0) * c0
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def to_uniform(w):
    return (np.asarray(w, dtype=np.float64) + 0.5) * 2.0 ** -32


def _block(seed, walkers, step, j):
    seed = int(seed)
    step = int(step)
    wv = np.asarray(walkers, dtype=np.uint64)
    z = np.zeros_like(wv)
    return philox4x32(z + np.uint64(j), wv, z + np.uint64(step & MASK), z + np.uint64(step >> 32),
                      seed & MASK, seed >> 32)


def normals(seed, walkers, step, n):
    """[len(walkers), n] standard normals."""
    walkers = np.asarray(walkers)
    out = np.empty((len(walkers), n))
    for j in range((n + 3) // 4):
        w = [to_uniform(x) for x in _block(seed, walkers, step, j)]
        for pair in range(2):
            u0, u1 = w[2 * pair], w[2 * pair + 1]
            rad = np.sqrt(-2.0 * np.log(u0))
            for k, val in ((0, rad * np.cos(2.0 * np.pi * u1)), (1, rad * np.sin(2.0 * np.pi * u1))):
                m = 4 * j + 2 * pair + k
                if m < n:
                    out[:, m] = val
    return out


def accept_uniform(seed, walkers, step, n_normals):
    return to_uniform(_block(seed, walkers, step, (n_normals + 3) // 4)[0])
