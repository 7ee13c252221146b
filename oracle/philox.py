"""Philox4x32-10 counter-based generator, written from its published definition.

TEST INFRASTRUCTURE ONLY.  This module belongs to the CPU oracle: only tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.

Definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 4): a 128-bit counter (c0, c1, c2, c3) and a 64-bit key
(k0, k1) go through 10 rounds.  One round multiplies c0 and c2 by the constants
M0 and M1 into 64-bit products and permutes:

    (c0, c1, c2, c3) <- (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),
                         hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))

after which the key is bumped by the Weyl constants (W0, W1) before the next
round.  All words are 32-bit unsigned.  The implementation below works on numpy
uint64 arrays that hold 32-bit values, so a whole tensor of counters is
processed at once.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
ROUNDS = 10


def _u64(x):
    return np.asarray(x, dtype=np.uint64) & MASK32


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words (as uint64 arrays) for counters/keys.

    All arguments broadcast against each other.
    """
    c0, c1, c2, c3 = _u64(c0), _u64(c1), _u64(c2), _u64(c3)
    k0, k1 = _u64(k0), _u64(k1)
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0, k1 = k0.copy(), k1.copy()
    s32 = np.uint64(32)
    for _ in range(ROUNDS):
        p0 = M0 * c0           # < 2^64: both factors are < 2^32
        p1 = M1 * c2
        hi0, lo0 = p0 >> s32, p0 & MASK32
        hi1, lo1 = p1 >> s32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
        k0 = (k0 + W0) & MASK32
        k1 = (k1 + W1) & MASK32
    return c0, c1, c2, c3


def seed_key(seed):
    """Split a 64-bit seed into the Philox key words (k0 = low, k1 = high)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32)
