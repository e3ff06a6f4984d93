"""Philox4x32-10 counter-based generator for the QMCUR oracle.

TEST INFRASTRUCTURE ONLY (see oracle/quat.py).

The paper draws its column and row indices "based on the sampling
probability" (Algorithm 1, steps 1-2) without naming a generator.  Both the
oracle and the CUDA library therefore implement the same published
counter-based generator, Philox4x32 with 10 rounds (Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), each from that
definition, so that index draws can be compared bit for bit.

One round maps counter (c0, c1, c2, c3) and key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the
Weyl constants (0x9E3779B9, 0xBB67AE85).  Parity: pinned against the
generator's published known-answer vectors (tests/golden/philox4x32_10_kat.txt).
"""
import numpy as np

_MASK = 0xFFFFFFFF
_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85


def philox4x32_10(counter, key):
    """One block: counter = 4 uint32, key = 2 uint32 -> 4 uint32 (Python ints)."""
    c0, c1, c2, c3 = (int(v) & _MASK for v in counter)
    k0, k1 = (int(v) & _MASK for v in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 32, p0 & _MASK
        hi1, lo1 = p1 >> 32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def philox4x32_10_vec(c0, c1, c2, c3, k0, k1):
    """Vectorised form over numpy uint64 arrays holding 32-bit values."""
    m = np.uint64(_MASK)
    c0 = np.asarray(c0, dtype=np.uint64) & m
    c1 = np.asarray(c1, dtype=np.uint64) & m
    c2 = np.asarray(c2, dtype=np.uint64) & m
    c3 = np.asarray(c3, dtype=np.uint64) & m
    k0 = np.uint64(int(k0) & _MASK)
    k1 = np.uint64(int(k1) & _MASK)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + _W0) & _MASK)
            k1 = np.uint64((int(k1) + _W1) & _MASK)
        p0 = np.uint64(_M0) * c0
        p1 = np.uint64(_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & m
        hi1, lo1 = p1 >> np.uint64(32), p1 & m
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3
