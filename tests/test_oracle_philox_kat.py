"""Pin of the oracle's Philox4x32-10 against the generator's published
known-answer vectors (tests/golden/philox4x32_10_kat.txt).

The paper names no generator for its index draws (Algorithm 1, steps 1-2), so
the pin is the generator's own definition: Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11), whose distribution
ships these counter/key -> output vectors.  The GPU index tests compare the
CUDA sampler bit for bit with this oracle, so this pin carries over to it.
"""
import os

import numpy as np
import pytest

from oracle import philox as P

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "philox4x32_10_kat.txt")


def _kat_lines():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x, 16) for x in line.split()]
            assert len(v) == 10, line
            rows.append((tuple(v[0:4]), tuple(v[4:6]), tuple(v[6:10])))
    return rows


def test_kat_file_has_the_published_vectors():
    rows = _kat_lines()
    assert len(rows) == 3
    # all-zero, all-ones and the pi-digit counter/key of the published test
    assert rows[0][0] == (0, 0, 0, 0) and rows[0][1] == (0, 0)
    assert rows[1][0] == (0xFFFFFFFF,) * 4 and rows[1][1] == (0xFFFFFFFF,) * 2
    assert rows[2][0] == (0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344)


@pytest.mark.parametrize("row", range(3))
def test_scalar_philox_matches_kat(row):
    ctr, key, want = _kat_lines()[row]
    assert P.philox4x32_10(ctr, key) == want


def test_vector_philox_matches_kat():
    for ctr, key, want in _kat_lines():
        out = P.philox4x32_10_vec(*[np.array([c], dtype=np.uint64) for c in ctr], key[0], key[1])
        assert tuple(int(o[0]) for o in out) == want


def _variant(counter, key, m0, m1, w0, w1, bump_first):
    """Philox with its constants or key schedule altered (a plausible slip)."""
    mask = 0xFFFFFFFF
    c0, c1, c2, c3 = counter
    k0, k1 = key
    for rnd in range(10):
        if rnd > 0 or bump_first:
            k0 = (k0 + w0) & mask
            k1 = (k1 + w1) & mask
        p0, p1 = m0 * c0, m1 * c2
        c0, c1, c2, c3 = (p1 >> 32) ^ c1 ^ k0, p1 & mask, (p0 >> 32) ^ c3 ^ k1, p0 & mask
    return c0, c1, c2, c3


def test_kat_rejects_plausible_slips():
    """Swapped multipliers, swapped Weyl constants or a key bumped before the
    first round each fail at least one known answer: the vectors pin every
    part of the round function."""
    rows = _kat_lines()
    right = (P._M0, P._M1, P._W0, P._W1, False)
    assert all(_variant(c, k, *right) == w for c, k, w in rows)
    for slip in ((P._M1, P._M0, P._W0, P._W1, False),
                 (P._M0, P._M1, P._W1, P._W0, False),
                 (P._M0, P._M1, P._W0, P._W1, True)):
        assert any(_variant(c, k, *slip) != w for c, k, w in rows)
