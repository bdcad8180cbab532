"""CPU check of the invariant-divisor division the histogram kernels use to
turn a 16-byte chunk index into its row (hist_common.cuh: make_fastdiv and
fastdiv).  The method is the round-up multiply-and-shift division of Granlund
and Montgomery ("Division by invariant integers using multiplication", PLDI
1994, Sec. 4): for a 32-bit divisor d with l = ceil(log2 d),
m' = floor(2^32 (2^l - d) / d) + 1, and for every 32-bit n
    t = floor(m' n / 2^32),  q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0)
equals floor(n / d).  This file restates the host and device code in exact
integer arithmetic (32-bit wrap where the device wraps) and checks the
quotient against Python's floor division: over every n below 2^22 for small
divisors, and for every divisor a row of chunks can have at quotient
boundaries k d - 1 and k d (the first 39 k, 40 random ones and the last two)
and at the top of the 32-bit range."""

import numpy as np
import pytest

M32 = (1 << 32) - 1


def make_fastdiv(d):
    l = 0
    while l < 32 and (1 << l) < d:
        l += 1
    m = ((1 << 32) * ((1 << l) - d)) // d + 1
    assert 0 <= m <= M32                 # fits the 32-bit field it is stored in
    return d, m, min(l, 1), max(l - 1, 0)


def fastdiv(n, f):
    _, m, s1, s2 = f
    t = (m * n) >> 32                    # __umulhi
    return ((t + (((n - t) & M32) >> s1)) & M32) >> s2


def fastdiv_np(n, f):
    _, m, s1, s2 = f
    n = n.astype(np.uint64)
    t = (np.uint64(m) * n) >> np.uint64(32)
    return (((t + (((n - t) & np.uint64(M32)) >> np.uint64(s1))) & np.uint64(M32)) >> np.uint64(s2))


@pytest.mark.parametrize("d", list(range(1, 40)) + [255, 256, 257, 1000])
def test_every_numerator_below_2_to_22(d):
    f = make_fastdiv(d)
    n = np.arange(1 << 22, dtype=np.uint64)
    assert (fastdiv_np(n, f) == n // np.uint64(d)).all()


def test_quotient_boundaries_for_every_row_of_chunks():
    # rows of up to 2^20 columns: 1 .. 65536 chunks of 16 bytes; numerators at
    # every quotient boundary a chunk index can reach, and the 32-bit extremes
    rng = np.random.default_rng(0)
    for d in list(range(1, 65537)):
        f = make_fastdiv(d)
        k = np.unique(np.concatenate([np.arange(1, 40), rng.integers(1, M32 // d + 1, 40),
                                      [M32 // d, M32 // d - 1]])).astype(np.uint64)
        k = k[(k >= 1) & (k * np.uint64(d) <= np.uint64(M32))]
        n = np.concatenate([k * np.uint64(d) - np.uint64(1), k * np.uint64(d),
                            np.array([0, M32, M32 - 1], dtype=np.uint64)])
        assert (fastdiv_np(n, f) == n // np.uint64(d)).all(), d


def test_divisors_at_powers_of_two_and_large():
    ds = [1, 2, 3] + [(1 << p) + e for p in range(2, 32) for e in (-1, 0, 1)] + [M32, M32 - 1, (1 << 31) + 12345]
    for d in ds:
        f = make_fastdiv(d)
        for n in (0, 1, d - 1, d, d + 1, 2 * d - 1, 2 * d, M32 - 1, M32, M32 // 2, (M32 // d) * d, (M32 // d) * d - 1):
            if 0 <= n <= M32:
                assert fastdiv(n, f) == n // d, (d, n)


def test_a_wrong_multiplier_fails():
    # the check is not vacuous: the multiplier without its + 1 breaks it
    d = 7
    _, m, s1, s2 = make_fastdiv(d)
    bad = (d, m - 1, s1, s2)
    n = np.arange(1 << 20, dtype=np.uint64)
    assert not (fastdiv_np(n, bad) == n // np.uint64(d)).all()
