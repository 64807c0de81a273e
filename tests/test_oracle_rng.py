"""Pins of the oracle's noise source (Philox-4x32-10 + Box-Muller).

The paper draws iid N(0,1) per face and step (Sec. 3, Eq. (3.7)); the
generator is this library's choice.  The oracle's generator is pinned here by
the known-answer vectors its authors publish for Philox-4x32-10 (Salmon,
Moraes, Dror, Shaw, SC'11, Random123 distribution) and by properties the
mathematics fixes -- independent of its code: uniformity of the raw 32-bit
words, the N(0,1) law of the deviates (moments and a KS test against scipy's
normal CDF), independence between slots and neighbouring counters, and
distinct blocks for distinct counters.  The GPU generator is compared against
this one bit for bit in the GPU tests.
"""
import numpy as np
import pytest
import scipy.stats

from oracle import she


def _blocks(n, seed=0, c1=0, c2=0, c3=0):
    return np.array([she.philox([i, c1, c2, c3], [seed & 0xFFFFFFFF, seed >> 32])
                     for i in range(n)], dtype=np.uint64)


# (counter, key) -> output of Philox-4x32-10, the published known answers
KNOWN_ANSWERS = [
    ([0x00000000, 0x00000000, 0x00000000, 0x00000000], [0x00000000, 0x00000000],
     [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
    ([0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff], [0xffffffff, 0xffffffff],
     [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
    ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
]


@pytest.mark.parametrize("ctr,key,out", KNOWN_ANSWERS)
def test_philox_known_answers(ctr, key, out):
    assert [int(x) for x in she.philox(ctr, key)] == out


def test_philox_words_uniform():
    b = _blocks(20000, seed=7, c1=3, c2=11)
    top = (b >> 28).ravel()                      # 16 bins from the top 4 bits
    counts = np.bincount(top.astype(np.int64), minlength=16)
    chi2, p = scipy.stats.chisquare(counts)
    assert p > 1e-4, (chi2, p)
    low = (b & 0xF).ravel()                      # low bits too
    chi2, p = scipy.stats.chisquare(np.bincount(low.astype(np.int64), minlength=16))
    assert p > 1e-4, (chi2, p)
    # every output bit is set about half the time
    bits = np.array([(b >> k) & 1 for k in range(32)], dtype=np.float64).mean(axis=(1, 2))
    assert np.all(np.abs(bits - 0.5) < 0.01)


def test_philox_distinct_counters_and_keys():
    b = _blocks(4096, seed=1)
    assert len({tuple(r) for r in b}) == 4096
    # changing only the key, the step word, or the tag changes the block
    base = she.philox([5, 6, 7, 8], [9, 10])
    assert she.philox([5, 6, 7, 8], [9, 11]) != base
    assert she.philox([5, 7, 7, 8], [9, 10]) != base
    assert she.philox([5, 6, 7, 9], [9, 10]) != base


def test_normals_law():
    z = np.array([she.normals4(123, i, 4, 5, 0) for i in range(25000)]).ravel()
    assert abs(z.mean()) < 4.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4.0 * np.sqrt(2.0 / z.size)
    # third and fourth moments of N(0,1): 0 and 3
    assert abs(np.mean(z ** 3)) < 4.0 * np.sqrt(15.0 / z.size)
    assert abs(np.mean(z ** 4) - 3.0) < 4.0 * np.sqrt(96.0 / z.size)
    d, p = scipy.stats.kstest(z, "norm")
    assert p > 1e-4, (d, p)


def test_normals_slots_independent():
    z = np.array([she.normals4(99, i, 0, 2, 0) for i in range(25000)])
    c = np.corrcoef(z.T)
    off = c[~np.eye(4, dtype=bool)]
    assert np.all(np.abs(off) < 5.0 / np.sqrt(z.shape[0]))
    # the two deviates of one Box-Muller pair share a radius: their squares
    # sum to a chi^2 with 2 degrees of freedom (exponential, mean 2)
    s = z[:, 0] ** 2 + z[:, 1] ** 2
    d, p = scipy.stats.kstest(s / 2.0, "expon")
    assert p > 1e-4


def test_normal_index_addressing():
    # normal g is slot g%4 of the block at counter g/4
    blk = she.normals4(3, 10, 20, 30, 0)
    for s in range(4):
        assert she.normal(3, 40 + s, 20, 30, 0) == blk[s]
    # the high-wall normal of step n is slot n%4 of counter (0, n/4, stream, 2)
    blk = she.normals4(3, 0, 5, 30, 2)
    for s in range(4):
        assert she.wall_normal(3, 20 + s, 30) == blk[s]


@pytest.mark.parametrize("tag", [0, 1, 2])
def test_tags_give_independent_streams(tag):
    a = np.array([she.normals4(0, i, 0, 0, tag) for i in range(5000)]).ravel()
    b = np.array([she.normals4(0, i, 0, 0, (tag + 1) % 3) for i in range(5000)]).ravel()
    assert abs(np.corrcoef(a, b)[0, 1]) < 5.0 / np.sqrt(a.size)
