"""Pins for the oracle's counter-based generator (Philox4x32-10).

The paper does not name its generator (Sec. 4, Fig. 2 discussion), so the
draws are our reading: Philox4x32-10 from Salmon et al. (SC'11).  The pins are
(a) the published known-answer vectors of Philox4x32-10 (the Random123
library's test file that accompanies Salmon et al.; tests/golden/
philox4x32_10_kat.txt), (b) a second implementation written here in pure
Python integer arithmetic from that paper's description, (c) the exact
uniform mapping, and (d) statistical properties of the stream.  What the
known answers do not fix is our own layout of the draws (which counter word
carries the event index, which draw comes from which output word); that is
a documented choice, checked on the GPU bit for bit against the oracle.
"""
import os
import math
import random

import numpy as np
import pytest
from scipy import stats

M32 = 0xFFFFFFFF


def philox_py(ctr, key, rounds=10):
    """Philox4x32: S-box = two 32x32 multiplies, P-box = fixed word swap,
    key schedule = Weyl sequence (golden ratio, sqrt(3)-1)."""
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for r in range(rounds):
        p0 = 0xD2511F53 * c0
        p1 = 0xCD9E8D57 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & M32, p1 & M32, ((p0 >> 32) ^ c3 ^ k1) & M32, p0 & M32
        k0 = (k0 + 0x9E3779B9) & M32
        k1 = (k1 + 0xBB67AE85) & M32
    return [c0, c1, c2, c3]


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            w = [int(x, 16) for x in line]
            assert len(w) == 10
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    # Salmon et al.'s published known answers pin the round function (the two
    # multipliers and which lane each one takes), the output word permutation
    # and the key schedule (Weyl increments, bumped after each round): a slip
    # in any of them changes every output word.
    kat = load_kat()
    assert len(kat) == 3
    for ctr, key, expect in kat:
        assert orc.philox4x32_10(ctr, key) == expect, (ctr, key)
        assert philox_py(ctr, key) == expect


def test_philox_known_answers_reject_plausible_slips():
    # the pins must fail for the mistakes a restatement could make
    ctr, key, expect = load_kat()[2]

    def swapped_multipliers(c, k):
        c0, c1, c2, c3 = c
        k0, k1 = k
        for _ in range(10):
            p0, p1 = 0xCD9E8D57 * c0, 0xD2511F53 * c2
            c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & M32, p1 & M32, ((p0 >> 32) ^ c3 ^ k1) & M32, p0 & M32
            k0, k1 = (k0 + 0x9E3779B9) & M32, (k1 + 0xBB67AE85) & M32
        return [c0, c1, c2, c3]

    def key_bumped_first(c, k):
        return philox_py(c, [(k[0] + 0x9E3779B9) & M32, (k[1] + 0xBB67AE85) & M32])

    assert swapped_multipliers(ctr, key) != expect
    assert key_bumped_first(ctr, key) != expect
    assert philox_py(ctr, key, rounds=9) != expect
    out = philox_py(ctr, key)
    assert [out[1], out[0], out[3], out[2]] != expect


def test_philox_two_implementations_agree(orc):
    rng = random.Random(12345)
    cases = [([0, 0, 0, 0], [0, 0]), ([M32] * 4, [M32, M32])]
    cases += [([rng.getrandbits(32) for _ in range(4)], [rng.getrandbits(32) for _ in range(2)]) for _ in range(500)]
    for ctr, key in cases:
        assert orc.philox4x32_10(ctr, key) == philox_py(ctr, key)


def test_philox_avalanche(orc):
    # flipping one counter bit flips about half of the 128 output bits
    rng = random.Random(7)
    flips = []
    for _ in range(200):
        ctr = [rng.getrandbits(32) for _ in range(4)]
        key = [rng.getrandbits(32) for _ in range(2)]
        a = orc.philox4x32_10(ctr, key)
        w, b = rng.randrange(4), rng.randrange(32)
        ctr2 = list(ctr)
        ctr2[w] ^= 1 << b
        bb = orc.philox4x32_10(ctr2, key)
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, bb)))
    assert abs(np.mean(flips) - 64.0) < 2.0


def test_uniform_mapping_exact(orc):
    # u_j of event ev uses counter (ev_lo, ev_hi, j>>1, 0), key (seed_lo, seed_hi),
    # words (2(j&1), 2(j&1)+1): u = ((a>>6) 2^26 + (b>>6) + 1/2) 2^-52
    for seed, ev, j in [(1, 0, 0), (1, 0, 1), (0xDEADBEEFCAFEF00D, 2**40 + 17, 33), (7, 2**26 - 1, 52)]:
        w = philox_py([ev & M32, ev >> 32, j >> 1, 0], [seed & M32, seed >> 32])
        a, b = w[2 * (j & 1)], w[2 * (j & 1) + 1]
        expect = ((a >> 6) * 2**26 + (b >> 6) + 0.5) / 2**52
        assert orc.uniform(seed, ev, j) == expect


def test_uniform_open_interval_extremes():
    # the mapping never returns 0 or 1 and is exact in double precision
    # (k + 1/2 needs 53 significant bits for k < 2^52)
    lo = (0 * 2**26 + 0 + 0.5) / 2**52
    hi = ((2**26 - 1) * 2**26 + (2**26 - 1) + 0.5) / 2**52
    assert 0.0 < lo < 1e-15 and hi < 1.0
    assert hi == 1.0 - 2.0**-53
    from fractions import Fraction
    assert Fraction(hi) == Fraction(2**53 - 1, 2**53)


def test_uniform_statistics(orc):
    n = 40000
    u = np.array([orc.uniform(99, ev, j) for ev in range(n // 8) for j in range(8)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    # chi^2 on 64 bins
    h, _ = np.histogram(u, bins=64, range=(0, 1))
    assert stats.chisquare(h).pvalue > 1e-3
    # neighbouring draws of one event and of neighbouring events are uncorrelated
    m = u.reshape(-1, 8)
    for a, b in [(0, 1), (1, 2), (0, 7)]:
        assert abs(np.corrcoef(m[:, a], m[:, b])[0, 1]) < 5 / math.sqrt(m.shape[0])
    assert abs(np.corrcoef(m[:-1, 0], m[1:, 0])[0, 1]) < 5 / math.sqrt(m.shape[0])


def test_draw_count_layout(orc):
    # x1, x2, 4 per final gluon, one helicity word, n-2 ordering draws
    for n in range(4, 13):
        assert orc.n_uniforms(n) == 2 + 4 * (n - 2) + 1 + (n - 2)
