"""Vectorised (numpy) restatement of the counter-based draws, for test-side
bookkeeping only: which events of a run sampled a helicity configuration
whose tree amplitude vanishes.  Philox4x32-10 as published by Salmon et al.
(SC'11), the same definition the oracle implements and the known-answer
vectors pin; no value here comes from the CUDA path.
"""
import numpy as np

M32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & M32 for x in (c0, c1, c2, c3))
    k0, k1 = np.uint64(k0) & M32, np.uint64(k1) & M32
    for _ in range(10):
        p0 = np.uint64(0xD2511F53) * c0
        p1 = np.uint64(0xCD9E8D57) * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0) & M32, p1 & M32, ((p0 >> np.uint64(32)) ^ c3 ^ k1) & M32, \
            p0 & M32
        k0 = (k0 + np.uint64(0x9E3779B9)) & M32
        k1 = (k1 + np.uint64(0xBB67AE85)) & M32
    return c0, c1, c2, c3


def unit_bits(seed, events, j):
    """52-bit integers k of draw j (u = (k + 1/2) 2^-52) for an array of events."""
    ev = np.asarray(events, dtype=np.uint64)
    w = philox4x32_10(ev & M32, ev >> np.uint64(32), np.full(ev.shape, j >> 1, dtype=np.uint64),
                      np.zeros(ev.shape, dtype=np.uint64), seed & 0xFFFFFFFF, seed >> 32)
    a, b = (w[0], w[1]) if (j & 1) == 0 else (w[2], w[3])
    return ((a >> np.uint64(6)) << np.uint64(26)) | (b >> np.uint64(6))


def helicity_bits(n, seed, first, count):
    """Helicity labels (bit i = leg i) of sampled-helicity events: the top n
    bits of the helicity draw, number 2 + 4(n - 2) of each event."""
    k = unit_bits(seed, np.arange(first, first + count, dtype=np.uint64), 2 + 4 * (n - 2))
    return (k >> np.uint64(52 - n)).astype(np.int64)


def vanishing_mask(n, hel):
    """Tree amplitudes vanish for all labels equal or exactly one different."""
    c = np.zeros(hel.shape, dtype=np.int64)
    for i in range(n):
        c += (hel >> i) & 1
    return (c <= 1) | (c >= n - 1)
