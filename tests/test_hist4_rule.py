"""The rule the initial-key kernel uses for one sequence whose key is whole 4-mers
(h0 = 4 * passes): every pass's 8-bit digit histogram follows from one histogram of
the text's 4-mer codes, corrected at the two ends, checked by brute force (CPU).

Pass q's digit of the suffix at p is the 4-mer code at p + o, o = h0 - 4 - 4q, for
the suffixes with at least h0 bases before the '$'; the others carry a key padded
with zero codes past their last base.  So pass q's histogram is the 4-mer histogram
over x = 0 .. N-5 without the codes at x < o and at x > N-1-h0+o, plus the padded
keys of the last h0 suffixes."""
import numpy as np
import pytest


def padded_key(bases, N, p, h0):
    lc = min(N - 1 - p, h0)
    v = 0
    for i in range(h0):
        v = (v << 2) | (int(bases[p + i]) if i < lc else 0)
    return v


def code(bases, x):
    return (int(bases[x]) << 6) | (int(bases[x + 1]) << 4) | (int(bases[x + 2]) << 2) | int(bases[x + 3])


@pytest.mark.parametrize("h0", [8, 12, 16, 20, 28])
@pytest.mark.parametrize("seed", range(3))
def test_digit_histograms_from_one_4mer_histogram(h0, seed):
    rng = np.random.default_rng(300 + seed)
    passes = h0 // 4
    for N in (2 * h0 + 8, int(rng.integers(2 * h0 + 9, 400))):
        bases = rng.integers(0, 4, N - 1)          # the text: N - 1 bases and the '$'
        direct = np.zeros((passes, 256), np.int64)
        for p in range(N):
            k = padded_key(bases, N, p, h0)
            for q in range(passes):
                direct[q, (k >> (8 * q)) & 255] += 1
        H = np.zeros(256, np.int64)
        for x in range(N - 4):                     # x = 0 .. N-5
            H[code(bases, x)] += 1
        for q in range(passes):
            o = h0 - 4 - 4 * q
            c = H.copy()
            for x in range(o):
                c[code(bases, x)] -= 1
            for x in range(N - h0 + o, N - 4):
                c[code(bases, x)] -= 1
            for p in range(N - h0, N):
                c[(padded_key(bases, N, p, h0) >> (8 * q)) & 255] += 1
            assert np.array_equal(c, direct[q]), (N, h0, q)
