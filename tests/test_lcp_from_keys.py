"""The rule round 0 of sa_lcp_build uses to write LCP entries without reading the
text, checked by brute force against the oracle's suffix array and Kasai LCP (CPU).

A suffix's initial key is its first h0 bases (2-bit codes, zero past the bases it
has before its '$') and lc = min(bases before its '$', h0).  For two SA neighbours
whose keys differ, the LCP (bases, a '$' never matching) is the number of equal
leading codes of their padded h0-mers, capped by both lc values; neighbours with
equal keys share at least h0 bases."""
import numpy as np
import pytest

import oracle
from paper_1404_3456_gb300 import synth

CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def keys(t, h0):
    n = t.size
    nxt = np.empty(n, np.int64)   # position of the next '$' at or after i
    j = n - 1
    for i in range(n - 1, -1, -1):
        if t[i] == ord("$"):
            j = i
        nxt[i] = j
    out = []
    for i in range(n):
        lc = min(int(nxt[i] - i), h0)
        out.append((tuple(CODE[int(t[i + k])] if k < lc else 0 for k in range(h0)), lc))
    return out


def lcp_from_keys(ka, kb, h0):
    (xa, la), (xb, lb) = ka, kb
    eq = next((k for k in range(h0) if xa[k] != xb[k]), h0)
    return min(eq, la, lb)


@pytest.mark.parametrize("h0", [3, 8, 16])
@pytest.mark.parametrize("seed", range(4))
def test_lcp_of_separated_pairs_from_keys(h0, seed):
    rng = np.random.default_rng(200 + seed)
    reads = []
    for _ in range(int(rng.integers(1, 6))):
        n = int(rng.integers(1, 80))
        if rng.random() < 0.4:   # periodic reads: long shared prefixes
            r = np.tile(synth.iid(rng, int(rng.integers(1, 4))), n)[:n]
        else:
            r = synth.iid(rng, n)
        reads.append(r)
    reads.append(reads[0].copy())   # a duplicated read: equal keys up to its '$'
    t = synth.join_reads(reads)
    sa = oracle.suffix_array(t)
    lcp = oracle.lcp_kasai(t, sa)
    k = keys(t, h0)
    separated = 0
    for j in range(1, t.size):
        a, b = int(sa[j - 1]), int(sa[j])
        if k[a] != k[b] or k[a][1] < h0:   # different keys, or a '$' inside the key (unique)
            assert lcp[j] == lcp_from_keys(k[a], k[b], h0), (j, a, b)
            separated += 1
        else:
            assert lcp[j] >= h0
    assert separated > 0
