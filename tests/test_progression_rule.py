"""The rule the in-group sorts use for groups whose positions form one arithmetic
progression, checked by brute force against the oracle's suffix array (CPU only).

For every h and every group of suffixes sharing their first h symbols (no '$'
inside), if the members sit at i, i+p, ..., i+(n-1)p with n >= 3 and p <= h, then
their true order is position order or its reverse, and the h-ranks of the suffixes
h past the last two members differ and say which; the LCP of two adjacent members
(Kasai's, from the oracle) is e minus the larger position, where e = last + h + the
common prefix of the suffixes h past the last two members.  The h-rank used here is the one
the doubling rounds hold: the smallest SA slot among the suffixes sharing the first
h symbols (a unique slot for a suffix whose '$' falls inside them)."""
import numpy as np
import pytest

import oracle
from paper_1404_3456_gb300 import synth


def h_ranks(t, isa, nxt, h):
    """Group of every suffix with at least h bases before its '$' (by its first h
    symbols), and the h-rank array."""
    n = t.size
    groups = {}
    for i in range(n):
        if nxt[i] - i >= h:
            groups.setdefault(bytes(t[i:i + h]), []).append(i)
    rank = isa.copy()
    for g in groups.values():
        if len(g) > 1:
            m = min(isa[x] for x in g)
            for x in g:
                rank[x] = m
    return groups, rank


def text_lcp(t, nxt, a, b, lim):
    """Common prefix of the suffixes at a and b in bases (a '$' never matches), at most lim."""
    m = min(lim, nxt[a] - a, nxt[b] - b)
    k = 0
    while k < m and t[a + k] == t[b + k]:
        k += 1
    return k


def progression_groups(t):
    """Checks the rule on every progression group of text t; returns how many."""
    n = t.size
    sa = oracle.suffix_array(t)
    isa = np.empty(n, np.int64)
    isa[sa] = np.arange(n)
    nxt = np.empty(n, np.int64)   # position of the next '$' at or after i
    j = n - 1
    for i in range(n - 1, -1, -1):
        if t[i] == ord("$"):
            j = i
        nxt[i] = j
    lcp = oracle.lcp_kasai(t, sa)
    checked = 0
    h = 1
    while h < n:
        groups, rank = h_ranks(t, isa, nxt, h)
        for g in groups.values():
            if len(g) < 3:
                continue
            g = sorted(g)
            d = g[-1] - g[0]
            if d % (len(g) - 1):
                continue
            p = d // (len(g) - 1)
            if p > h or any((x - g[0]) % p for x in g):
                continue
            last = g[-1]
            before, after = rank[last - p + h], rank[last + h]
            assert before != after
            want = g if before < after else g[::-1]
            assert sorted(g, key=lambda x: isa[x]) == want, (h, p, g[:4])
            # the LCP of adjacent members in closed form: e - the larger position, e the
            # position where the period breaks, found past the last two members
            e = last + h + text_lcp(t, nxt, last - p + h, last + h, h)
            for a, b in zip(want, want[1:]):
                assert lcp[isa[b]] == e - max(a, b), (h, p, a, b)
            checked += 1
        h *= 2
    return checked


def tandem_reads(rng, n_reads):
    reads = []
    for _ in range(n_reads):
        parts = []
        for _ in range(int(rng.integers(1, 4))):
            parts.append(synth.iid(rng, int(rng.integers(0, 20))))
            unit = synth.iid(rng, int(rng.integers(1, 6)))
            parts.append(np.tile(unit, int(rng.integers(2, 30))))
        if rng.random() < 0.5:
            parts.append(synth.iid(rng, 5))
        reads.append(np.concatenate(parts))
    return synth.join_reads(reads)


@pytest.mark.parametrize("seed", range(6))
def test_progression_rule_on_tandem_texts(seed):
    rng = np.random.default_rng(100 + seed)
    total = 0
    for _ in range(5):
        total += progression_groups(tandem_reads(rng, int(rng.integers(1, 4))))
    assert total > 0


def test_progression_rule_homopolymer_ends():
    # runs of one base ending at '$', before a larger base, before a smaller base
    for text in (b"AAAAAAAAAAAA$", b"AAAAAAAAAAAAC$", b"CCCCCCCCCCCA$", b"ACACACACACACACG$ACACACAC$"):
        assert progression_groups(np.frombuffer(text, np.uint8)) > 0
