"""Property checks of the oracle on generated texts (CPU; skipped without hypothesis).

Each property is fixed by the definitions alone, independently of the oracle's
own code: the suffix order with distinct position-ordered sentinels, the LCP as
the directly measured common prefix, and the overlap relation by brute force.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402

fragments = st.lists(st.text(alphabet="ACGT", min_size=1, max_size=24), min_size=1, max_size=6)


def as_text(frags):
    return np.frombuffer(("$".join(frags) + "$").encode(), dtype=np.uint8)


def suffix_key(t, p):
    # symbols up to and including the fragment's '$'; '$' sorts first, and two
    # suffixes ending at the same offset order by position (distinct sentinels)
    out = []
    for q in range(p, t.size):
        c = int(t[q])
        if c == ord("$"):
            out.append((0, q))
            break
        out.append((1 + b"ACGT".index(c), 0))
    return out


@settings(max_examples=150, deadline=None)
@given(fragments)
def test_suffix_array_is_the_definition(frags):
    t = as_text(frags)
    want = sorted(range(t.size), key=lambda p: suffix_key(t, p))
    assert list(oracle.suffix_array(t)) == want


@settings(max_examples=150, deadline=None)
@given(fragments)
def test_lcp_is_the_measured_common_prefix(frags):
    t = as_text(frags)
    sa = oracle.suffix_array(t)
    lcp = oracle.lcp_kasai(t, sa)
    assert lcp[0] == 0
    for j in range(1, t.size):
        a, b = int(sa[j - 1]), int(sa[j])
        h = 0
        while a + h < t.size and b + h < t.size and t[a + h] == t[b + h] and t[a + h] != ord("$"):
            h += 1
        assert lcp[j] == h


@settings(max_examples=100, deadline=None)
@given(fragments, st.integers(min_value=1, max_value=6))
def test_overlaps_are_the_brute_force_relation(frags, lmin):
    t = as_text(frags)
    want = {}
    for j, a in enumerate(frags):
        for k, b in enumerate(frags):
            if j == k:
                continue
            for L in range(min(len(a), len(b)) - 1, lmin - 1, -1):
                if a[-L:] == b[:L]:
                    want[(j, k)] = L
                    break
    ej, ek, eL = oracle.overlaps_sorted(t, lmin)
    got = {(int(x), int(y)): int(z) for x, y, z in zip(ej, ek, eL)}
    assert got == want
    assert list(zip(ej, ek)) == sorted(zip(ej, ek))
