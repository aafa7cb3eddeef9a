"""Pins of the oracle's two-cut "fir" reconstruction (Sec. III, Figs. 2 and 5-8).

The oracle's depth-first search is checked against what the paper's model fixes,
not against a second copy of itself:
* exact recovery: a genome cut by two shotguns with every break position
  different (Fig. 4) is rebuilt exactly, each fragment at its true offset;
* back-tracking (Fig. 7): a hand-built set where the first fir pair tried is a
  dead end and the search must back up to the true start pair;
* completeness and soundness by brute force on tiny sets: a reconstruction is
  found exactly when the fragments split into two sequences that spell the same
  string with no common inner break (enumerated over every split and order), and
  the one found is such a split;
* no-solution and step-bound cases.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1404_3456_gb300 import synth

A = np.frombuffer(b"ACGT", np.uint8)


def two_tilings(frags):
    """Every way to split the fragments into two ordered sequences that spell the
    same string, with no inner break position shared (n >= 3).  Returns a set of
    frozensets of (fragment index, offset)."""
    n = len(frags)
    out = set()
    if n < 3:
        return out
    for mask in range(1, (1 << n) - 1):
        a = [i for i in range(n) if mask >> i & 1]
        b = [i for i in range(n) if not mask >> i & 1]
        if a > b:
            continue   # each split once (the two sides are interchangeable)
        spell_b = {}
        for pb in itertools.permutations(b):
            s = b"".join(frags[i] for i in pb)
            spell_b.setdefault(s, []).append(pb)
        for pa in itertools.permutations(a):
            s = b"".join(frags[i] for i in pa)
            for pb in spell_b.get(s, []):
                offs = {}
                cuts_a, cuts_b = set(), set()
                o = 0
                for i in pa:
                    offs[i] = o
                    o += len(frags[i])
                    cuts_a.add(o)
                o = 0
                for i in pb:
                    offs[i] = o
                    o += len(frags[i])
                    cuts_b.add(o)
                if (cuts_a & cuts_b) == {len(s)}:
                    out.add(frozenset(offs.items()))
    return out


@pytest.mark.parametrize("seed", range(12))
def test_two_cut_genome_recovered_exactly(seed):
    d = synth.two_cut(seed, int(5_000 + 2_000 * seed), mean_len=300 + 40 * seed)
    st, start, rs, steps = oracle.fir_reconstruct(d["text"])
    assert st == oracle.FIR_SOLVED
    assert rs == d["genome"].tobytes()
    assert np.array_equal(start, d["frag_start"])
    n = int((d["text"] == ord("$")).sum())
    assert steps >= n - 1   # one step per fragment placed after the start pair


def test_back_tracking_from_a_dead_start_pair():
    """Fig. 7: one short fragment u is a prefix of two fragments, the true first
    piece x of the other cutting and a later piece z that also starts with u.
    z has the smaller index, so (u, z) is tried first; its remainder matches no
    fragment, the search backs up and continues from (u, x)."""
    rng = np.random.default_rng(3)
    u = A[rng.integers(0, 4, 30)]
    r1 = A[rng.integers(0, 4, 100)]
    r2 = A[rng.integers(0, 4, 100)]
    S = np.concatenate([u, r1, u, r2])       # 260 bases, u at 0 and at 130
    cut1 = [(0, 30), (30, 175), (175, 260)]
    cut2 = [(0, 130), (130, 200), (200, 260)]
    z, x, uu = (130, 200), (0, 130), (0, 30)
    pieces = [z, x, uu] + [p for p in cut1 + cut2 if p not in (z, x, uu)]
    text = synth.join_reads([S[a:b] for a, b in pieces])
    st, start, rs, steps = oracle.fir_reconstruct(text)
    assert st == oracle.FIR_SOLVED
    assert rs == S.tobytes()
    assert start.tolist() == [a for a, _ in pieces]
    assert steps == 6   # the dead start pair, the true one, four more placements
    # with a bound of one step the search gives up on the dead start pair
    st1, start1, rs1, steps1 = oracle.fir_reconstruct(text, max_steps=1)
    assert st1 == oracle.FIR_GAVE_UP and rs1 == b"" and np.all(start1 == -1)


@pytest.mark.parametrize("seed", range(40))
def test_tiny_sets_against_brute_force(seed):
    rng = np.random.default_rng(1000 + seed)
    if seed % 2 == 0:
        # two cuttings of a short two-letter genome: many ambiguous fir relations
        G = int(rng.integers(8, 16))
        g = np.frombuffer(b"AC", np.uint8)[rng.integers(0, 2, G)]
        k = int(rng.integers(2, 5))
        br = np.sort(rng.choice(np.arange(1, G), size=min(k, G - 1), replace=False))
        side = rng.integers(0, 2, br.size)
        frags = []
        for c in (0, 1):
            b = np.concatenate([[0], br[side == c], [G]])
            frags += [g[a:e] for a, e in zip(b[:-1], b[1:])]
        frags = [frags[i] for i in rng.permutation(len(frags))][:6]
    else:
        frags = [np.frombuffer(b"AC", np.uint8)[rng.integers(0, 2, int(rng.integers(1, 5)))]
                 for _ in range(int(rng.integers(2, 6)))]
    fb = [f.tobytes() for f in frags]
    sols = two_tilings(fb)
    st, start, rs, _ = oracle.fir_reconstruct(synth.join_reads(frags))
    assert (st == oracle.FIR_SOLVED) == bool(sols)
    if st == oracle.FIR_SOLVED:
        assert frozenset((i, int(start[i])) for i in range(len(fb))) in sols
        for i, f in enumerate(fb):
            assert rs[start[i]: start[i] + len(f)] == f


def test_no_reconstruction():
    # no fragment is a prefix of another: no fir pair to start from
    st, start, rs, steps = oracle.fir_reconstruct(b"ACGT$CATG$GGA$")
    assert st == oracle.FIR_NONE and steps == 0 and rs == b""
    # a fir pair exists but nothing continues its remainder
    st, _, _, steps = oracle.fir_reconstruct(b"AC$ACGT$TTT$")
    assert st == oracle.FIR_NONE and steps == 1
