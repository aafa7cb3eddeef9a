"""Pins of the oracle's overlaps under the paper's DEFINITION (Sec. III):
fragments read on either strand, with a rate mu of substitution errors.

* mu = 0 on one strand reduces to the exact overlap set (the pinned
  overlaps_brute);
* planted reads: a genome, reads at known starts, each on a random strand and
  with planted substitutions; every true overlap between neighbouring reads is
  found between the right orientations, with the length given by the starts and
  the mismatch count given by the planted substitutions;
* reverse-complement symmetry: (a, b, L, e) is an edge exactly when
  (rc(b), rc(a), L, e) is one.
"""
import numpy as np
import pytest

import oracle
from paper_1404_3456_gb300 import synth

COMP = {ord("A"): ord("T"), ord("C"): ord("G"), ord("G"): ord("C"), ord("T"): ord("A")}


def revcomp(x: np.ndarray) -> np.ndarray:
    return np.array([COMP[int(c)] for c in x[::-1]], dtype=np.uint8)


@pytest.mark.parametrize("seed", range(5))
def test_mu_zero_one_strand_is_exact_overlaps(seed):
    rng = np.random.default_rng(50 + seed)
    reads = []
    for _ in range(int(rng.integers(3, 25))):
        n = int(rng.integers(20, 120))
        if rng.random() < 0.4:
            unit = synth.iid(rng, int(rng.integers(1, 5)))
            reads.append(np.tile(unit, n // unit.size + 1)[:n])
        else:
            reads.append(synth.iid(rng, n))
    text = synth.join_reads(reads)
    a, b, L, mm = oracle.overlaps_approx(text, 5, 0, 1, rc=False)
    j, k, L2 = oracle.overlaps_brute(text, 5)
    assert np.array_equal(a, j) and np.array_equal(b, k) and np.array_equal(L, L2)
    assert np.all(mm == 0)


def planted(seed, G=4000, read_len=300, step=150, subs=2):
    rng = np.random.default_rng(seed)
    genome = synth.iid(rng, G)
    starts = list(range(0, G - read_len + 1, step))
    reads, strands, muts = [], [], []
    for s in starts:
        r = genome[s: s + read_len].copy()
        pos = rng.choice(read_len, size=subs, replace=False)
        m = {}
        for p in pos:
            nb = synth.BASES[(np.searchsorted(synth.BASES, r[p]) + int(rng.integers(1, 4))) % 4]
            r[p] = nb
            m[s + int(p)] = int(nb)          # genome coordinate -> planted base
        rc = bool(rng.random() < 0.5)
        reads.append(revcomp(r) if rc else r)
        strands.append(rc)
        muts.append(m)
    return genome, starts, reads, strands, muts


@pytest.mark.parametrize("seed", range(4))
def test_planted_two_strand_overlaps(seed):
    genome, starts, reads, strands, muts = planted(700 + seed)
    text = synth.join_reads(reads)
    a, b, L, mm = oracle.overlaps_approx(text, 40, 1, 30, rc=True)
    edges = {(int(x), int(y)): (int(l), int(e)) for x, y, l, e in zip(a, b, L, mm)}
    for i in range(len(starts) - 1):
        fi = 2 * i + (1 if strands[i] else 0)            # read i as on the genome's strand
        fj = 2 * (i + 1) + (1 if strands[i + 1] else 0)
        L0 = starts[i] + 300 - starts[i + 1]
        lo, hi = starts[i + 1], starts[i] + 300          # genome interval of the overlap
        expect = sum(1 for g in range(lo, hi)
                     if muts[i].get(g, int(genome[g])) != muts[i + 1].get(g, int(genome[g])))
        assert edges.get((fi, fj)) == (L0, expect), i
        # the same overlap read on the other strand
        assert edges.get((fj ^ 1, fi ^ 1)) == (L0, expect), i


@pytest.mark.parametrize("seed", range(3))
def test_reverse_complement_symmetry(seed):
    rng = np.random.default_rng(900 + seed)
    g = synth.iid(rng, 800)
    reads = []
    for _ in range(12):
        s = int(rng.integers(0, 700))
        n = int(rng.integers(40, 100))
        r = g[s: s + n]
        reads.append(revcomp(r) if rng.random() < 0.5 else r.copy())
    text = synth.join_reads(reads)
    a, b, L, mm = oracle.overlaps_approx(text, 12, 1, 20, rc=True)
    E = {(int(x), int(y), int(l), int(e)) for x, y, l, e in zip(a, b, L, mm)}
    assert E, "expected some overlaps"
    assert E == {(y ^ 1, x ^ 1, l, e) for x, y, l, e in E}
    assert all(x // 2 != y // 2 for x, y, _, _ in E)
