"""Pins for the oracle: each test checks it against something other than itself
(a printed example, a textbook value, brute force over every small input, a
library routine, or the ground truth the generator knows), chosen so that a
dropped term, a wrong sign, an off-by-one or a swapped operand fails one."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1404_3456_gb300 import synth

SEP = ord("$")


def distinct_sentinel_bytes(text: bytes) -> bytes:
    """The text with the r-th '$' replaced by byte r: every sentinel distinct,
    ordered by position, and smaller than every letter.  Plain Python bytes
    comparison of T[i:] is then the suffix order (no two suffixes tie)."""
    out = bytearray(text)
    r = 0
    for i, c in enumerate(out):
        if c == SEP:
            out[i] = r
            r += 1
    assert r < 0x24
    return bytes(out)


def sa_by_python_sort(text: bytes):
    t2 = distinct_sentinel_bytes(text)
    return np.array(sorted(range(len(t2)), key=lambda i: t2[i:]), dtype=np.int64)


def random_reads_text(rng, n_reads, lo, hi, alphabet=b"ACGT", periodic=False):
    reads = []
    for _ in range(n_reads):
        n = int(rng.integers(lo, hi + 1))
        if periodic and rng.random() < 0.5:
            unit = bytes(rng.choice(list(alphabet), size=int(rng.integers(1, 4))).tolist())
            r = (unit * (n // len(unit) + 1))[:n]
        else:
            r = bytes(rng.choice(list(alphabet), size=n).tolist())
        reads.append(r)
    # repeat some reads and embed some in others to exercise ties and containment
    if n_reads >= 3:
        reads[1] = reads[0]
        reads[2] = reads[0][1:] if len(reads[0]) > 1 else reads[2]
    return b"$".join(reads) + b"$", reads


# ---------------------------------------------------------------- fixtures


def test_banana_golden(golden):
    g = golden("banana.txt")
    text = g["text"].encode()
    sa = oracle.suffix_array(text)
    assert sa.tolist() == [int(x) for x in g["sa"].split()]
    assert oracle.lcp_kasai(text, sa).tolist() == [int(x) for x in g["lcp"].split()]
    assert oracle.lcp_direct(text, sa).tolist() == [int(x) for x in g["lcp"].split()]
    assert oracle.sa_check(text, sa) == 0


def test_superstring_worked_example(golden):
    """Sec. III, Fig. 3: the five fragments give abthatbabhhatbpaabtabhaabtpb."""
    g = golden("superstring_example.txt")
    frags = g["fragments"].split()
    text = ("$".join(frags) + "$").encode()
    for fn in (oracle.overlaps_brute, oracle.overlaps_sorted):
        buf, off = oracle.assemble(text, 1, overlap_fn=fn)
        assert oracle.contigs_as_list(buf, off) == [g["superstring"].encode()]
    # the accepted chain is the paper's path
    ej, ek, eL = oracle.overlaps_brute(text, 1)
    path = [int(x) for x in g["path"].split()]
    got = {(int(a), int(b)): int(c) for a, b, c in zip(ej, ek, eL)}
    for a, b in zip(path, path[1:]):
        assert (a, b) in got
    assert [got[(a, b)] for a, b in zip(path, path[1:])] == [2, 7, 4, 2]


# ---------------------------------------------------------------- suffix array


def test_sa_all_short_dna_strings():
    """Every string over {A,C,G,T} of length <= 6 (5461 texts) against a plain
    Python sort of its suffixes."""
    for n in range(0, 7):
        for tup in itertools.product(b"ACGT", repeat=n):
            text = bytes(tup) + b"$"
            sa = oracle.suffix_array(text)
            assert sa.tolist() == sa_by_python_sort(text).tolist(), text


@pytest.mark.parametrize("seed", range(20))
def test_sa_multi_read_texts(seed):
    rng = np.random.default_rng(seed)
    text, _ = random_reads_text(rng, int(rng.integers(1, 12)), 1, 30, periodic=True)
    sa = oracle.suffix_array(text)
    assert sa.tolist() == sa_by_python_sort(text).tolist()
    assert oracle.sa_check(text, sa) == 0


def test_sa_separator_semantics():
    """'$' is smaller than A; equal strings ending at '$' order by position;
    nothing is compared past a '$'."""
    text = b"A$A$AA$"
    sa = oracle.suffix_array(text).tolist()
    # suffixes: 0 'A$..', 1 '$..', 2 'A$..', 3 '$..', 4 'AA$', 5 'A$', 6 '$'
    assert sa == [1, 3, 6, 0, 2, 5, 4]
    lcp = oracle.lcp_kasai(text, np.array(sa)).tolist()
    assert lcp == [0, 0, 0, 0, 1, 1, 1]


def test_sa_rejects_unterminated():
    with pytest.raises(ValueError):
        oracle.suffix_array(b"ACGT")


# ---------------------------------------------------------------- LCP


@pytest.mark.parametrize("seed", range(10))
def test_kasai_equals_direct(seed):
    rng = np.random.default_rng(100 + seed)
    text, _ = random_reads_text(rng, int(rng.integers(1, 40)), 1, 200, periodic=True)
    sa = oracle.suffix_array(text)
    a = oracle.lcp_kasai(text, sa)
    b = oracle.lcp_direct(text, sa)
    assert np.array_equal(a, b)
    # and against Python: the common prefix of the two suffixes up to a '$'
    t = text
    for j in range(1, len(sa)):
        p, q = int(sa[j - 1]), int(sa[j])
        h = 0
        while t[p + h] == t[q + h] and t[p + h] != SEP:
            h += 1
        assert a[j] == h


def test_lcp_tandem_repeat():
    """(AC)^50$: every adjacent pair of suffixes from the same phase shares all
    but the shorter's tail; the maximum LCP is 98."""
    text = b"AC" * 50 + b"$"
    sa = oracle.suffix_array(text)
    lcp = oracle.lcp_kasai(text, sa)
    assert lcp.max() == 98
    assert np.array_equal(lcp, oracle.lcp_direct(text, sa))


# ---------------------------------------------------------------- checker


def test_checker_rejects_perturbations():
    rng = np.random.default_rng(7)
    text, _ = random_reads_text(rng, 8, 5, 60, periodic=True)
    sa = oracle.suffix_array(text)
    assert oracle.sa_check(text, sa) == 0
    n = len(sa)
    for _ in range(50):
        i, j = rng.choice(n, size=2, replace=False)
        bad = sa.copy()
        bad[i], bad[j] = bad[j], bad[i]
        assert oracle.sa_check(text, bad) != 0
        dup = sa.copy()
        dup[i] = dup[j]
        assert oracle.sa_check(text, dup) == 1
    # a rotation of a correct SA is a permutation but wrong
    assert oracle.sa_check(text, np.roll(sa, 1)) != 0


@pytest.mark.parametrize("seed", range(4))
def test_threaded_checker_and_kasai_equal_whole(seed):
    """The range-split checker and Kasai (one range per thread, each range of
    Kasai restarting at h = 0) give exactly the whole-array results: the LCP of
    the pinned Kasai, acceptance of the true SA, and rejection of planted swaps
    (naming the same first failing pair as the whole checker), duplicates and
    rotations."""
    rng = np.random.default_rng(40 + seed)
    text, _ = random_reads_text(rng, int(rng.integers(1, 30)), 1, 300, periodic=True)
    sa = oracle.suffix_array(text)
    code, lcp = oracle.sa_check_and_lcp_threaded(text, sa, threads=1 + seed)
    assert code == 0
    assert np.array_equal(lcp, oracle.lcp_kasai(text, sa))
    n = len(sa)
    for _ in range(20):
        i, j = rng.choice(n, size=2, replace=False)
        bad = sa.copy()
        bad[i], bad[j] = bad[j], bad[i]
        c, l2 = oracle.sa_check_and_lcp_threaded(text, bad, threads=3)
        assert c >= 2 and l2 is None
        # each range reports its first failing pair, so the smallest is the
        # whole checker's first failing pair
        assert c == oracle.sa_check(text, bad)
    dup = sa.copy()
    dup[0] = dup[1]
    assert oracle.sa_check_and_lcp_threaded(text, dup)[0] == 1
    assert oracle.sa_check_and_lcp_threaded(text, np.roll(sa, 1))[0] != 0


def test_check_pairs_finds_planted_errors():
    """The sampled checker accepts the true SA and LCP and flags a planted swap
    and a planted LCP error (mistakes planted in oracle data, on the CPU)."""
    rng = np.random.default_rng(5)
    text, _ = random_reads_text(rng, 10, 5, 80, periodic=True)
    sa = oracle.suffix_array(text)
    lcp = oracle.lcp_kasai(text, sa)
    idx = np.arange(1, len(sa))
    assert oracle.check_pairs(text, sa, lcp, idx) == 0
    bad = sa.copy()
    bad[10], bad[11] = bad[11], bad[10]
    assert oracle.check_pairs(text, bad, None, idx) >= 1
    badl = lcp.copy()
    badl[7] += 1
    assert oracle.check_pairs(text, sa, badl, idx) == 1


# ---------------------------------------------------------------- Algorithm 1


@pytest.mark.parametrize("seed", range(5))
def test_split_sort_is_stable_sort(seed):
    """32 (or 64) 1-bit splits equal a stable sort: numpy's stable argsort."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    hi = [8, 32, 64][seed % 3]
    keys = rng.integers(0, 2**63, size=n, dtype=np.uint64)
    if hi < 64:
        keys &= np.uint64((1 << hi) - 1)
    keys[: n // 3] = keys[0]  # many equal keys: stability matters
    vals = np.arange(n, dtype=np.uint64)
    k, v = oracle.split_sort(keys, vals, 0, hi)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(k, keys[order])
    assert np.array_equal(v, vals[order])


def test_split_sort_partial_bits():
    keys = np.array([0b101, 0b011, 0b100, 0b001, 0b110], dtype=np.uint64)
    k, v = oracle.split_sort(keys, np.arange(5, dtype=np.uint64), 0, 1)
    # one split on bit 0: evens (0b100, 0b110) first, in input order, then odds
    assert v.tolist() == [2, 4, 0, 1, 3]


# ---------------------------------------------------------------- overlaps


@pytest.mark.parametrize("seed", range(15))
def test_overlaps_sorted_equals_brute(seed):
    rng = np.random.default_rng(200 + seed)
    text, _ = random_reads_text(rng, int(rng.integers(2, 25)), 1, 40, alphabet=b"AC",
                                periodic=True)
    lmin = int(rng.integers(1, 4))
    a = oracle.overlaps_brute(text, lmin)
    b = oracle.overlaps_sorted(text, lmin)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def python_overlaps(reads, lmin):
    out = []
    for j, rj in enumerate(reads):
        for k, rk in enumerate(reads):
            if j == k:
                continue
            for L in range(min(len(rj), len(rk)) - 1, lmin - 1, -1):
                if rj[len(rj) - L:] == rk[:L]:
                    out.append((j, k, L))
                    break
    return out


def test_overlaps_small_by_python():
    rng = np.random.default_rng(3)
    text, reads = random_reads_text(rng, 12, 1, 15, alphabet=b"AC", periodic=True)
    ej, ek, eL = oracle.overlaps_brute(text, 1)
    assert list(zip(ej.tolist(), ek.tolist(), eL.tolist())) == python_overlaps(reads, 1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_overlaps_tiny_ground_truth(seed):
    """tiny workload: every 31-mer is unique, so the overlap set is exactly the
    set of read pairs whose genome intervals overlap by 31..399 bases."""
    inst = synth.tiny(seed)
    starts = inst["starts"]
    R = 400
    want = []
    for j, sj in enumerate(starts):
        for k, sk in enumerate(starts):
            L = R - (int(sk) - int(sj))
            if j != k and sk > sj and 31 <= L <= R - 1:
                want.append((j, k, L))
    want.sort()
    ej, ek, eL = oracle.overlaps_sorted(inst["text"], 31)
    assert list(zip(ej.tolist(), ek.tolist(), eL.tolist())) == want


# ---------------------------------------------------------------- containment


def test_contained_cases():
    reads = [b"ACGTAC", b"CGTA", b"ACGTAC", b"TTTT", b"GTACG", b"TTTT", b"A"]
    text = b"$".join(reads) + b"$"
    c = oracle.contained(text).tolist()
    # 1 lies inside 0; 2 duplicates 0 (larger index marked); 5 duplicates 3;
    # 6 'A' lies inside 0; 4 'GTACG' occurs nowhere else
    assert c == [0, 1, 1, 0, 0, 1, 1]


@pytest.mark.parametrize("seed", [0, 1])
def test_contained_ground_truth(seed):
    """i.i.d. genome, reads >= 100 bp: containment is interval containment."""
    inst = synth.batched_instance(seed, 0, g_lo=2000, g_hi=3000)
    s = inst["starts"]
    e = s + np.array([r.size for r in inst["reads"]])
    want = []
    for k in range(s.size):
        ck = 0
        for j in range(s.size):
            if j == k:
                continue
            if s[j] <= s[k] and e[k] <= e[j]:
                if s[j] == s[k] and e[j] == e[k] and j > k:
                    continue
                ck = 1
                break
        want.append(ck)
    assert oracle.contained(inst["text"]).tolist() == want


# ---------------------------------------------------------------- layout


@pytest.mark.parametrize("seed", range(8))
def test_tiny_genome_recovery(seed):
    """tiny workload: the layout spells the genome exactly (one contig)."""
    inst = synth.tiny(seed)
    buf, off = oracle.assemble(inst["text"], inst["min_overlap"])
    assert oracle.contigs_as_list(buf, off) == [inst["genome"].tobytes()]


def test_layout_two_chains_and_cycle():
    # a cycle A->B->C->A: union-find must refuse the closing edge
    reads = [b"AAACCC", b"CCCGGG", b"GGGAAA"]
    text = b"$".join(reads) + b"$"
    buf, off = oracle.assemble(text, 3)
    contigs = oracle.contigs_as_list(buf, off)
    # the closing edge (2, 0, 3) ties with the others on L; ties go by (j, k),
    # so (0,1) and (1,2) are taken first and (2,0) would close the cycle
    assert contigs == [b"AAACCCGGGAAA"]
    # no overlap at all: each read is its own contig, in index order
    text = b"ACGT$TTTT$GGGG$"
    buf, off = oracle.assemble(text, 2)
    assert oracle.contigs_as_list(buf, off) == [b"ACGT", b"TTTT", b"GGGG"]


# ---------------------------------------------------------------- generator


@pytest.mark.parametrize("seed", range(5))
def test_tiny_generator_preconditions(seed):
    inst = synth.tiny(seed)
    s = np.sort(inst["starts"])
    assert s.size == 202 and np.unique(s).size == 202       # distinct break positions
    assert s[0] == 0 and s[-1] == 10_000 - 400               # pinned ends
    assert np.all(np.diff(s) <= 400 - 31)                    # chained by >= 31
    assert synth._kmers_unique(inst["genome"], 31)
    assert inst["text"].size == 202 * 401


def test_repeat_genome_composition():
    rng = synth.rng_for(0, 9)
    g = synth.genome_with_repeats(rng, 200_000, 0.05, (2, 50), (10, 200), 0.05, 300, 0.01)
    assert g.size == 200_000
    assert set(np.unique(g).tolist()) <= set(b"ACGT")
    # repeats show up as far more repeated 32-mers than an i.i.d. genome has
    view = np.lib.stride_tricks.sliding_window_view(g, 32)
    u = np.unique(np.ascontiguousarray(view).view(np.dtype((np.void, 32))).ravel())
    assert u.size < 0.95 * view.shape[0]
