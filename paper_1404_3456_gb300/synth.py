"""Seeded synthetic genomes and shotgun fragment sets.

This module is shared by the tests, the benchmark and the oracle's checks.  It
holds none of the method's arithmetic: it only draws genomes and fragments and
joins fragments into a '$'-separated ASCII text (the input format the library
and the oracle both accept).  All randomness comes from numpy's PCG64 seeded
per instance, so every input is reproducible from (workload, seed).

The paper's dataset (Bacillus megaterium MSP20.1 from NCBI, Sec. V) is not
available; these workloads stand in for it, with the paper's shotgun model
(Sec. III, Fig. 2): a genome over {A, C, G, T} is cut into error-free fragments
whose break positions are all different (Sec. III, Fig. 4).

Workloads
---------
``tiny``     10,000 bp i.i.d. genome, 200 reads of 400 bp at distinct uniform
             starts plus reads pinned at both ends, consecutive starts at most
             400 - 31 apart and every 31-mer of the genome unique (so the only
             overlaps >= 31 are the true ones); reads in shuffled order.
``sa64m``    64,000,000 bp genome: 90 % i.i.d., 5 % tandem arrays (period
             U{2..50}, U{10..200} exact copies), 5 % copies of one 300 bp
             element, each copy with 1 % point substitutions.  One '$'.
``batched``  independent instances: genome log-uniform [2 kbp, 200 kbp] i.i.d.;
             reads of length U{100..1000} at uniform starts until 8x coverage.
``served``   jobs: genome log-uniform [5 kbp, 5 Mbp] with 2 % tandem arrays
             (period U{2..50}, copies U{10..200}); 150 bp reads at 10x.
``large``    1.5 Gbp genome: 85 % i.i.d., 10 % tandem (period U{2..100},
             copies U{10..200}), 5 % copies of a 6 kbp element with 0.5 %
             substitutions; plus 10 M reads of 150 bp at 1x.
``two_cut``  the paper's own model (Sec. III, Fig. 2): one genome cut by two
             shotguns into two sets of consecutive pieces, all break positions
             different (Fig. 4) and at least ``min_gap`` apart; the pieces of
             both cuttings shuffled into one fragment set.  Optionally with
             tandem arrays or repeated elements (ambiguous fir relations).
"""
from __future__ import annotations

import numpy as np

BASES = np.frombuffer(b"ACGT", dtype=np.uint8)
SEP = ord("$")


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def iid(rng: np.random.Generator, n: int) -> np.ndarray:
    """n i.i.d. uniform bases as ASCII bytes."""
    return BASES[rng.integers(0, 4, size=int(n), dtype=np.uint8)]


def substitute(rng: np.random.Generator, seq: np.ndarray, p: float) -> np.ndarray:
    """Each position replaced with probability p by one of the 3 other bases, uniformly."""
    codes = np.searchsorted(BASES, seq).astype(np.uint8)  # A,C,G,T -> 0..3 (BASES is sorted)
    hit = rng.random(seq.shape) < p
    shift = rng.integers(1, 4, size=seq.shape, dtype=np.uint8)
    codes = np.where(hit, (codes + shift) % 4, codes).astype(np.uint8)
    return BASES[codes]


def genome_with_repeats(rng, G: int, frac_tandem: float, period: tuple, copies: tuple,
                        frac_elem: float = 0.0, elem_len: int = 0, elem_subst: float = 0.0):
    """A genome of exactly G bases: i.i.d. segments with tandem arrays and
    element copies inserted at uniformly shuffled points between them."""
    blocks = []
    budget = int(round(frac_tandem * G))
    used = 0
    while used < budget:
        P = int(rng.integers(period[0], period[1] + 1))
        C = int(rng.integers(copies[0], copies[1] + 1))
        arr = np.tile(iid(rng, P), C)[: budget - used]
        blocks.append(arr)
        used += arr.size
    if frac_elem > 0 and elem_len > 0:
        elem = iid(rng, elem_len)
        n_copies = int(round(frac_elem * G)) // elem_len
        if n_copies:
            mat = np.broadcast_to(elem, (n_copies, elem_len))
            mat = substitute(rng, mat, elem_subst)
            blocks.extend(list(mat))
    order = rng.permutation(len(blocks)) if blocks else np.zeros(0, dtype=np.int64)
    blocks = [blocks[i] for i in order]
    n_iid = G - sum(b.size for b in blocks)
    if n_iid < 0:
        raise ValueError("repeat fractions exceed the genome")
    body = iid(rng, n_iid)
    cuts = np.sort(rng.integers(0, n_iid + 1, size=len(blocks)))
    parts = []
    prev = 0
    for c, b in zip(cuts, blocks):
        parts.append(body[prev:c])
        parts.append(b)
        prev = c
    parts.append(body[prev:])
    g = np.concatenate(parts) if parts else body
    assert g.size == G
    return g


def join_reads(reads) -> np.ndarray:
    """Fragments joined into one text, each followed by '$'."""
    total = sum(int(r.size) + 1 for r in reads)
    out = np.empty(total, dtype=np.uint8)
    pos = 0
    for r in reads:
        out[pos: pos + r.size] = r
        out[pos + r.size] = SEP
        pos += r.size + 1
    return out


def genome_text(genome: np.ndarray) -> np.ndarray:
    """A single genome as a one-fragment text (genome + '$')."""
    return join_reads([genome])


def _kmers_unique(g: np.ndarray, k: int) -> bool:
    if g.size < k:
        return True
    view = np.lib.stride_tricks.sliding_window_view(g, k)
    packed = np.ascontiguousarray(view).view(np.dtype((np.void, k))).ravel()
    return np.unique(packed).size == packed.size


def tiny(seed: int, G: int = 10_000, read_len: int = 400, n_random: int = 200,
         min_overlap: int = 31):
    """The tiny workload.  Returns dict(genome, reads, starts, text, min_overlap)."""
    rng = rng_for(seed, 1)
    while True:
        genome = iid(rng, G)
        if _kmers_unique(genome, min_overlap):
            break
    max_gap = read_len - min_overlap
    while True:
        pick = rng.choice(np.arange(1, G - read_len), size=n_random, replace=False)
        starts = np.sort(np.concatenate([[0, G - read_len], pick]))
        if np.all(np.diff(starts) <= max_gap):
            break
    order = rng.permutation(starts.size)
    starts = starts[order]
    reads = [genome[s: s + read_len] for s in starts]
    return dict(genome=genome, reads=reads, starts=starts, text=join_reads(reads),
                min_overlap=min_overlap)


def shotgun(rng, genome: np.ndarray, coverage: float, len_lo: int, len_hi: int):
    """Error-free reads of length U{len_lo..len_hi} at uniform starts until the
    read bases reach coverage x |genome|.  Returns (reads, starts)."""
    G = genome.size
    target = coverage * G
    mean = (len_lo + len_hi) / 2.0
    lens = np.zeros(0, dtype=np.int64)
    while lens.sum() < target:
        more = rng.integers(len_lo, len_hi + 1, size=int(target / mean * 1.1) + 16)
        lens = np.concatenate([lens, np.minimum(more, G)])
    cut = int(np.searchsorted(np.cumsum(lens), target)) + 1
    lens = lens[:cut]
    starts = rng.integers(0, G - lens + 1)
    reads = [genome[s: s + n] for s, n in zip(starts, lens)]
    return reads, starts.astype(np.int64)


def shotgun_fixed_text(rng, genome: np.ndarray, coverage: float, read_len: int):
    """Reads of one length at uniform starts until coverage x |genome| bases, as a
    '$'-joined text (vectorised).  Returns (text, starts)."""
    G = genome.size
    L = min(read_len, G)
    n = int(np.ceil(coverage * G / L))
    starts = rng.integers(0, G - L + 1, size=n)
    text = np.empty((n, L + 1), dtype=np.uint8)
    text[:, :L] = genome[starts[:, None] + np.arange(L)[None, :]]
    text[:, L] = SEP
    return text.ravel(), starts.astype(np.int64)


def log_uniform(rng, lo: float, hi: float) -> int:
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))


def batched_instance(seed: int, index: int, g_lo: int = 2_000, g_hi: int = 200_000,
                     coverage: float = 8.0, len_lo: int = 100, len_hi: int = 1000,
                     min_overlap: int = 31):
    rng = rng_for(seed * 1_000_003 + index, 3)
    G = log_uniform(rng, g_lo, g_hi)
    genome = iid(rng, G)
    reads, starts = shotgun(rng, genome, coverage, len_lo, len_hi)
    return dict(genome=genome, reads=reads, starts=starts, text=join_reads(reads),
                min_overlap=min_overlap)


def batched(seed: int, n_instances: int = 4096, **kw):
    return [batched_instance(seed, i, **kw) for i in range(n_instances)]


def served_job(seed: int, index: int, g_lo: int = 5_000, g_hi: int = 5_000_000,
               coverage: float = 10.0, read_len: int = 150, min_overlap: int = 41):
    rng = rng_for(seed * 1_000_003 + index, 4)
    G = log_uniform(rng, g_lo, g_hi)
    genome = genome_with_repeats(rng, G, 0.02, (2, 50), (10, 200))
    text, starts = shotgun_fixed_text(rng, genome, coverage, read_len)
    return dict(genome=genome, starts=starts, text=text, min_overlap=min_overlap)


def sa64m_genome(seed: int, G: int = 64_000_000) -> np.ndarray:
    rng = rng_for(seed, 2)
    return genome_with_repeats(rng, G, 0.05, (2, 50), (10, 200), 0.05, 300, 0.01)


def large_genome(seed: int, G: int = 1_500_000_000) -> np.ndarray:
    rng = rng_for(seed, 5)
    return genome_with_repeats(rng, G, 0.10, (2, 100), (10, 200), 0.05, 6000, 0.005)


def large_reads(seed: int, genome: np.ndarray, n_reads: int = 10_000_000, read_len: int = 150):
    """n_reads fragments of read_len at uniform starts, as one '$'-joined text."""
    rng = rng_for(seed, 6)
    starts = rng.integers(0, genome.size - read_len + 1, size=n_reads)
    text = np.empty((n_reads, read_len + 1), dtype=np.uint8)
    cols = np.arange(read_len)[None, :]
    for c0 in range(0, n_reads, 1 << 20):   # bounded index arrays
        c1 = min(n_reads, c0 + (1 << 20))
        text[c0:c1, :read_len] = genome[starts[c0:c1, None] + cols]
    text[:, read_len] = SEP
    return text.ravel(), starts


def two_cut(seed: int, G: int, mean_len: int = 500, min_gap: int = 24, frac_tandem: float = 0.0,
            period: tuple = (2, 50), copies: tuple = (10, 200), frac_elem: float = 0.0,
            elem_len: int = 0, elem_subst: float = 0.0, genome: np.ndarray | None = None):
    """A genome cut twice (Sec. III, Fig. 2).  About G / mean_len pieces per
    cutting; the union of both cuttings' break positions is drawn with every two
    breaks at least min_gap apart (so every piece and every remainder is at
    least min_gap long), and each break goes to one of the two cuttings at
    random.  Returns dict(genome, text, frag_start (true offset of each fragment
    in the genome, in text order), cut (0/1 per fragment))."""
    rng = rng_for(seed, 7)
    if genome is None:
        genome = (genome_with_repeats(rng, G, frac_tandem, period, copies, frac_elem, elem_len,
                                      elem_subst)
                  if (frac_tandem > 0 or frac_elem > 0) else iid(rng, G))
    G = int(genome.size)
    K = max(2, 2 * int(round(G / mean_len)) - 2)        # breaks of both cuttings together
    K = min(K, G // min_gap - 1)
    free = G - (K + 1) * min_gap
    if K < 2 or free < 0:
        raise ValueError("genome too short for two cuttings with this min_gap")
    u = np.sort(rng.integers(0, free + 1, size=K))
    breaks = u + min_gap * np.arange(1, K + 1)           # strictly increasing, gaps >= min_gap
    side = rng.integers(0, 2, size=K)
    side[0], side[1] = 0, 1                              # each cutting breaks at least once
    frags, starts, cuts = [], [], []
    for c in (0, 1):
        b = np.concatenate([[0], breaks[side == c], [G]])
        for a, e in zip(b[:-1], b[1:]):
            frags.append(genome[a:e])
            starts.append(int(a))
            cuts.append(c)
    order = rng.permutation(len(frags))
    frags = [frags[i] for i in order]
    return dict(genome=genome, text=join_reads(frags), frag_start=np.array(starts)[order],
                cut=np.array(cuts)[order])
