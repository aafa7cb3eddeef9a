"""GPU-vs-oracle parity through the C ABI.  Everything is integer/index work,
so the bar is bit-exact equality on every output array."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1404_3456_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3456_gb300 import binding

    c = binding.Context(0)
    yield c
    c.close()


def B():
    from paper_1404_3456_gb300 import binding

    return binding


def dev(a: np.ndarray):
    return torch.from_numpy(np.array(a, dtype=np.uint8, copy=True)).cuda()


def random_text(rng, n_reads, lo, hi, periodic_frac=0.3, dup=True):
    reads = []
    for _ in range(n_reads):
        n = int(rng.integers(lo, hi + 1))
        if rng.random() < periodic_frac:
            unit = synth.iid(rng, int(rng.integers(1, 6)))
            r = np.tile(unit, n // unit.size + 1)[:n]
        else:
            r = synth.iid(rng, n)
        reads.append(r)
    if dup and n_reads >= 4:
        reads[1] = reads[0].copy()
        reads[2] = reads[0][1:].copy() if reads[0].size > 1 else reads[2]
    return synth.join_reads(reads)


def gpu_sa(ctx, text_np, dtype=torch.int32, opts=None):
    text = dev(text_np)
    sa, packed, toff, nr = B().suffix_array(ctx, text, dtype=dtype, opts=opts)
    return sa, packed, toff, nr, text


# ---------------------------------------------------------------- pack


def test_pack_offsets_and_codes(ctx):
    rng = np.random.default_rng(1)
    t = random_text(rng, 50, 1, 300)
    text = dev(t)
    packed, toff, nr = B().pack_text(ctx, text)
    assert nr == int((t == ord("$")).sum())
    assert np.array_equal(toff.cpu().numpy(), oracle.read_offsets(t))
    # decode the 2-bit words and compare with the bases of the text
    words = packed.cpu().numpy().view(np.uint64)
    bases = t[t != ord("$")]
    idx = np.arange(bases.size)
    codes = (words[idx // 32] >> (62 - 2 * (idx % 32)).astype(np.uint64)) & np.uint64(3)
    assert np.array_equal(np.frombuffer(b"ACGT", np.uint8)[codes.astype(np.int64)], bases)
    assert np.all(words[(bases.size + 31) // 32:] == 0)


@pytest.mark.parametrize("bad", [b"ACGN$", b"ACGT", b"AC$$GT$", b"$AC$", b"$", b"acgt$"])
def test_pack_rejects_bad_text(ctx, bad):
    text = dev(np.frombuffer(bad, np.uint8))
    with pytest.raises(B().DnasaError) as e:
        B().pack_text(ctx, text)
    assert e.value.status == B().BAD_ALPHABET


# ---------------------------------------------------------------- suffix array


@pytest.mark.parametrize("text", [b"A$", b"AAAAAAAA$", b"ACGTACGTACGT$", b"A$A$AA$",
                                  b"T$G$C$A$", b"ACGT" * 40 + b"$"])
def test_sa_small_texts(ctx, text):
    t = np.frombuffer(text, np.uint8)
    sa = gpu_sa(ctx, t)[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))


@pytest.mark.parametrize("seed,n_reads,lo,hi", [(0, 1, 100_000, 100_000), (1, 40, 1, 200),
                                                (2, 300, 50, 2000), (3, 2000, 1, 60),
                                                (4, 8, 20_000, 40_000)])
def test_sa_random_multi_read(ctx, seed, n_reads, lo, hi):
    rng = np.random.default_rng(seed)
    t = random_text(rng, n_reads, lo, hi)
    sa = gpu_sa(ctx, t)[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))


def test_sa_repeat_genome(ctx):
    """Tandem arrays and element copies: deep doubling rounds, several tiles, ragged tail."""
    rng = synth.rng_for(7, 11)
    g = synth.genome_with_repeats(rng, 400_003, 0.05, (2, 50), (10, 200), 0.05, 300, 0.01)
    t = synth.genome_text(g)
    want = oracle.suffix_array(t)
    sa = gpu_sa(ctx, t, opts=B().make_opts(finish_threshold=-1))[0]   # doubling only
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), want)
    tr = ctx.trace()
    assert tr["rounds"] >= 2 and tr["finished_direct"] == 0
    sa, packed, toff, nr, _ = gpu_sa(ctx, t)                           # default switch
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), want)
    lcp = torch.empty_like(sa)
    B().lcp_build(ctx, packed, toff, nr, t.size, sa, lcp)              # long LCPs: warp path
    assert np.array_equal(lcp.cpu().numpy(), oracle.lcp_kasai(t, want))


@pytest.mark.parametrize("finish", [-1, 1 << 40])
def test_sa_finisher_and_doubling_agree(ctx, finish):
    rng = synth.rng_for(8, 11)
    g = synth.genome_with_repeats(rng, 200_000, 0.10, (2, 50), (10, 100), 0.05, 300, 0.01)
    t = synth.genome_text(g)
    opts = B().make_opts(finish_threshold=finish)
    sa = gpu_sa(ctx, t, opts=opts)[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))
    assert ctx.trace()["finished_direct"] == (1 if finish > 0 else 0)


@pytest.mark.parametrize("seg_max", [8, 32, 256, 2048, 12288])
def test_sa_group_sort_tiers(ctx, seg_max):
    """Doubling rounds only, on a text whose groups span every in-group sorting
    tier (thread, warp registers, CTA radix in shared memory, global radix passes): 3,000 copies
    of a 40 bp element give groups of thousands of members."""
    rng = synth.rng_for(12, 11)
    g = synth.genome_with_repeats(rng, 400_000, 0.05, (2, 50), (10, 200), 0.30, 40, 0.01)
    t = synth.genome_text(g)
    sa = gpu_sa(ctx, t, opts=B().make_opts(finish_threshold=-1, seg_max=seg_max))[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))
    assert ctx.trace()["rounds"] >= 2


def tandem_text(rng, arrays, flank=(0, 400), reads=1, end_with_array=True):
    """Random flanks around tandem arrays (p, c, name): c copies of a unit of p
    bases, one unit per name (arrays of one name repeat one unit); several reads
    if asked, the last array of each read running up to its '$' unless
    end_with_array is False."""
    parts = [[] for _ in range(reads)]
    units = {}
    for k, (p, c, name) in enumerate(arrays):
        if name not in units:
            units[name] = synth.iid(rng, p)
        r = k % reads
        parts[r].append(synth.iid(rng, int(rng.integers(flank[0], flank[1] + 1))))
        parts[r].append(np.tile(units[name], c))
    if not end_with_array:
        for r in range(reads):
            parts[r].append(synth.iid(rng, 50))
    return synth.join_reads([np.concatenate(x) if x else synth.iid(rng, 10) for x in parts])


# (unit length, copies, unit name): phase groups of 3..8, 9..32, 33..256 and 257..6000
# members, periods below and above the initial key length, a homopolymer, and one
# unit in two arrays (its phase groups are then no single progression)
TANDEM_ARRAYS = [(1, 40, "a"), (2, 6, "b"), (3, 50, "c"), (5, 400, "d"), (7, 1000, "e"),
                 (19, 20, "f"), (20, 300, "g"), (33, 40, "h"), (50, 12, "i"), (64, 100, "j"),
                 (2, 3000, "k"), (4, 8, "l"), (11, 200, "m"), (7, 700, "e")]


@pytest.mark.parametrize("seg_max", [8, 256, 12288])
@pytest.mark.parametrize("reads,end_with_array", [(1, True), (1, False), (5, True), (5, False)])
def test_sa_tandem_progressions(ctx, seg_max, reads, end_with_array):
    """Groups whose members form one arithmetic progression (a phase of a tandem
    array) are ordered at once in every on-chip tier; the SA equals the oracle's."""
    rng = np.random.default_rng(31 + reads)
    t = tandem_text(rng, TANDEM_ARRAYS, reads=reads, end_with_array=end_with_array)
    sa = gpu_sa(ctx, t, opts=B().make_opts(finish_threshold=-1, seg_max=seg_max))[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))


def test_sa_tandem_rounds(ctx):
    """One 21,000 bp array of a 7 bp unit: its phase groups are progressions with
    p = 7 below the initial key length, so they are ordered in the first doubling
    round instead of log2(21,000 / h0) rounds later."""
    rng = np.random.default_rng(5)
    g = np.concatenate([synth.iid(rng, 200), np.tile(synth.iid(rng, 7), 3000), synth.iid(rng, 200)])
    t = synth.genome_text(g)
    sa = gpu_sa(ctx, t, opts=B().make_opts(finish_threshold=-1))[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))
    tr = ctx.trace()
    assert tr["h0"] >= 7 and tr["rounds"] <= 2, tr


GRAPH_TEXTS = ["repeat", "tandem", "multi", "tiny"]


def graph_text(kind):
    if kind == "repeat":
        rng = synth.rng_for(7, 11)
        return synth.genome_text(synth.genome_with_repeats(rng, 400_003, 0.05, (2, 50), (10, 200),
                                                           0.05, 300, 0.01))
    if kind == "tandem":
        return tandem_text(np.random.default_rng(40), TANDEM_ARRAYS, reads=3)
    if kind == "multi":
        return random_text(np.random.default_rng(41), 300, 50, 2000)
    return np.frombuffer(b"ACGTACGTAC$ACGTT$", np.uint8)


class FixedBuffers:
    """One text packed once and one SA buffer, so that repeated builds present the
    same configuration (the graph of the doubling rounds is captured on the second)."""

    def __init__(self, ctx, t):
        self.ctx, self.t = ctx, t
        self.packed, self.toff, self.nr = B().pack_text(ctx, dev(t))
        self.sa = torch.empty(t.size, dtype=torch.int32, device="cuda")

    def build(self, opts=None):
        B().sa_build(self.ctx, self.packed, self.toff, self.nr, self.t.size, self.sa, opts)
        return self.sa.cpu().numpy().astype(np.int64), self.ctx.trace()


@pytest.mark.parametrize("kind", GRAPH_TEXTS)
def test_sa_graph_rounds_equal_host_rounds(ctx, kind):
    """The doubling rounds run as one captured graph (a device-side WHILE loop)
    or from the host: the same SA (the oracle's), the same rounds and actives.  The
    first build of a configuration runs its rounds from the host; a repeat is
    captured and runs in the graph."""
    t = graph_text(kind)
    want = oracle.suffix_array(t)
    fb = FixedBuffers(ctx, t)
    got, host = fb.build(B().make_opts(rounds_on_host=1))
    assert np.array_equal(got, want) and host["graph_rounds"] == 0
    got, first = fb.build()
    assert np.array_equal(got, want) and first["graph_rounds"] == 0   # first sight: host rounds
    got, dev_tr = fb.build()
    assert np.array_equal(got, want)
    assert dev_tr["rounds"] == host["rounds"] and dev_tr["active"] == host["active"]
    assert dev_tr["graph_rounds"] == dev_tr["rounds"]
    got, again = fb.build()                                            # the cached graph
    assert np.array_equal(got, want) and again["graph_rounds"] == again["rounds"]


def test_sa_graph_recaptured_for_new_sizes(ctx):
    """Graphs are kept per configuration (buffers and sizes) and reused: builds of
    several texts interleaved, each repeated, all equal the oracle; from the second
    build of a configuration on, its rounds run in the graph."""
    bufs = [FixedBuffers(ctx, graph_text(k)) for k in ("repeat", "multi", "tandem")]
    wants = [oracle.suffix_array(fb.t) for fb in bufs]
    for it in range(3):
        for fb, want in zip(bufs, wants):
            got, tr = fb.build()
            assert np.array_equal(got, want)
            if it > 0 and tr["rounds"] > 0:
                assert tr["graph_rounds"] == tr["rounds"]


@pytest.mark.parametrize("seg_max", [8, 256])
def test_sa_graph_hands_large_groups_to_host(ctx, seg_max):
    """A group larger than the on-chip limit ends the device loop; the host runs
    the remaining rounds (global radix passes) and the SA still equals the oracle's."""
    rng = synth.rng_for(12, 11)
    t = synth.genome_text(synth.genome_with_repeats(rng, 400_000, 0.05, (2, 50), (10, 200), 0.30, 40, 0.01))
    sa = gpu_sa(ctx, t, opts=B().make_opts(seg_max=seg_max))[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))
    tr = ctx.trace()
    assert tr["graph_rounds"] < tr["rounds"]


def test_sa_graph_max_rounds(ctx):
    """max_rounds bounds the device loop as it bounds the host loop (the first
    build of the configuration runs from the host, the second in the graph)."""
    t = graph_text("repeat")
    fb = FixedBuffers(ctx, t)
    for _ in range(2):
        with pytest.raises(B().DnasaError) as e:
            fb.build(B().make_opts(max_rounds=2))
        assert e.value.status == B().INVALID_ARG
    got, _ = fb.build()   # the context is still usable
    assert np.array_equal(got, oracle.suffix_array(t))


def lcp_texts():
    rng = np.random.default_rng(50)
    return {
        "repeat": graph_text("repeat"),
        "tandem": graph_text("tandem"),
        "multi": random_text(rng, 300, 1, 2000),
        "short_reads": random_text(rng, 3000, 1, 40),
        "endings": synth.genome_text(np.tile(synth.iid(rng, 7), 40)),
        "tiny": np.frombuffer(b"ACGTACGTAC$ACGTT$A$", np.uint8),
    }


@pytest.mark.parametrize("kind", ["repeat", "tandem", "multi", "short_reads", "endings", "tiny"])
@pytest.mark.parametrize("opts_kw", [{}, {"pack_position": -1}, {"rounds_on_host": 1}, {"builder": 1},
                                     {"finish_threshold": 1 << 40}, {"seg_max": 8}],
                         ids=["packed", "pairs", "host_rounds", "dc3", "finisher", "global_radix"])
def test_sa_lcp_build(ctx, kind, opts_kw):
    """SA and LCP in one call: round 0 writes the LCP of every pair its keys separate,
    the rest is compared on the text; both arrays equal the oracle's."""
    t = lcp_texts()[kind]
    want = oracle.suffix_array(t)
    text = dev(t)
    packed, toff, nr = B().pack_text(ctx, text)
    for dtype in (torch.int32, torch.int64):
        sa = torch.empty(t.size, dtype=dtype, device="cuda")
        lcp = torch.full((t.size,), -7, dtype=torch.int32, device="cuda")
        B().sa_lcp_build(ctx, packed, toff, nr, t.size, sa, lcp, B().make_opts(**opts_kw))
        assert np.array_equal(sa.cpu().numpy().astype(np.int64), want)
        assert np.array_equal(lcp.cpu().numpy(), oracle.lcp_kasai(t, want))


def test_sa_lcp_build_graph_cache_follows_buffers(ctx):
    """The captured rounds write LCP entries through the buffer they were captured
    with: a second LCP buffer, a plain sa_build after sa_lcp_build, and a second text
    of the same length must each get their own results and leave the others alone."""
    t1 = graph_text("tandem")
    rng = np.random.default_rng(77)
    t2 = synth.genome_text(np.concatenate([synth.iid(rng, 500), np.tile(synth.iid(rng, 5), (t1.size - 502) // 5)]))
    t2 = np.concatenate([t2[:-1], synth.iid(rng, t1.size - t2.size), np.frombuffer(b"$", np.uint8)])
    assert t2.size == t1.size
    packed1, toff1, nr1 = B().pack_text(ctx, dev(t1))
    packed2, toff2, nr2 = B().pack_text(ctx, dev(t2))
    sa = torch.empty(t1.size, dtype=torch.int32, device="cuda")
    lcp_a = torch.full((t1.size,), -7, dtype=torch.int32, device="cuda")
    lcp_b = torch.full_like(lcp_a, -7)
    want1 = oracle.suffix_array(t1)
    want2 = oracle.suffix_array(t2)
    for _ in range(2):   # the second build of each configuration runs in its captured graph
        B().sa_lcp_build(ctx, packed1, toff1, nr1, t1.size, sa, lcp_a)
        assert np.array_equal(lcp_a.cpu().numpy(), oracle.lcp_kasai(t1, want1))
    assert ctx.trace()["graph_rounds"] >= 1
    a_copy = lcp_a.clone()
    for _ in range(2):
        lcp_b.fill_(-7)
        B().sa_lcp_build(ctx, packed1, toff1, nr1, t1.size, sa, lcp_b)   # another LCP buffer
        assert np.array_equal(lcp_b.cpu().numpy(), oracle.lcp_kasai(t1, want1))
        assert torch.equal(lcp_a, a_copy)
    lcp_a.fill_(-9)
    for _ in range(2):
        B().sa_build(ctx, packed2, toff2, nr2, t2.size, sa)               # no LCP, other text
        assert np.array_equal(sa.cpu().numpy().astype(np.int64), want2)
        assert bool((lcp_a == -9).all()) and torch.equal(lcp_b.cpu(), a_copy.cpu())
    for _ in range(2):
        B().sa_lcp_build(ctx, packed2, toff2, nr2, t2.size, sa, lcp_a)   # other text, first buffer
        assert np.array_equal(lcp_a.cpu().numpy(), oracle.lcp_kasai(t2, want2))
    B().sa_lcp_build(ctx, packed1, toff1, nr1, t1.size, sa, lcp_b)       # back to a cached graph
    assert np.array_equal(lcp_b.cpu().numpy(), oracle.lcp_kasai(t1, want1))
    assert ctx.trace()["graph_rounds"] >= 1


def test_sa_lcp_build_unaligned_lcp(ctx):
    """An LCP buffer that starts 4 bytes into an allocation (not 16-byte aligned)
    is filled entirely and correctly."""
    t = graph_text("repeat")
    want = oracle.suffix_array(t)
    packed, toff, nr = B().pack_text(ctx, dev(t))
    sa = torch.empty(t.size, dtype=torch.int32, device="cuda")
    big = torch.full((t.size + 1,), -7, dtype=torch.int32, device="cuda")
    lcp = big[1:]
    assert lcp.data_ptr() % 16 != 0
    B().sa_lcp_build(ctx, packed, toff, nr, t.size, sa, lcp)
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), want)
    assert np.array_equal(lcp.cpu().numpy(), oracle.lcp_kasai(t, want))
    assert int(big[0]) == -7


def test_sa_lcp_build_64m_sampled(ctx):
    """The fused call on the 64 Mbp benchmark genome equals the separate calls."""
    g = synth.sa64m_genome(1)
    t = synth.genome_text(g)
    text = dev(t)
    packed, toff, nr = B().pack_text(ctx, text)
    del text
    sa1 = torch.empty(t.size, dtype=torch.int32, device="cuda")
    lcp1 = torch.empty_like(sa1)
    B().sa_build(ctx, packed, toff, nr, t.size, sa1)
    B().lcp_build(ctx, packed, toff, nr, t.size, sa1, lcp1)
    sa2 = torch.empty_like(sa1)
    lcp2 = torch.empty_like(sa1)
    B().sa_lcp_build(ctx, packed, toff, nr, t.size, sa2, lcp2)
    assert torch.equal(sa1, sa2) and torch.equal(lcp1, lcp2)


@pytest.mark.parametrize("pack", [0, -1])
@pytest.mark.parametrize("seed,n_reads,lo,hi", [(21, 1, 300_001, 300_001), (22, 700, 1, 900)])
def test_sa_packed_and_pair_initial_sort(ctx, pack, seed, n_reads, lo, hi):
    """The initial sort on one packed (key, position) word and on (key, position)
    pairs: the same suffix array; the trace says which form ran."""
    rng = np.random.default_rng(seed)
    t = random_text(rng, n_reads, lo, hi)
    sa = gpu_sa(ctx, t, opts=B().make_opts(pack_position=pack))[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))
    pb = ctx.trace()["pack_bits"]
    if pack < 0:
        assert pb == 0
    else:
        assert pb == int(t.size - 1).bit_length()


def test_sa_pack_position_rejected(ctx):
    rng = np.random.default_rng(23)
    t = random_text(rng, 3, 10, 20)
    with pytest.raises(B().DnasaError):
        gpu_sa(ctx, t, opts=B().make_opts(pack_position=1))


@pytest.mark.parametrize("tile", [2048, 3840, 5120])
def test_sa_tile_sizes(ctx, tile):
    rng = np.random.default_rng(9)
    t = random_text(rng, 500, 10, 600)
    sa = gpu_sa(ctx, t, opts=B().make_opts(tile_items=tile))[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))


def test_sa_int64(ctx):
    rng = np.random.default_rng(10)
    t = random_text(rng, 30, 1, 500)
    sa = gpu_sa(ctx, t, dtype=torch.int64)[0]
    assert sa.dtype == torch.int64
    assert np.array_equal(sa.cpu().numpy(), oracle.suffix_array(t))


@pytest.mark.parametrize("seed", range(6))
def test_sa_single_sequence_endings(ctx, seed):
    """One sequence: its last h0 suffixes reach the '$' inside the initial key and
    sort before every suffix that shares their bases (shorter first).  Endings made
    of A's (whose bases equal the zero padding), runs of one base, periodic tails
    and random lengths around the key and tile sizes."""
    rng = np.random.default_rng(400 + seed)
    A = np.frombuffer(b"ACGT", np.uint8)
    cases = [np.full(int(rng.integers(1, 40)), ord("A"), np.uint8),
             np.concatenate([A[rng.integers(0, 4, int(rng.integers(1, 3000)))],
                             np.full(int(rng.integers(1, 40)), ord("A"), np.uint8)]),
             np.tile(A[rng.integers(0, 4, int(rng.integers(1, 5)))], int(rng.integers(1, 400))),
             A[rng.integers(0, 4, int(rng.integers(1, 20)))],
             np.concatenate([np.tile(np.frombuffer(b"CA", np.uint8), 2000),
                             A[rng.integers(0, 4, int(rng.integers(0, 17)))]])]
    for g in cases:
        t = synth.genome_text(g)
        sa = gpu_sa(ctx, t)[0]
        assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t)), g[-40:].tobytes()


def test_sa_all_same_base(ctx):
    t = synth.genome_text(np.full(50_000, ord("A"), np.uint8))
    sa = gpu_sa(ctx, t)[0]
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), np.arange(t.size)[::-1])


# ---------------------------------------------------------------- LCP


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lcp_parity(ctx, seed):
    rng = np.random.default_rng(20 + seed)
    t = random_text(rng, 200, 1, 800)
    sa, packed, toff, nr, text = gpu_sa(ctx, t)
    lcp = torch.empty_like(sa)
    B().lcp_build(ctx, packed, toff, nr, t.size, sa, lcp)
    want = oracle.lcp_kasai(t, oracle.suffix_array(t))
    assert np.array_equal(lcp.cpu().numpy(), want)


# ---------------------------------------------------------------- overlaps and containment


def overlaps_gpu(ctx, t, lmin):
    sa, packed, toff, nr, text = gpu_sa(ctx, t)
    lcp = torch.empty_like(sa)
    B().lcp_build(ctx, packed, toff, nr, t.size, sa, lcp)
    cap = nr * nr + 16
    edges = torch.empty((cap, 3), dtype=torch.int32, device="cuda")
    contained = torch.empty(nr, dtype=torch.uint8, device="cuda")
    ne = B().overlap_search(ctx, packed, toff, nr, t.size, sa, lcp, lmin, edges, contained)
    e = edges[:ne].cpu().numpy()
    return e, contained.cpu().numpy()


@pytest.mark.parametrize("seed,lmin", [(0, 1), (1, 3), (2, 8), (3, 2)])
def test_overlap_parity_random(ctx, seed, lmin):
    rng = np.random.default_rng(30 + seed)
    t = random_text(rng, 120, 1, 80, periodic_frac=0.4)
    e, c = overlaps_gpu(ctx, t, lmin)
    ej, ek, eL = oracle.overlaps_sorted(t, lmin)
    assert np.array_equal(e[:, 0], ej) and np.array_equal(e[:, 1], ek) and np.array_equal(e[:, 2], eL)
    assert np.array_equal(c, oracle.contained(t))


def test_overlap_parity_tiny(ctx):
    inst = synth.tiny(3)
    e, c = overlaps_gpu(ctx, inst["text"], 31)
    ej, ek, eL = oracle.overlaps_sorted(inst["text"], 31)
    assert np.array_equal(e, np.stack([ej, ek, eL], 1))
    assert not c.any()


def test_overlap_parity_batched_instance(ctx):
    inst = synth.batched_instance(5, 0, g_lo=3000, g_hi=5000)
    e, c = overlaps_gpu(ctx, inst["text"], 31)
    ej, ek, eL = oracle.overlaps_sorted(inst["text"], 31)
    assert np.array_equal(e, np.stack([ej, ek, eL], 1))
    assert np.array_equal(c, oracle.contained(inst["text"]))


def test_overlap_parity_reads_with_repeats(ctx):
    """30,000 reads of 150 bp (4.5x) from a 1 Mbp genome with tandem arrays and
    60 copies of a 500 bp element: 4.5 M symbols, hundreds of SA tiles and
    thousands of query tiles, repeat-driven overlap sets of hundreds of
    fragments -- every edge and every containment flag against the oracle."""
    rng = synth.rng_for(40, 12)
    g = synth.genome_with_repeats(rng, 1_000_000, 0.05, (2, 50), (10, 200), 0.03, 500, 0.01)
    t, _ = synth.large_reads(41, g, 30_000, 150)
    ej, ek, eL = oracle.overlaps_sorted(t, 31)
    sa, packed, toff, nr, _ = gpu_sa(ctx, t)
    lcp = torch.empty_like(sa)
    B().lcp_build(ctx, packed, toff, nr, t.size, sa, lcp)
    edges = torch.empty((ej.size + 1024, 3), dtype=torch.int32, device="cuda")
    contained = torch.empty(nr, dtype=torch.uint8, device="cuda")
    ne = B().overlap_search(ctx, packed, toff, nr, t.size, sa, lcp, 31, edges, contained)
    assert ne == ej.size
    assert np.array_equal(edges[:ne].cpu().numpy(), np.stack([ej, ek, eL], 1))
    assert np.array_equal(contained.cpu().numpy(), oracle.contained(t))


# ---------------------------------------------------------------- assemble


@pytest.mark.parametrize("seed", range(10))
def test_assemble_tiny_recovers_genome(ctx, seed):
    inst = synth.tiny(seed)
    contigs = B().assemble_text(ctx, dev(inst["text"]), inst["min_overlap"])
    assert contigs == [inst["genome"].tobytes()]


def test_assemble_parity_with_oracle(ctx):
    inst = synth.batched_instance(6, 1, g_lo=4000, g_hi=6000)
    got = B().assemble_text(ctx, dev(inst["text"]), 31)
    buf, off = oracle.assemble(inst["text"], 31)
    assert got == oracle.contigs_as_list(buf, off)


def test_assemble_worked_example_dna(ctx):
    """The paper's Sec. III example re-spelt over ACGT (a->A, b->C, h->G, p->T, t->A is
    not injective, so use a DNA instance with the same overlap structure)."""
    reads = [b"ACGTTGCA", b"TTGCAGGA", b"CAGGATCC", b"GATCCTAA"]
    t = np.frombuffer(b"$".join(reads) + b"$", np.uint8)
    got = B().assemble_text(ctx, dev(t), 2)
    buf, off = oracle.assemble(t, 2)
    assert got == oracle.contigs_as_list(buf, off)


# ---------------------------------------------------------------- radix sort (Algorithm 1)


@pytest.mark.parametrize("kind", ["all_equal", "sorted", "reverse", "two_values"])
def test_sort_pairs_special_orders(ctx, kind):
    """Stable order on key distributions that stress the digit ranking: one key
    for all, already sorted, reversed, two alternating keys."""
    n = 3840 * 7 + 123
    if kind == "all_equal":
        k = np.full(n, 0x1234_5678_9ABC, dtype=np.uint64)
    elif kind == "sorted":
        k = np.arange(n, dtype=np.uint64) * np.uint64(0x10001)
    elif kind == "reverse":
        k = (np.arange(n, dtype=np.uint64)[::-1] * np.uint64(0x10001)).copy()
    else:
        k = np.where(np.arange(n) % 2 == 0, 7, 3).astype(np.uint64)
    v = np.arange(n, dtype=np.uint32)
    kt = torch.from_numpy(k.view(np.int64).copy()).cuda()
    vt = torch.from_numpy(v.view(np.int32).copy()).cuda()
    B().dnasa_sort_pairs(ctx, kt, vt, 48, 3840, 8)
    order = np.argsort(k, kind="stable")
    assert np.array_equal(kt.cpu().numpy().view(np.uint64), k[order])
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), v[order])


@pytest.mark.parametrize("n,bits,tile,lb,with_vals", [
    (1, 64, 0, 0, True), (1000, 8, 2048, 1, True), (100_003, 63, 3840, 8, True),
    (300_000, 52, 5120, 8, True), (70_000, 32, 0, 1, False), (3840 * 5 + 17, 17, 3840, 1, True)])
def test_sort_pairs_equals_split_sort(ctx, n, bits, tile, lb, with_vals):
    """The onesweep radix sort equals Algorithm 1's 1-bit stable splits."""
    rng = np.random.default_rng(n + bits)
    keys = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n).astype(np.uint64)
    if bits < 64:
        keys &= np.uint64((1 << bits) - 1)
    keys[: n // 4] = keys[0]          # a long run of equal keys: order must be kept
    keys[n // 2: n // 2 + n // 8] = keys[-1]
    vals = np.arange(n, dtype=np.uint32)
    k_t = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v_t = torch.from_numpy(vals.view(np.int32).copy()).cuda() if with_vals else None
    B().dnasa_sort_pairs(ctx, k_t, v_t, key_bits=bits, tile_items=tile, lookback=lb)
    want_k, want_v = oracle.split_sort(keys, vals.astype(np.uint64), 0, bits)
    assert np.array_equal(k_t.cpu().numpy().view(np.uint64), want_k)
    if with_vals:
        assert np.array_equal(v_t.cpu().numpy().view(np.uint32).astype(np.uint64), want_v)


def test_sa_lookback_variants_agree(ctx):
    rng = np.random.default_rng(11)
    t = random_text(rng, 400, 10, 1000)
    want = oracle.suffix_array(t)
    for lb in (1, 8):
        sa = gpu_sa(ctx, t, opts=B().make_opts(lookback=lb))[0]
        assert np.array_equal(sa.cpu().numpy().astype(np.int64), want)
