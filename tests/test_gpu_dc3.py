"""The DC3 (difference-cover, skew) suffix-array builder (sa_build option
builder = 1; the construction the paper's GPU kernel is named after, Sec. IV)
against the oracle's suffix array, through the C ABI: bit-exact."""
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


def dc3_sa(ctx, t, dtype=torch.int32):
    text = torch.from_numpy(np.array(t, dtype=np.uint8, copy=True)).cuda()
    sa, packed, toff, nr = B().suffix_array(ctx, text, dtype=dtype, opts=B().make_opts(builder=1))
    return sa.cpu().numpy().astype(np.int64), packed, toff, nr, text


@pytest.mark.parametrize("text", [b"A$", b"C$", b"AA$", b"ACG$", b"AAAAAAAA$", b"A$A$AA$",
                                  b"T$G$C$A$", b"ACGT" * 40 + b"$", b"GATTACA$"])
def test_dc3_small_texts(ctx, text):
    t = np.frombuffer(text, np.uint8)
    assert np.array_equal(dc3_sa(ctx, t)[0], oracle.suffix_array(t))


@pytest.mark.parametrize("n", list(range(2, 40)))
def test_dc3_every_length_mod_3(ctx, n):
    """Lengths 2..39 (every residue mod 3 at several recursion depths): runs of one
    base recurse the deepest."""
    rng = np.random.default_rng(n)
    for t in (synth.genome_text(np.full(n - 1, ord("A"), np.uint8)),
              synth.genome_text(synth.iid(rng, n - 1))):
        assert np.array_equal(dc3_sa(ctx, t)[0], oracle.suffix_array(t)), t.tobytes()


@pytest.mark.parametrize("seed,n_reads,lo,hi", [(1, 40, 1, 200), (2, 300, 50, 2000), (3, 2000, 1, 60)])
def test_dc3_multi_fragment(ctx, seed, n_reads, lo, hi):
    rng = np.random.default_rng(seed)
    reads = []
    for _ in range(n_reads):
        n = int(rng.integers(lo, hi + 1))
        if rng.random() < 0.3:
            unit = synth.iid(rng, int(rng.integers(1, 6)))
            reads.append(np.tile(unit, n // unit.size + 1)[:n])
        else:
            reads.append(synth.iid(rng, n))
    t = synth.join_reads(reads)
    assert np.array_equal(dc3_sa(ctx, t)[0], oracle.suffix_array(t))


def test_dc3_repeat_genome_and_lcp(ctx):
    rng = synth.rng_for(7, 11)
    g = synth.genome_with_repeats(rng, 400_003, 0.05, (2, 50), (10, 200), 0.05, 300, 0.01)
    t = synth.genome_text(g)
    want = oracle.suffix_array(t)
    got, packed, toff, nr, _ = dc3_sa(ctx, t)
    assert np.array_equal(got, want)
    assert ctx.trace()["rounds"] >= 3   # recursion levels
    sa = torch.from_numpy(got.astype(np.int32)).cuda()
    lcp = torch.empty_like(sa)
    B().lcp_build(ctx, packed, toff, nr, t.size, sa, lcp)
    assert np.array_equal(lcp.cpu().numpy(), oracle.lcp_kasai(t, want))


def test_dc3_all_same_base_int64(ctx):
    t = synth.genome_text(np.full(30_000, ord("A"), np.uint8))
    got = dc3_sa(ctx, t, dtype=torch.int64)[0]
    assert np.array_equal(got, np.arange(t.size)[::-1])


def test_dc3_equals_doubling_on_64mbp_prefix(ctx):
    """A 4 Mbp prefix of the benchmark genome: both builders give one array, and
    the oracle's linear checker accepts it."""
    t = synth.genome_text(synth.sa64m_genome(1)[:4_000_000])
    got = dc3_sa(ctx, t)[0]
    text = torch.from_numpy(t).cuda()
    sa2 = B().suffix_array(ctx, text)[0].cpu().numpy().astype(np.int64)
    assert np.array_equal(got, sa2)
    assert oracle.sa_check(t, got) == 0


def test_dc3_refused_for_batches(ctx):
    texts = [np.frombuffer(b"ACGT$", np.uint8).copy(), np.frombuffer(b"GGA$", np.uint8).copy()]
    inst_off = np.array([0, 5, 9], dtype=np.int64)
    joined = torch.from_numpy(np.concatenate(texts)).cuda()
    packed, toff, nr = B().pack_text(ctx, joined)
    sa = torch.empty(9, dtype=torch.int32, device="cuda")
    with pytest.raises(B().DnasaError):
        B().sa_build_batched(ctx, packed, toff, nr, 9, inst_off, sa, B().make_opts(builder=1))
