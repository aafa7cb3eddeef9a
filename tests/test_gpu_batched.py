"""Batched: many independent fragment sets in one pass.  Each instance's
result must equal the oracle's and, byte for byte, the same instance
assembled alone (integer work: tolerance zero)."""
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


def small_batch(seed, n, g_lo=2000, g_hi=12_000):
    return [synth.batched_instance(seed, i, g_lo=g_lo, g_hi=g_hi)["text"] for i in range(n)]


def test_sa_build_batched_per_instance(ctx):
    texts = small_batch(1, 24)
    # a tiny instance and a periodic one to exercise ragged and deep cases
    texts.append(np.frombuffer(b"ACGT$A$", np.uint8).copy())
    texts.append(synth.join_reads([np.tile(np.frombuffer(b"AC", np.uint8), 700)]))
    inst_off = np.concatenate([[0], np.cumsum([t.size for t in texts])]).astype(np.int64)
    joined = torch.from_numpy(np.concatenate(texts)).cuda()
    packed, toff, nr = B().pack_text(ctx, joined)
    sa = torch.empty(int(inst_off[-1]), dtype=torch.int32, device="cuda")
    B().sa_build_batched(ctx, packed, toff, nr, int(inst_off[-1]), inst_off, sa)
    got = sa.cpu().numpy()
    for i, t in enumerate(texts):
        want = oracle.suffix_array(t)
        assert np.array_equal(got[inst_off[i]: inst_off[i + 1]].astype(np.int64), want), i


def test_assemble_batched_equals_oracle_and_alone(ctx):
    texts = small_batch(2, 40)
    got = B().assemble_texts_batched(ctx, texts, 31)
    assert len(got) == len(texts)
    for i, t in enumerate(texts):
        buf, off = oracle.assemble(t, 31)
        assert got[i] == oracle.contigs_as_list(buf, off), i
        if i % 8 == 0:   # alone == in the mix, byte for byte
            assert B().assemble_text(ctx, torch.from_numpy(t).cuda(), 31) == got[i], i


def test_assemble_batched_tiny_genomes(ctx):
    insts = [synth.tiny(s) for s in range(6)]
    got = B().assemble_texts_batched(ctx, [x["text"] for x in insts], 31)
    for x, g in zip(insts, got):
        assert g == [x["genome"].tobytes()]


def test_batched_rejects_bad_offsets(ctx):
    t = np.frombuffer(b"ACGT$ACG$", np.uint8).copy()
    joined = torch.from_numpy(t).cuda()
    contigs = torch.empty(16, dtype=torch.uint8, device="cuda")
    off = torch.empty(8, dtype=torch.int64, device="cuda")
    with pytest.raises(B().DnasaError) as e:   # 3 is not a fragment start
        B().assemble_batched(ctx, joined, [0, 3, 9], 2, contigs, off)
    assert e.value.status == B().INVALID_ARG


def test_autotune_picks_valid_options(ctx, tmp_path):
    texts = small_batch(3, 12)
    inst_off = np.concatenate([[0], np.cumsum([t.size for t in texts])]).astype(np.int64)
    joined = torch.from_numpy(np.concatenate(texts)).cuda()
    packed, toff, nr = B().pack_text(ctx, joined)
    cache = str(tmp_path / "tune.tsv")
    opts, ms = B().dnasa_autotune(ctx, packed, toff, nr, int(inst_off[-1]), inst_off, cache_path=cache)
    assert opts.tile_items in (2048, 3840, 5120) and ms > 0
    again, ms2 = B().dnasa_autotune(ctx, packed, toff, nr, int(inst_off[-1]), inst_off, cache_path=cache)
    assert (again.tile_items, again.finish_threshold) == (opts.tile_items, opts.finish_threshold)
    sa = torch.empty(int(inst_off[-1]), dtype=torch.int32, device="cuda")
    B().sa_build_batched(ctx, packed, toff, nr, int(inst_off[-1]), inst_off, sa, opts)
    got = sa.cpu().numpy()
    for i in (0, 5, 11):
        t = texts[i]
        assert np.array_equal(got[inst_off[i]: inst_off[i + 1]].astype(np.int64), oracle.suffix_array(t))


def test_assemble_batched_c3_512_instances(ctx):
    """512 instances of the batched workload's own generator (genome log-uniform
    2-200 kbp, reads 100-1000 bp at 8x, min overlap 31), one batched call; every
    instance's contigs equal the oracle's.  The oracle runs on host threads (its
    C calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    import os

    texts = [synth.batched_instance(21, i)["text"] for i in range(512)]
    with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        want = list(ex.map(lambda t: oracle.contigs_as_list(*oracle.assemble(t, 31)), texts))
    got = B().assemble_texts_batched(ctx, texts, 31)
    assert len(got) == 512
    bad = [i for i in range(512) if got[i] != want[i]]
    assert not bad, f"{len(bad)} instances differ, first {bad[:5]}"
