"""The greedy layout on fragment sets above 4,096 fragments per instance.

Up to 4,096 fragments an instance's successor, predecessor and union-find
arrays live in shared memory; above that the layout kernel keeps them in global
memory.  These tests reach that second branch (the size of the served jobs) and
compare every contig byte for byte with the oracle's assembly (Sec. III, Fig. 3:
the path through the overlap graph spelled as a superstring)."""
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


def reads_text(seed, G, coverage=10.0, read_len=150, tandem=0.02):
    rng = synth.rng_for(seed, 9)
    g = synth.genome_with_repeats(rng, G, tandem, (2, 50), (10, 200))
    text, starts = synth.shotgun_fixed_text(rng, g, coverage, read_len)
    return text, starts.size


def oracle_contigs(text, lmin):
    buf, off = oracle.assemble(text, lmin)
    return oracle.contigs_as_list(buf, off)


@pytest.mark.parametrize("seed,G", [(1, 100_000), (2, 150_000)])
def test_assemble_above_shared_memory_layout(ctx, seed, G):
    text, n_reads = reads_text(seed, G)
    assert n_reads > 4096
    got = B().assemble_text(ctx, torch.from_numpy(text).cuda(), 41)
    assert got == oracle_contigs(text, 41)


def test_assemble_served_job_300kbp(ctx):
    """One job of the served workload's generator at >= 300 kbp (about 20,000
    fragments of 150 bp at 10x, 2 % tandem arrays), min overlap 41."""
    j = synth.served_job(3, 0, g_lo=300_000, g_hi=320_000)
    assert j["text"].size // 151 > 4096
    got = B().assemble_text(ctx, torch.from_numpy(j["text"]).cuda(), j["min_overlap"])
    assert got == oracle_contigs(j["text"], j["min_overlap"])


def test_assemble_batched_mixed_sizes_above_4096(ctx):
    """Instances on both sides of 4,096 fragments in one batched call: each
    equals the oracle, and the large ones equal their alone runs."""
    texts = [reads_text(10, 80_000)[0], synth.batched_instance(7, 0)["text"],
             reads_text(11, 120_000)[0], synth.batched_instance(7, 1)["text"]]
    got = B().assemble_texts_batched(ctx, texts, 41)
    for i, t in enumerate(texts):
        assert got[i] == oracle_contigs(t, 41), i
    assert got[2] == B().assemble_text(ctx, torch.from_numpy(texts[2]).cuda(), 41)
