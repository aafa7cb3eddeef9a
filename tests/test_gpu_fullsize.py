"""Parity at the full benchmark sizes.

* sa64m (the bench workload, 64,000,001 suffixes, same seed and options the
  bench uses): the whole SA through the oracle's linear-time suffix-array checker
  and the whole LCP against the oracle's Kasai LCP.
* large (1.5 Gbp, int64 SA): the whole SA through the same checker and the
  whole LCP against Kasai's, both split into ranges on the host's cores (the
  oracle's range functions, pinned against the whole-array ones on the CPU).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1404_3456_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def B():
    from paper_1404_3456_gb300 import binding

    return binding


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B().Context(0)
    yield c
    c.close()


def build(ctx, text_np, dtype):
    text = torch.from_numpy(text_np).cuda()
    packed, toff, nr = B().pack_text(ctx, text)
    del text
    N = text_np.size
    sa = torch.empty(N, dtype=dtype, device="cuda")
    B().sa_build(ctx, packed, toff, nr, N, sa)
    lcp = torch.empty(N, dtype=torch.int32, device="cuda")
    B().lcp_build(ctx, packed, toff, nr, N, sa, lcp)
    torch.cuda.synchronize()
    return sa, lcp


def test_sa64m_full(ctx):
    text = synth.genome_text(synth.sa64m_genome(1))
    sa, lcp = build(ctx, text, torch.int32)
    sa64 = sa.cpu().numpy().astype(np.int64)
    assert oracle.sa_check(text, sa64) == 0
    assert np.array_equal(lcp.cpu().numpy(), oracle.lcp_kasai(text, sa64))


def _mem_available_bytes() -> int:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def test_large_int64_full(ctx):
    """1.5 Gbp genome, int64 SA and int32 LCP, checked in full: the linear
    suffix-array checker over every adjacent pair and Kasai's LCP over every
    entry (the oracle's, split into ranges on the host's cores).  Host memory:
    text 1.5 GB, SA 12 GB, inverse SA 12 GB, two LCP arrays 12 GB."""
    text = synth.genome_text(synth.large_genome(1))
    N = text.size
    sa, lcp = build(ctx, text, torch.int64)
    seen = torch.zeros(N, dtype=torch.bool, device="cuda")
    seen[sa] = True
    assert bool(seen.all()) and int(sa.min()) == 0 and int(sa.max()) == N - 1
    del seen
    need = N * (1 + 8 + 8 + 4 + 4) + (4 << 30)
    if _mem_available_bytes() >= need:
        sa_h = sa.cpu().numpy()
        lcp_h = lcp.cpu().numpy()
        del sa, lcp
        code, want = oracle.sa_check_and_lcp_threaded(text, sa_h)
        assert code == 0, f"suffix-array checker failed at pair {code - 2}"
        bad = np.flatnonzero(lcp_h != want)
        assert bad.size == 0, f"{bad.size} LCP entries differ, first at {bad[:5]}"
    else:
        # not enough host memory for the whole arrays: 200,000 sampled pairs
        # plus both ends, each checked by direct comparison against the text
        rng = np.random.default_rng(2)
        js = np.concatenate([np.arange(1, 1001), np.arange(N - 1000, N),
                             rng.integers(1, N, size=200_000)]).astype(np.int64)
        jt = torch.from_numpy(js).cuda()
        pairs = torch.stack([sa[jt - 1], sa[jt]], 1).reshape(-1).cpu().numpy()
        lp = torch.stack([torch.zeros_like(jt, dtype=torch.int32), lcp[jt]], 1).reshape(-1).cpu().numpy()
        idx = np.arange(1, pairs.size, 2, dtype=np.int64)
        assert oracle.check_pairs(text, pairs, lp, idx) == 0
        pytest.xfail(f"host memory {_mem_available_bytes() >> 30} GB < {need >> 30} GB: "
                     "sampled check only")
