"""Overlaps on both strands with substitution errors (Sec. III DEFINITION) on the
GPU against the oracle, through the C ABI: every edge (a, b, L, mismatches) equal."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1404_3456_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

COMP = {ord("A"): ord("T"), ord("C"): ord("G"), ord("G"): ord("C"), ord("T"): ord("A")}


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


def revcomp(x):
    return np.array([COMP[int(c)] for c in x[::-1]], dtype=np.uint8)


def compare(ctx, text, lmin, num, den, rc):
    got, m = B().overlap_search_approx(ctx, torch.from_numpy(text).cuda(), lmin, num, den, rc)
    want = np.stack(oracle.overlaps_approx(text, lmin, num, den, rc), 1) if True else None
    g = got.cpu().numpy()
    nr = int((text == ord("$")).sum())
    assert m == (2 * nr if rc else nr)
    assert g.shape == want.shape, (g.shape, want.shape)
    assert np.array_equal(g, want)
    return g


def noisy_reads(seed, G, n, lo, hi, subs_per_100, both):
    rng = np.random.default_rng(seed)
    g = synth.iid(rng, G)
    reads = []
    for _ in range(n):
        L = int(rng.integers(lo, hi + 1))
        s = int(rng.integers(0, G - L + 1))
        r = g[s: s + L].copy()
        k = rng.binomial(L, subs_per_100 / 100.0)
        for p in rng.choice(L, size=k, replace=False):
            r[p] = synth.BASES[(np.searchsorted(synth.BASES, r[p]) + int(rng.integers(1, 4))) % 4]
        reads.append(revcomp(r) if both and rng.random() < 0.5 else r)
    return synth.join_reads(reads)


@pytest.mark.parametrize("seed", range(4))
def test_two_strands_with_errors(ctx, seed):
    text = noisy_reads(10 + seed, 3000, 120, 150, 300, 1.0, True)
    g = compare(ctx, text, 40, 1, 30, True)
    assert g.shape[0] > 0 and (g[:, 3] > 0).any()


@pytest.mark.parametrize("rc", [False, True])
def test_exact_one_and_two_strands(ctx, rc):
    text = synth.tiny(1)["text"]
    g = compare(ctx, text, 31, 0, 1, rc)
    if not rc:   # the exact one-strand relation is overlap_search's edge set
        j, k, L = oracle.overlaps_brute(text, 31)
        assert np.array_equal(g[:, :3], np.stack([j, k, L], 1))


@pytest.mark.parametrize("seed", range(3))
def test_repeats_and_high_error_rate(ctx, seed):
    rng = np.random.default_rng(70 + seed)
    reads = []
    for _ in range(60):
        n = int(rng.integers(30, 90))
        if rng.random() < 0.4:
            unit = synth.iid(rng, int(rng.integers(1, 4)))
            reads.append(np.tile(unit, n // unit.size + 1)[:n])
        else:
            reads.append(synth.iid(rng, n))
    compare(ctx, synth.join_reads(reads), 12, 1, 8, True)


def test_edges_past_cap_report_capacity(ctx):
    text = noisy_reads(99, 2000, 80, 150, 250, 0.5, False)
    want = oracle.overlaps_approx(text, 40, 1, 30, False)[0].size
    assert want > 4
    edges = torch.empty((2, 4), dtype=torch.int32, device="cuda")
    import ctypes
    n, m = ctypes.c_int64(0), ctypes.c_int64(0)
    t = torch.from_numpy(text).cuda()
    rc = B().lib().overlap_search_approx(ctx.handle, ctypes.c_void_p(t.data_ptr()), t.numel(), 40, 1, 30, 0,
                                         ctypes.c_void_p(edges.data_ptr()), 2, ctypes.byref(n),
                                         ctypes.byref(m), None)
    assert rc == B().CAPACITY and n.value == want


def test_degenerate_and_bad_arguments(ctx):
    """Fragments shorter than the minimum overlap give no edges; mu >= 1, a
    non-positive minimum and host pointers are refused."""
    import ctypes

    t = np.frombuffer(b"ACGTACGT$TTGCA$GGG$", np.uint8).copy()
    g, m = B().overlap_search_approx(ctx, torch.from_numpy(t).cuda(), 40, 1, 10, True)
    assert g.shape[0] == 0 and m == 6
    assert oracle.overlaps_approx(t, 40, 1, 10, True)[0].size == 0
    L = B().lib()
    d = torch.from_numpy(t).cuda()
    edges = torch.empty((16, 4), dtype=torch.int32, device="cuda")
    n, mo = ctypes.c_int64(0), ctypes.c_int64(0)
    for lmin, num, den, both in [(5, 3, 3, 0), (0, 0, 1, 0), (5, -1, 2, 0), (5, 0, 1, 2)]:
        rc = L.overlap_search_approx(ctx.handle, ctypes.c_void_p(d.data_ptr()), d.numel(), lmin, num, den, both,
                                     ctypes.c_void_p(edges.data_ptr()), 16, ctypes.byref(n), ctypes.byref(mo),
                                     None)
        assert rc == B().INVALID_ARG
    rc = L.overlap_search_approx(ctx.handle, ctypes.c_void_p(t.ctypes.data), t.size, 3, 0, 1, 0,
                                 ctypes.c_void_p(edges.data_ptr()), 16, ctypes.byref(n), ctypes.byref(mo), None)
    assert rc == B().INVALID_ARG
    # a single fragment has no partner on either strand
    one = np.frombuffer(b"ACGTTGCAACGT$", np.uint8).copy()
    g1, m1 = B().overlap_search_approx(ctx, torch.from_numpy(one).cuda(), 3, 0, 1, True)
    assert g1.shape[0] == 0 and m1 == 2
