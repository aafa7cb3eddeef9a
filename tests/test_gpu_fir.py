"""Two-cut fir reconstruction (Sec. III, Figs. 2, 5-8) on the GPU against the
oracle, through the C ABI.  Everything is integer work: status, step count,
every fragment offset and every byte of the result must be equal."""
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


def check_one(ctx, text, max_steps=1 << 40):
    st, start, rs, steps = B().fir_reconstruct(ctx, torch.from_numpy(text).cuda(), max_steps)
    ost, ostart, ors, osteps = oracle.fir_reconstruct(text, max_steps)
    assert (st, steps) == (ost, osteps)
    assert np.array_equal(start.cpu().numpy(), ostart)
    assert rs == ors
    return st, rs


@pytest.mark.parametrize("seed", range(6))
def test_two_cut_iid_recovers_genome(ctx, seed):
    d = synth.two_cut(seed, 20_000 + 15_000 * seed, mean_len=400)
    st, rs = check_one(ctx, d["text"])
    assert st == B().FIR_SOLVED and rs == d["genome"].tobytes()


@pytest.mark.parametrize("seed", range(4))
def test_two_cut_with_repeats(ctx, seed):
    """Tandem arrays and copies of an element make fir relations ambiguous: the
    search backs up; whatever it finds (or not) must be the oracle's."""
    d = synth.two_cut(100 + seed, 60_000, mean_len=300, min_gap=40, frac_tandem=0.05,
                      frac_elem=0.05, elem_len=400, elem_subst=0.002)
    check_one(ctx, d["text"], max_steps=200_000)


def test_dead_start_pair_backtracks(ctx):
    rng = np.random.default_rng(3)
    A = np.frombuffer(b"ACGT", np.uint8)
    u, r1, r2 = (A[rng.integers(0, 4, n)] for n in (30, 100, 100))
    S = np.concatenate([u, r1, u, r2])
    pieces = [(130, 200), (0, 130), (0, 30), (30, 175), (175, 260), (200, 260)]
    text = synth.join_reads([S[a:b] for a, b in pieces])
    st, rs = check_one(ctx, text)
    assert st == B().FIR_SOLVED and rs == S.tobytes()
    assert check_one(ctx, text, max_steps=1)[0] == B().FIR_GAVE_UP


@pytest.mark.parametrize("seed", range(30))
def test_tiny_two_letter_sets(ctx, seed):
    rng = np.random.default_rng(5000 + seed)
    frags = [np.frombuffer(b"AC", np.uint8)[rng.integers(0, 2, int(rng.integers(1, 6)))]
             for _ in range(int(rng.integers(1, 8)))]
    check_one(ctx, synth.join_reads(frags))


def test_batched_mix_equals_oracle(ctx):
    texts = [synth.two_cut(200 + i, int(3_000 + 4_000 * (i % 5)), mean_len=250)["text"] for i in range(20)]
    texts.append(np.frombuffer(b"ACGT$CATG$", np.uint8).copy())       # no fir pair at all
    texts.append(synth.two_cut(300, 40_000, mean_len=200, min_gap=30, frac_tandem=0.1)["text"])
    texts.append(np.frombuffer(b"A$", np.uint8).copy())               # one fragment
    got = B().fir_reconstruct_batched(ctx, texts, max_steps=50_000)
    for i, t in enumerate(texts):
        ost, ostart, ors, osteps = oracle.fir_reconstruct(t, 50_000)
        st, start, rs, steps = got[i]
        assert (st, steps) == (ost, osteps), i
        assert np.array_equal(start, ostart), i
        assert rs == ors, i


def test_capacity_and_argument_errors(ctx):
    """Undersized outputs report DNASA_CAPACITY with the size needed; bad
    arguments and host pointers are refused before any launch."""
    import ctypes

    d = synth.two_cut(77, 6_000, mean_len=300)
    text = torch.from_numpy(d["text"]).cuda()
    nf = int((d["text"] == ord("$")).sum())
    start = torch.empty(nf, dtype=torch.int64, device="cuda")
    rs = torch.empty(10, dtype=torch.uint8, device="cuda")          # far too small
    rl, st, steps = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int64(0)
    L = B().lib()
    rc = L.fir_reconstruct(ctx.handle, ctypes.c_void_p(text.data_ptr()), text.numel(), 1 << 30,
                           ctypes.c_void_p(start.data_ptr()), nf, ctypes.c_void_p(rs.data_ptr()), rs.numel(),
                           ctypes.byref(rl), ctypes.byref(st), ctypes.byref(steps), None)
    assert rc == B().CAPACITY and rl.value == d["genome"].size
    rc = L.fir_reconstruct(ctx.handle, ctypes.c_void_p(text.data_ptr()), text.numel(), 1 << 30,
                           ctypes.c_void_p(start.data_ptr()), nf - 1, ctypes.c_void_p(rs.data_ptr()),
                           rs.numel(), ctypes.byref(rl), ctypes.byref(st), ctypes.byref(steps), None)
    assert rc == B().CAPACITY
    host = np.zeros(nf, dtype=np.int64)
    rc = L.fir_reconstruct(ctx.handle, ctypes.c_void_p(text.data_ptr()), text.numel(), 1 << 30,
                           ctypes.c_void_p(host.ctypes.data), nf, ctypes.c_void_p(rs.data_ptr()), rs.numel(),
                           ctypes.byref(rl), ctypes.byref(st), ctypes.byref(steps), None)
    assert rc == B().INVALID_ARG
    rc = L.fir_reconstruct(ctx.handle, ctypes.c_void_p(text.data_ptr()), text.numel(), 0,
                           ctypes.c_void_p(start.data_ptr()), nf, ctypes.c_void_p(rs.data_ptr()), rs.numel(),
                           ctypes.byref(rl), ctypes.byref(st), ctypes.byref(steps), None)
    assert rc == B().INVALID_ARG
    # the context still works afterwards
    st2, rs2 = check_one(ctx, d["text"])
    assert st2 == B().FIR_SOLVED and rs2 == d["genome"].tobytes()
