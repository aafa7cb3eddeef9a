"""Failure paths, none of which faults or hangs the GPU: a bounded device wait
that runs out, a workspace cap that refuses an allocation, malformed input and
host pointers.  After each the context must keep working."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1404_3456_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def B():
    from paper_1404_3456_gb300 import binding

    return binding


def small_sort_ok(ctx):
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 2**40, size=50_000, dtype=np.uint64)
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    B().dnasa_sort_pairs(ctx, k, None, key_bits=40)
    return np.array_equal(k.cpu().numpy().view(np.uint64), np.sort(keys))


def test_lookback_timeout_is_reported_and_recoverable():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = B().Context(0)
    assert B().dnasa_selftest_timeout(ctx) == B().DEVICE_TIMEOUT
    assert small_sort_ok(ctx)                     # the context still works
    assert B().dnasa_selftest_timeout(ctx) == B().DEVICE_TIMEOUT
    t = synth.tiny(0)["text"]
    sa, *_ = B().suffix_array(ctx, torch.from_numpy(t).cuda())
    assert np.array_equal(sa.cpu().numpy().astype(np.int64), oracle.suffix_array(t))
    ctx.close()


def test_workspace_cap_gives_oom_then_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = B().Context(0, workspace_cap=1 << 20)   # 1 MB: far too small for 400 kbp
    g = synth.genome_text(synth.iid(synth.rng_for(1, 1), 400_000))
    text = torch.from_numpy(g).cuda()
    with pytest.raises(B().DnasaError) as e:
        B().suffix_array(ctx, text)
    assert e.value.status == B().OOM
    ctx.close()
    ctx = B().Context(0)                           # an uncapped context on the same device works
    sa, *_ = B().suffix_array(ctx, text)
    assert sa.shape[0] == g.size
    ctx.close()


def test_host_pointer_rejected():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = B().Context(0)
    host = np.frombuffer(b"ACGT$", np.uint8).copy()
    packed = torch.empty(8, dtype=torch.int64, device="cuda")
    toff = torch.empty(8, dtype=torch.int64, device="cuda")
    n = ctypes.c_int64(0)
    rc = B().lib().dnasa_pack(ctx.handle, host.ctypes.data_as(ctypes.c_void_p), host.size,
                              ctypes.c_void_p(packed.data_ptr()), ctypes.c_void_p(toff.data_ptr()),
                              8, ctypes.byref(n), None)
    assert rc == B().INVALID_ARG
    assert small_sort_ok(ctx)
    ctx.close()


def test_fragment_shorter_than_min_overlap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = B().Context(0)
    reads = [b"ACGTACGTTT", b"TTGCA", b"A", b"GCATTTACGT"]
    t = np.frombuffer(b"$".join(reads) + b"$", np.uint8).copy()
    got = B().assemble_text(ctx, torch.from_numpy(t).cuda(), 8)
    buf, off = oracle.assemble(t, 8)
    assert got == oracle.contigs_as_list(buf, off)
    ctx.close()
