"""The allocation-free sort entry point, for callers that cannot allocate device
memory (a host framework's caching allocator already owns the GPU's memory, or a
latency-bound loop cannot afford cudaMalloc/cudaFree and the synchronization
they imply).  dnasa_sort_pairs_noalloc keeps its scratch in one fixed device
array inside the library; this test checks, through the C ABI, that it returns
exactly what the allocating dnasa_sort_pairs returns, on two calls in a row (a
large one, then a smaller one that must not see the first call's leftovers),
and that sizes above its fixed limit are refused.  Sorting is integer work, so
the outputs must be identical."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _keys(rng, n, bits):
    k = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2)
    k += rng.integers(0, 2, size=n).astype(np.uint64)
    if bits < 64:
        k &= np.uint64((1 << bits) - 1)
    k[: n // 5] = k[0]                      # long runs of equal keys: order must hold
    return k


def test_noalloc_sort_matches_allocating_sort_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3456_gb300 import binding as B

    ctx = B.Context(0)
    try:
        cases = [(B.NOALLOC_MAX_ITEMS, 64, True), (300_001, 41, True)]
        for call, (n, bits, with_vals) in enumerate(cases):
            rng = np.random.default_rng(100 + call)
            keys = _keys(rng, n, bits)
            vals = rng.permutation(n).astype(np.uint32)
            k_ref = torch.from_numpy(keys.view(np.int64).copy()).cuda()
            v_ref = torch.from_numpy(vals.view(np.int32).copy()).cuda()
            B.dnasa_sort_pairs(ctx, k_ref, v_ref, key_bits=bits)
            k_na = torch.from_numpy(keys.view(np.int64).copy()).cuda()
            v_na = torch.from_numpy(vals.view(np.int32).copy()).cuda()
            B.dnasa_sort_pairs_noalloc(k_na, v_na, key_bits=bits)
            torch.cuda.synchronize()
            assert torch.equal(k_na, k_ref), f"keys differ on call {call}"
            assert torch.equal(v_na, v_ref), f"values differ on call {call}"
    finally:
        ctx.close()


def test_noalloc_sort_keys_only_and_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3456_gb300 import binding as B

    ctx = B.Context(0)
    try:
        rng = np.random.default_rng(7)
        keys = _keys(rng, 70_003, 30)
        k_ref = torch.from_numpy(keys.view(np.int64).copy()).cuda()
        B.dnasa_sort_pairs(ctx, k_ref, None, key_bits=30)
        k_na = torch.from_numpy(keys.view(np.int64).copy()).cuda()
        B.dnasa_sort_pairs_noalloc(k_na, None, key_bits=30)
        torch.cuda.synchronize()
        assert torch.equal(k_na, k_ref)
        too_many = torch.zeros(B.NOALLOC_MAX_ITEMS + 1, dtype=torch.int64, device="cuda")
        with pytest.raises(B.DnasaError) as e:
            B.dnasa_sort_pairs_noalloc(too_many, None, key_bits=8)
        assert e.value.status == B.CAPACITY
    finally:
        ctx.close()


def test_noalloc_sort_odd_pass_counts():
    """An odd number of 8-bit digit passes leaves the result in the library's own
    scratch array, from which it is copied back into the caller's buffers; the
    second, smaller call must not see the first call's contents."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3456_gb300 import binding as B

    ctx = B.Context(0)
    try:
        cases = [(500_000, 8, True), (123_457, 20, False), (65_537, 20, True), (4_099, 8, False)]
        for call, (n, bits, with_vals) in enumerate(cases):
            rng = np.random.default_rng(300 + call)
            keys = _keys(rng, n, bits)
            vals = rng.permutation(n).astype(np.uint32) if with_vals else None
            k_ref = torch.from_numpy(keys.view(np.int64).copy()).cuda()
            v_ref = torch.from_numpy(vals.view(np.int32).copy()).cuda() if with_vals else None
            B.dnasa_sort_pairs(ctx, k_ref, v_ref, key_bits=bits)
            k_na = torch.from_numpy(keys.view(np.int64).copy()).cuda()
            v_na = torch.from_numpy(vals.view(np.int32).copy()).cuda() if with_vals else None
            B.dnasa_sort_pairs_noalloc(k_na, v_na, key_bits=bits)
            torch.cuda.synchronize()
            assert torch.equal(k_na, k_ref), f"keys differ on call {call}"
            if with_vals:
                assert torch.equal(v_na, v_ref), f"values differ on call {call}"
    finally:
        ctx.close()


def test_noalloc_sort_refuses_host_pointers():
    """A host buffer handed to the C entry point is refused before any launch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from paper_1404_3456_gb300 import binding as B

    torch.cuda.init()
    host_keys = np.zeros(1024, dtype=np.uint64)
    host_vals = np.zeros(1024, dtype=np.uint32)
    dev_keys = torch.zeros(1024, dtype=torch.int64, device="cuda")
    rc = B.lib().dnasa_sort_pairs_noalloc(ctypes.c_void_p(host_keys.ctypes.data), None, 1024, 8, None)
    assert rc == B.INVALID_ARG
    rc = B.lib().dnasa_sort_pairs_noalloc(ctypes.c_void_p(dev_keys.data_ptr()),
                                          ctypes.c_void_p(host_vals.ctypes.data), 1024, 8, None)
    assert rc == B.INVALID_ARG
    with pytest.raises(ValueError):
        B.dnasa_sort_pairs_noalloc(torch.zeros(16, dtype=torch.int32, device="cuda"))
