"""Thin Python binding of libdnasa.so (the C ABI in include/dnasa.h).

Argument marshalling only: every function here passes torch tensors'
``data_ptr()`` and the current CUDA stream to the C entry point of the same
name and raises :class:`DnasaError` on a non-zero status.  Every step of the
path runs in the library's CUDA kernels; there is no CPU fallback, and a
missing library is an ImportError-like failure on first use, not a silent
substitute.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdnasa.so")

OK, INVALID_ARG, BAD_ALPHABET, OOM, CAPACITY, DEVICE_TIMEOUT, CUDA_ERROR = 0, -1, -2, -3, -4, -5, -6
I32, I64 = 4, 8
_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "BAD_ALPHABET", -3: "OOM", -4: "CAPACITY",
          -5: "DEVICE_TIMEOUT", -6: "CUDA_ERROR"}


class DnasaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("reserved0", ctypes.c_int32), ("tile_items", ctypes.c_int32),
                ("finish_threshold", ctypes.c_int64), ("max_rounds", ctypes.c_int32),
                ("lookback", ctypes.c_int32), ("seg_max", ctypes.c_int32),
                ("pack_position", ctypes.c_int32), ("builder", ctypes.c_int32),
                ("rounds_on_host", ctypes.c_int32)]


class Trace(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("finished_direct", ctypes.c_int32),
                ("h0", ctypes.c_int32), ("pack_bits", ctypes.c_int32),
                ("active", ctypes.c_int64 * 64), ("graph_rounds", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ProfEntry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("launches", ctypes.c_int32), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


PROF_KINDS = ["onesweep", "hist", "rerank", "gather", "init_keys", "finish", "lcp", "overlap",
              "layout", "pack", "other", "segsort", "apply"]

class Job(ctypes.Structure):
    _fields_ = [("text", ctypes.c_void_p), ("N", ctypes.c_int64), ("min_overlap", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_contigs", ctypes.c_int64), ("bytes", ctypes.c_int64),
                ("contigs", ctypes.POINTER(ctypes.c_uint8)), ("contig_off", ctypes.POINTER(ctypes.c_int64)),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_P, _I64, _I32, _INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
_SIGS = {
    "dnasa_create": (_INT, [_INT, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "dnasa_destroy": (None, [_P]),
    "dnasa_last_error": (ctypes.c_char_p, [_P]),
    "dnasa_sync_status": (_INT, [_P, _P]),
    "dnasa_get_trace": (_INT, [_P, ctypes.POINTER(Trace)]),
    "dnasa_packed_words": (_I64, [_I64]),
    "dnasa_profile": (_INT, [_P, _INT]),
    "dnasa_profile_read": (_INT, [_P, ctypes.POINTER(ProfEntry), _INT, ctypes.POINTER(_INT)]),
    "dnasa_launch_count": (ctypes.c_uint64, [_P]),
    "dnasa_sort_pairs": (_INT, [_P, _P, _P, _I64, _INT, _INT, _INT, _P]),
    "dnasa_selftest_timeout": (_INT, [_P, _P]),
    "dnasa_sort_pairs_noalloc": (_INT, [_P, _P, _I64, _INT, _P]),
    "dnasa_pack": (_INT, [_P, _P, _I64, _P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "sa_build": (_INT, [_P, _P, _P, _I64, _I64, _P, _INT, ctypes.POINTER(Opts), _P]),
    "lcp_build": (_INT, [_P, _P, _P, _I64, _I64, _P, _INT, _P, _P]),
    "sa_lcp_build": (_INT, [_P, _P, _P, _I64, _I64, _P, _INT, _P, ctypes.POINTER(Opts), _P]),
    "overlap_search": (_INT, [_P, _P, _P, _I64, _I64, _P, _P, _INT, _I32, _P, _I64,
                              ctypes.POINTER(_I64), _P, _P]),
    "assemble": (_INT, [_P, _P, _I64, _I32, _P, _I64, _P, _I64, ctypes.POINTER(_I64),
                        ctypes.POINTER(_I64), _P]),
    "dnasa_autotune": (_INT, [_P, _P, _P, _I64, _I64, _P, _I32, ctypes.c_char_p, ctypes.POINTER(Opts),
                              ctypes.POINTER(ctypes.c_double), _P]),
    "dnasa_server_create": (_INT, [_INT, ctypes.c_size_t, _I32, _I32, ctypes.POINTER(_P)]),
    "dnasa_server_submit": (_INT, [_P, ctypes.POINTER(Job), ctypes.c_uint64]),
    "dnasa_server_poll": (_INT, [_P, ctypes.POINTER(Result), _I32, _I32, ctypes.POINTER(_I32)]),
    "dnasa_server_pending": (_INT, [_P]),
    "dnasa_server_job_bytes": (_I64, [_I64, _I64]),
    "dnasa_server_destroy": (None, [_P]),
    "overlap_search_approx": (_INT, [_P, _P, _I64, _I32, _I32, _I32, _I32, _P, _I64,
                                     ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P]),
    "fir_reconstruct": (_INT, [_P, _P, _I64, _I64, _P, _I64, _P, _I64, ctypes.POINTER(_I64),
                               ctypes.POINTER(_I32), ctypes.POINTER(_I64), _P]),
    "fir_reconstruct_batched": (_INT, [_P, _P, _P, _I32, _I64, _P, _I64, _P, _I64, _P, _P, _P,
                                       ctypes.POINTER(_I64), _P]),
    "sa_build_batched": (_INT, [_P, _P, _P, _I64, _I64, _P, _I32, _P, ctypes.POINTER(Opts), _P]),
    "assemble_batched": (_INT, [_P, _P, _P, _I32, _I32, ctypes.POINTER(Opts), _P, _I64, _P, _I64,
                                _P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P]),
}


def lib():
    """The loaded library; raises if libdnasa.so has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name, None)
                if f is None:
                    continue
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device (no CPU fallback)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """Owns a dnasa_ctx (its device workspace) on one CUDA device."""

    def __init__(self, device: int = 0, workspace_cap: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        torch.cuda.init()
        rc = lib().dnasa_create(device, workspace_cap, ctypes.byref(h))
        if rc != 0:
            raise DnasaError(rc, "dnasa_create failed")
        self.handle = h

    def check(self, rc: int):
        if rc != 0:
            raise DnasaError(rc, lib().dnasa_last_error(self.handle).decode())

    def trace(self) -> dict:
        tr = Trace()
        self.check(lib().dnasa_get_trace(self.handle, ctypes.byref(tr)))
        return dict(rounds=tr.rounds, finished_direct=tr.finished_direct, h0=tr.h0,
                    pack_bits=tr.pack_bits, active=list(tr.active[: tr.rounds + 1]),
                    graph_rounds=tr.graph_rounds)

    def profile(self, enable: bool = True):
        """Start (or stop) recording CUDA events around every kernel launch."""
        self.check(lib().dnasa_profile(self.handle, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel class: dict(launches, ms, bytes)} since profile(True); clears."""
        arr = (ProfEntry * len(PROF_KINDS))()
        n = ctypes.c_int(0)
        self.check(lib().dnasa_profile_read(self.handle, arr, len(PROF_KINDS), ctypes.byref(n)))
        return {PROF_KINDS[e.kind]: dict(launches=e.launches, ms=e.ms, bytes=e.bytes)
                for e in arr[: n.value]}

    def launch_count(self) -> int:
        return int(lib().dnasa_launch_count(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().dnasa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_opts(reserved0=0, tile_items=0, finish_threshold=0, max_rounds=0, lookback=0, seg_max=0,
              pack_position=0, builder=0, rounds_on_host=0):
    return Opts(reserved0, tile_items, finish_threshold, max_rounds, lookback, seg_max,
                pack_position, builder, rounds_on_host)


# ---------------------------------------------------------------- entry points


def packed_words(N: int) -> int:
    return int(lib().dnasa_packed_words(N))


def _check_sort_args(keys, vals):
    """The C side reads 8 bytes per key and 4 per value over keys.numel() items."""
    if keys.dtype != torch.int64 or not keys.is_contiguous() or keys.device.type != "cuda":
        raise ValueError("keys must be a contiguous int64 CUDA tensor")
    if vals is not None:
        if vals.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)) \
                or not vals.is_contiguous() or vals.device != keys.device:
            raise ValueError("vals must be a contiguous int32 tensor on the keys' device")
        if vals.numel() != keys.numel():
            raise ValueError("vals must have as many items as keys")


def dnasa_sort_pairs(ctx: Context, keys, vals=None, key_bits: int = 64, tile_items: int = 0,
                     lookback: int = 0, stream=None):
    """Stable radix sort in place: keys int64 (bit pattern of uint64), vals int32/uint32."""
    _check_sort_args(keys, vals)
    ctx.check(lib().dnasa_sort_pairs(ctx.handle, _ptr(keys), _ptr(vals) if vals is not None else None,
                                     keys.numel(), key_bits, tile_items, lookback, _stream(stream)))


def dnasa_selftest_timeout(ctx: Context, stream=None) -> int:
    """Returns the status of the bounded-wait self-test (DEVICE_TIMEOUT expected)."""
    return int(lib().dnasa_selftest_timeout(ctx.handle, _stream(stream)))


NOALLOC_MAX_ITEMS = 1 << 20   # DNASA_NOALLOC_MAX_ITEMS in dnasa.h


def dnasa_sort_pairs_noalloc(keys, vals=None, key_bits: int = 64, stream=None):
    """dnasa_sort_pairs without a context or any allocation (n <= NOALLOC_MAX_ITEMS);
    raises DnasaError with the C status on failure."""
    _check_sort_args(keys, vals)
    with torch.cuda.device(keys.device):   # the C side sorts on the current device
        rc = lib().dnasa_sort_pairs_noalloc(_ptr(keys), _ptr(vals) if vals is not None else None,
                                            keys.numel(), key_bits, _stream(stream))
    if rc != 0:
        raise DnasaError(rc, "dnasa_sort_pairs_noalloc failed")


def dnasa_pack(ctx: Context, text, packed, toff, stream=None) -> int:
    n = ctypes.c_int64(0)
    ctx.check(lib().dnasa_pack(ctx.handle, _ptr(text), text.numel(), _ptr(packed), _ptr(toff),
                               toff.numel(), ctypes.byref(n), _stream(stream)))
    return n.value


def sa_build(ctx: Context, packed, toff, n_reads: int, N: int, sa, opts: Opts | None = None,
             stream=None):
    width = I64 if sa.dtype == torch.int64 else I32
    ctx.check(lib().sa_build(ctx.handle, _ptr(packed), _ptr(toff), n_reads, N, _ptr(sa), width,
                             ctypes.byref(opts) if opts is not None else None, _stream(stream)))


def lcp_build(ctx: Context, packed, toff, n_reads: int, N: int, sa, lcp, stream=None):
    width = I64 if sa.dtype == torch.int64 else I32
    ctx.check(lib().lcp_build(ctx.handle, _ptr(packed), _ptr(toff), n_reads, N, _ptr(sa), width,
                              _ptr(lcp), _stream(stream)))


def sa_lcp_build(ctx: Context, packed, toff, n_reads: int, N: int, sa, lcp, opts: Opts | None = None,
                 stream=None):
    """Suffix array and LCP in one call (sa_build + lcp_build results)."""
    width = I64 if sa.dtype == torch.int64 else I32
    ctx.check(lib().sa_lcp_build(ctx.handle, _ptr(packed), _ptr(toff), n_reads, N, _ptr(sa), width,
                                 _ptr(lcp), ctypes.byref(opts) if opts is not None else None,
                                 _stream(stream)))


def overlap_search(ctx: Context, packed, toff, n_reads: int, N: int, sa, lcp, min_overlap: int,
                   edges, contained, stream=None, count_only_past_cap: bool = False) -> int:
    """edges: int32 tensor (cap, 3) of (j, k, L).  Returns the edge count.  With
    count_only_past_cap, an edge set larger than the buffer is not an error: the
    first `cap` edges are written and the full count is returned."""
    width = I64 if sa.dtype == torch.int64 else I32
    n = ctypes.c_int64(0)
    cap = edges.shape[0] if edges is not None else 0
    rc = lib().overlap_search(ctx.handle, _ptr(packed), _ptr(toff), n_reads, N, _ptr(sa),
                              _ptr(lcp), width, min_overlap,
                              _ptr(edges) if cap else None, cap, ctypes.byref(n),
                              _ptr(contained), _stream(stream))
    if not (count_only_past_cap and rc == CAPACITY):
        ctx.check(rc)
    return n.value


def assemble(ctx: Context, text, min_overlap: int, contigs, contig_off, stream=None):
    """Returns (n_contigs, bytes)."""
    nc = ctypes.c_int64(0)
    need = ctypes.c_int64(0)
    ctx.check(lib().assemble(ctx.handle, _ptr(text), text.numel(), min_overlap, _ptr(contigs),
                             contigs.numel(), _ptr(contig_off), contig_off.numel(),
                             ctypes.byref(nc), ctypes.byref(need), _stream(stream)))
    return nc.value, need.value


# ---------------------------------------------------------------- conveniences
# (allocate outputs with torch, then call the entry points above)


def pack_text(ctx: Context, text: torch.Tensor, stream=None):
    """text (cuda uint8) -> (packed uint64-as-int64, toff int64, n_reads)."""
    N = text.numel()
    dev = text.device
    packed = torch.empty(packed_words(N), dtype=torch.int64, device=dev)
    toff = torch.empty(N // 2 + 2, dtype=torch.int64, device=dev)
    nr = dnasa_pack(ctx, text, packed, toff, stream)
    return packed, toff[: nr + 1], nr


def suffix_array(ctx: Context, text: torch.Tensor, dtype=torch.int32, opts=None, stream=None):
    packed, toff, nr = pack_text(ctx, text, stream)
    sa = torch.empty(text.numel(), dtype=dtype, device=text.device)
    sa_build(ctx, packed, toff, nr, text.numel(), sa, opts, stream)
    return sa, packed, toff, nr


def assemble_text(ctx: Context, text: torch.Tensor, min_overlap: int, stream=None):
    """Contigs of one fragment text as a list of bytes."""
    N = text.numel()
    cap = N
    contigs = torch.empty(max(cap, 1), dtype=torch.uint8, device=text.device)
    off = torch.empty(N // 2 + 2, dtype=torch.int64, device=text.device)
    nc, nb = assemble(ctx, text, min_overlap, contigs, off, stream)
    buf = contigs[:nb].cpu().numpy().tobytes()
    o = off[: nc + 1].cpu().tolist()
    return [buf[o[i]: o[i + 1]] for i in range(nc)]


def _host_i64(offsets):
    import numpy as np

    a = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def sa_build_batched(ctx: Context, packed, toff, n_reads: int, N: int, inst_off, sa,
                     opts: Opts | None = None, stream=None):
    """Per-instance suffix arrays (local coordinates) of concatenated instance texts."""
    arr, p = _host_i64(inst_off)
    ctx.check(lib().sa_build_batched(ctx.handle, _ptr(packed), _ptr(toff), n_reads, N, p,
                                     arr.size - 1, _ptr(sa),
                                     ctypes.byref(opts) if opts is not None else None,
                                     _stream(stream)))


def assemble_batched(ctx: Context, texts, inst_off, min_overlap: int, contigs, contig_off,
                     inst_contig_off=None, opts: Opts | None = None, stream=None):
    """Returns (n_contigs, bytes)."""
    arr, p = _host_i64(inst_off)
    nc = ctypes.c_int64(0)
    need = ctypes.c_int64(0)
    ctx.check(lib().assemble_batched(ctx.handle, _ptr(texts), p, arr.size - 1, min_overlap,
                                     ctypes.byref(opts) if opts is not None else None,
                                     _ptr(contigs), contigs.numel(), _ptr(contig_off),
                                     contig_off.numel(),
                                     _ptr(inst_contig_off) if inst_contig_off is not None else None,
                                     ctypes.byref(nc), ctypes.byref(need), _stream(stream)))
    return nc.value, need.value


def assemble_texts_batched(ctx: Context, texts_np, min_overlap: int, opts=None, stream=None):
    """Contigs of several fragment texts (numpy uint8 arrays), assembled in one
    batched call; returns one list of contig bytes per instance."""
    import numpy as np

    sizes = [int(t.size) for t in texts_np]
    inst_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    joined = torch.from_numpy(np.concatenate(texts_np)).cuda()
    N = int(inst_off[-1])
    contigs = torch.empty(max(N, 1), dtype=torch.uint8, device="cuda")
    off = torch.empty(N // 2 + 2, dtype=torch.int64, device="cuda")
    ioff = torch.empty(len(texts_np) + 1, dtype=torch.int64, device="cuda")
    nc, nb = assemble_batched(ctx, joined, inst_off, min_overlap, contigs, off, ioff, opts, stream)
    buf = contigs[:nb].cpu().numpy().tobytes()
    o = off[: nc + 1].cpu().tolist()
    io = ioff.cpu().tolist()
    return [[buf[o[c]: o[c + 1]] for c in range(io[i], io[i + 1])] for i in range(len(texts_np))]


def overlap_search_approx(ctx: Context, text: torch.Tensor, min_overlap: int, mu_num: int = 0,
                          mu_den: int = 1, both_strands: bool = False, cap: int = 0, stream=None):
    """Overlaps between oriented fragments with at most floor(L * mu) substitutions.
    Returns (edges int32 tensor (n, 4) of (a, b, L, mismatches), n_oriented)."""
    n = ctypes.c_int64(0)
    m = ctypes.c_int64(0)
    cap = cap or max(1024, 8 * int((text == ord("$")).sum().item()) * (2 if both_strands else 1))
    for _ in range(2):
        edges = torch.empty((cap, 4), dtype=torch.int32, device=text.device)
        rc = lib().overlap_search_approx(ctx.handle, _ptr(text), text.numel(), min_overlap, mu_num, mu_den,
                                         int(both_strands), _ptr(edges), cap, ctypes.byref(n),
                                         ctypes.byref(m), _stream(stream))
        if rc == CAPACITY and n.value > cap:
            cap = n.value
            continue
        ctx.check(rc)
        break
    return edges[: n.value], int(m.value)


FIR_SOLVED, FIR_NONE, FIR_GAVE_UP = 0, 1, 2   # DNASA_FIR_* in dnasa.h


def fir_reconstruct(ctx: Context, text: torch.Tensor, max_steps: int = 1 << 40, stream=None):
    """Two-cut reconstruction of one fragment text (device uint8).  Returns
    (status, frag_start int64 tensor, result bytes, steps)."""
    N = text.numel()
    nf = int((text == ord("$")).sum().item())
    start = torch.empty(max(nf, 1), dtype=torch.int64, device=text.device)
    rs = torch.empty(max(N, 1), dtype=torch.uint8, device=text.device)
    rl, st, steps = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int64(0)
    ctx.check(lib().fir_reconstruct(ctx.handle, _ptr(text), N, max_steps, _ptr(start), start.numel(),
                                    _ptr(rs), rs.numel(), ctypes.byref(rl), ctypes.byref(st),
                                    ctypes.byref(steps), _stream(stream)))
    return int(st.value), start[:nf], rs[: rl.value].cpu().numpy().tobytes(), int(steps.value)


def fir_reconstruct_batched_into(ctx: Context, joined, inst_off, max_steps, start, rs, rs_off,
                                 status, steps, stream=None) -> int:
    """fir_reconstruct_batched into caller buffers (device tensors); returns the
    result bytes of all instances."""
    total = ctypes.c_int64(0)
    arr, p = _host_i64(inst_off)
    ctx.check(lib().fir_reconstruct_batched(ctx.handle, _ptr(joined), p, arr.size - 1, max_steps,
                                            _ptr(start), start.numel(), _ptr(rs), rs.numel(),
                                            _ptr(rs_off), _ptr(status), _ptr(steps),
                                            ctypes.byref(total), _stream(stream)))
    return int(total.value)


def fir_reconstruct_batched(ctx: Context, texts_np, max_steps: int = 1 << 40, stream=None):
    """Two-cut reconstruction of several fragment texts (numpy uint8) in one call.
    Returns one (status, frag_start numpy int64, result bytes, steps) per text."""
    import numpy as np

    sizes = [int(t.size) for t in texts_np]
    inst_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    joined_np = np.concatenate(texts_np)
    nf = int((joined_np == ord("$")).sum())
    joined = torch.from_numpy(joined_np).cuda()
    n = len(texts_np)
    N = int(inst_off[-1])
    start = torch.empty(max(nf, 1), dtype=torch.int64, device="cuda")
    rs = torch.empty(max(N, 1), dtype=torch.uint8, device="cuda")
    rs_off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    steps = torch.empty(n, dtype=torch.int64, device="cuda")
    total = ctypes.c_int64(0)
    arr, p = _host_i64(inst_off)
    ctx.check(lib().fir_reconstruct_batched(ctx.handle, _ptr(joined), p, n, max_steps, _ptr(start),
                                            start.numel(), _ptr(rs), rs.numel(), _ptr(rs_off),
                                            _ptr(status), _ptr(steps), ctypes.byref(total),
                                            _stream(stream)))
    st, so, sp = status.cpu().numpy(), rs_off.cpu().numpy(), steps.cpu().numpy()
    buf = rs[: total.value].cpu().numpy().tobytes()
    fs = start[:nf].cpu().numpy()
    foff = np.concatenate([[0], np.cumsum([int((t == ord("$")).sum()) for t in texts_np])])
    return [(int(st[i]), fs[foff[i]: foff[i + 1]], buf[so[i]: so[i + 1]], int(sp[i])) for i in range(n)]


class Server:
    """Continuous-batching assembly server (dnasa_server_* in the C ABI)."""

    @staticmethod
    def job_bytes(N: int, n_reads: int) -> int:
        """Device bytes the server reserves for one job (dnasa_server_job_bytes)."""
        return int(lib().dnasa_server_job_bytes(N, n_reads))

    def __init__(self, device: int = 0, hbm_budget: int = 0, slots: int = 2, max_batch: int = 64):
        torch.cuda.init()
        h = ctypes.c_void_p()
        rc = lib().dnasa_server_create(device, hbm_budget, slots, max_batch, ctypes.byref(h))
        if rc != 0:
            raise DnasaError(rc, "dnasa_server_create failed")
        self.handle = h

    def submit(self, text, min_overlap: int, job_id: int):
        """text: numpy uint8 array (host); copied by the server."""
        import numpy as np

        t = np.ascontiguousarray(text, dtype=np.uint8)
        job = Job(t.ctypes.data_as(ctypes.c_void_p), t.size, min_overlap, 0)
        rc = lib().dnasa_server_submit(self.handle, ctypes.byref(job), job_id)
        if rc != 0:
            raise DnasaError(rc, "dnasa_server_submit failed")

    def poll(self, max_results: int = 256, wait_ms: int = 0):
        """Finished jobs: list of dicts (id, status, contigs [bytes...], times in ms)."""
        arr = (Result * max(max_results, 1))()
        n = ctypes.c_int32(0)
        rc = lib().dnasa_server_poll(self.handle, arr, max_results, wait_ms, ctypes.byref(n))
        if rc != 0:
            raise DnasaError(rc, "dnasa_server_poll failed")
        out = []
        for r in arr[: n.value]:
            buf = ctypes.string_at(r.contigs, r.bytes) if r.bytes else b""
            offs = [r.contig_off[i] for i in range(r.n_contigs + 1)] if r.n_contigs else [0]
            out.append(dict(id=r.id, status=r.status,
                            contigs=[buf[offs[i]: offs[i + 1]] for i in range(r.n_contigs)],
                            t_submit_ms=r.t_submit_ms, t_start_ms=r.t_start_ms, t_done_ms=r.t_done_ms))
        return out

    def pending(self) -> int:
        return int(lib().dnasa_server_pending(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().dnasa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dnasa_autotune(ctx: Context, packed, toff, n_reads: int, N: int, inst_off=None,
                   cache_path: str | None = None, stream=None):
    """Fastest build options for this text (and instance split); returns (Opts, ms)."""
    best = Opts()
    ms = ctypes.c_double(0.0)
    if inst_off is None:
        arr, p, n_inst = None, None, 1
    else:
        arr, p = _host_i64(inst_off)
        n_inst = arr.size - 1
    ctx.check(lib().dnasa_autotune(ctx.handle, _ptr(packed), _ptr(toff), n_reads, N, p, n_inst,
                                   cache_path.encode() if cache_path else None, ctypes.byref(best),
                                   ctypes.byref(ms), _stream(stream)))
    return best, ms.value

