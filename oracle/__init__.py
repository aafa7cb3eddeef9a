"""The oracle: a plain CPU statement of what the GPU path computes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1404_3456_gb300``) never imports it, and it imports nothing from the
product path: the two share no code.  The arithmetic lives in the plain C file
``dnasa_oracle.c`` (single-threaded, slow, direct); this module only marshals
numpy arrays into it and composes its functions.

Every function follows one passage of the paper (arxiv 1404.3456):

* :func:`suffix_array`     -- Sec. IV, the suffix array "Pos": all suffixes of the
  fragment text sorted, by direct comparison.
* :func:`lcp_kasai`, :func:`lcp_direct` -- longest common prefix of SA neighbours
  (needed by the prefix/containment queries of Sec. III-IV).
* :func:`sa_check`         -- Burkhardt & Kaerkkaeinen linear suffix-array checker.
* :func:`split_sort`       -- Algorithm 1 (Sec. V): LSD radix sort by 1-bit splits.
* :func:`overlaps_brute`, :func:`overlaps_sorted` -- Sec. III "fir" prefix relation,
  as suffix-prefix overlaps between fragments; the second by binary search over
  sorted fragments as Sec. IV describes.
* :func:`contained`        -- Sec. III, fragments lying inside another fragment.
* :func:`layout`, :func:`assemble` -- Sec. III, Fig. 3 (path -> superstring) and the
  RS concatenation: greedy unique-overlap layout and spelling.
* :func:`overlaps_approx` -- Sec. III DEFINITION: overlaps of fragments read on
  either strand (reverse complements) with at most a rate mu of substitutions.
* :func:`fir_reconstruct` -- Sec. III, Figs. 2 and 5-8: a sequence cut by two
  shotguns rebuilt from "fir" (prefix) relations by depth-first search with
  back-tracking.

Readings of the paper that these functions fix (the paper is silent on them):
every fragment ends with its own '$' sentinel, smaller than A < C < G < T, and
sentinels compare by position; an LCP never counts a '$'; overlaps are proper
(L < both lengths) with the maximum L kept per ordered pair; of two identical
fragments the larger index is the contained one; the layout is greedy by
(L desc, j asc, k asc) with union-find against cycles.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dnasa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SEP = ord("$")


def build(force: bool = False) -> str:
    """Compile ``dnasa_oracle.c`` into ``liboracle.so`` (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I32 = ctypes.c_int32
            lib.oracle_suffix_array.argtypes = [P, I64, P]
            lib.oracle_suffix_array.restype = ctypes.c_int
            lib.oracle_lcp_kasai.argtypes = [P, I64, P, P]
            lib.oracle_lcp_kasai.restype = ctypes.c_int
            lib.oracle_lcp_direct.argtypes = [P, I64, P, P]
            lib.oracle_lcp_direct.restype = ctypes.c_int
            lib.oracle_sa_check.argtypes = [P, I64, P]
            lib.oracle_sa_check.restype = I64
            lib.oracle_inverse_sa.argtypes = [P, I64, P]
            lib.oracle_inverse_sa.restype = I64
            lib.oracle_sa_check_range.argtypes = [P, I64, P, P, I64, I64]
            lib.oracle_sa_check_range.restype = I64
            lib.oracle_lcp_kasai_range.argtypes = [P, I64, P, P, I64, I64, P]
            lib.oracle_lcp_kasai_range.restype = ctypes.c_int
            lib.oracle_check_pairs.argtypes = [P, I64, P, P, P, I64]
            lib.oracle_check_pairs.restype = I64
            lib.oracle_split_sort_u64.argtypes = [P, P, I64, ctypes.c_int, ctypes.c_int]
            lib.oracle_split_sort_u64.restype = ctypes.c_int
            for name in ("oracle_overlaps_brute", "oracle_overlaps_sorted"):
                f = getattr(lib, name)
                f.argtypes = [P, P, I64, I32, P, P, P, I64]
                f.restype = I64
            lib.oracle_contained.argtypes = [P, P, I64, P]
            lib.oracle_contained.restype = ctypes.c_int
            lib.oracle_layout.argtypes = [P, P, I64, P, P, P, I64, P, P, I64, P, I64, P, P]
            lib.oracle_layout.restype = ctypes.c_int
            lib.oracle_overlaps_approx.argtypes = [P, P, I64, I32, I32, I32, ctypes.c_int, P, P, P, P, I64]
            lib.oracle_overlaps_approx.restype = I64
            lib.oracle_fir_reconstruct.argtypes = [P, P, I64, I64, P, P, P]
            lib.oracle_fir_reconstruct.restype = I64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _text(text) -> np.ndarray:
    if isinstance(text, (bytes, bytearray)):
        text = np.frombuffer(bytes(text), dtype=np.uint8)
    t = np.ascontiguousarray(text, dtype=np.uint8)
    if t.size == 0 or t[-1] != SEP:
        raise ValueError("text must be non-empty and end with '$'")
    return t


def read_offsets(text) -> np.ndarray:
    """toff[r] = start of fragment r in the text; toff[n_reads] = N."""
    t = _text(text)
    ends = np.flatnonzero(t == SEP) + 1
    return np.concatenate([[0], ends]).astype(np.int64)


def suffix_array(text) -> np.ndarray:
    t = _text(text)
    sa = np.empty(t.size, dtype=np.int64)
    rc = _load().oracle_suffix_array(_ptr(t), t.size, _ptr(sa))
    if rc != 0:
        raise RuntimeError(f"oracle_suffix_array failed ({rc})")
    return sa


def lcp_kasai(text, sa) -> np.ndarray:
    t = _text(text)
    sa = np.ascontiguousarray(sa, dtype=np.int64)
    lcp = np.empty(t.size, dtype=np.int32)
    rc = _load().oracle_lcp_kasai(_ptr(t), t.size, _ptr(sa), _ptr(lcp))
    if rc != 0:
        raise RuntimeError(f"oracle_lcp_kasai failed ({rc})")
    return lcp


def lcp_direct(text, sa) -> np.ndarray:
    t = _text(text)
    sa = np.ascontiguousarray(sa, dtype=np.int64)
    lcp = np.empty(t.size, dtype=np.int32)
    rc = _load().oracle_lcp_direct(_ptr(t), t.size, _ptr(sa), _ptr(lcp))
    if rc != 0:
        raise RuntimeError(f"oracle_lcp_direct failed ({rc})")
    return lcp


def sa_check(text, sa) -> int:
    """0 when ``sa`` is the suffix array of ``text``; a positive code otherwise."""
    t = _text(text)
    sa = np.ascontiguousarray(sa, dtype=np.int64)
    if sa.size != t.size:
        return 1
    return int(_load().oracle_sa_check(_ptr(t), t.size, _ptr(sa)))


def _ranges(n0: int, n1: int, parts: int):
    step = max(1, -(-(n1 - n0) // max(parts, 1)))
    return [(a, min(a + step, n1)) for a in range(n0, n1, step)]


def sa_check_and_lcp_threaded(text, sa, threads: int = 0):
    """The Burkhardt-Kaerkkaeinen check of ``sa`` and Kasai's LCP, each split into
    ranges run on host threads (ctypes releases the GIL during the C calls).
    Returns (check code, lcp): code 0 means ``sa`` is the suffix array (same codes
    as :func:`sa_check`; 2 + j names the smallest failing pair found in its range).
    ``lcp`` is None when the check fails."""
    from concurrent.futures import ThreadPoolExecutor

    t = _text(text)
    N = t.size
    sa = np.ascontiguousarray(sa, dtype=np.int64)
    if sa.size != N:
        return 1, None
    lib = _load()
    isa = np.empty(N, dtype=np.int64)
    rc = int(lib.oracle_inverse_sa(_ptr(sa), N, _ptr(isa)))
    if rc != 0:
        return rc, None
    threads = threads or (os.cpu_count() or 1)
    with ThreadPoolExecutor(threads) as ex:
        codes = list(ex.map(lambda r: int(lib.oracle_sa_check_range(_ptr(t), N, _ptr(sa), _ptr(isa),
                                                                    r[0], r[1])),
                            _ranges(1, N, 4 * threads)))
        bad = [c for c in codes if c != 0]
        if bad:
            return min(bad), None
        lcp = np.empty(N, dtype=np.int32)
        rcs = list(ex.map(lambda r: int(lib.oracle_lcp_kasai_range(_ptr(t), N, _ptr(sa), _ptr(isa),
                                                                  r[0], r[1], _ptr(lcp))),
                          _ranges(0, N, 4 * threads)))
    if any(rcs):
        raise RuntimeError("oracle_lcp_kasai_range failed")
    return 0, lcp


def check_pairs(text, sa, lcp, idx) -> int:
    """Violations among the sampled SA neighbours (j-1, j), j in idx: order, and
    LCP when lcp is not None.  For arrays too large to check in full."""
    t = _text(text)
    sa = np.ascontiguousarray(sa, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    lp = None
    if lcp is not None:
        lcp = np.ascontiguousarray(lcp, dtype=np.int32)
        lp = _ptr(lcp)
    n = _load().oracle_check_pairs(_ptr(t), t.size, _ptr(sa), lp, _ptr(idx), idx.size)
    if n < 0:
        raise RuntimeError("oracle_check_pairs: bad arguments")
    return int(n)


def split_sort(keys, vals, lo_bit: int, hi_bit: int):
    """Algorithm 1: stable LSD sort of (keys, vals) on key bits [lo_bit, hi_bit)."""
    k = np.array(keys, dtype=np.uint64, copy=True)
    v = np.array(vals, dtype=np.uint64, copy=True)
    if k.shape != v.shape:
        raise ValueError("keys and vals differ in length")
    rc = _load().oracle_split_sort_u64(_ptr(k), _ptr(v), k.size, lo_bit, hi_bit)
    if rc != 0:
        raise RuntimeError(f"oracle_split_sort_u64 failed ({rc})")
    return k, v


def _overlaps(fn, text, lmin):
    t = _text(text)
    toff = read_offsets(t)
    nr = toff.size - 1
    f = getattr(_load(), fn)
    n = f(_ptr(t), _ptr(toff), nr, lmin, None, None, None, 0)
    if n < 0:
        raise RuntimeError(f"{fn} failed ({n})")
    ej = np.empty(max(n, 1), dtype=np.int32)
    ek = np.empty(max(n, 1), dtype=np.int32)
    eL = np.empty(max(n, 1), dtype=np.int32)
    n2 = f(_ptr(t), _ptr(toff), nr, lmin, _ptr(ej), _ptr(ek), _ptr(eL), n)
    assert n2 == n
    return ej[:n].copy(), ek[:n].copy(), eL[:n].copy()


def overlaps_brute(text, lmin: int):
    """Edges (j, k, L) with the max proper suffix-prefix overlap L >= lmin, in (j, k) order."""
    return _overlaps("oracle_overlaps_brute", text, lmin)


def overlaps_sorted(text, lmin: int):
    """The same edge set as :func:`overlaps_brute`, by binary search over sorted fragments."""
    return _overlaps("oracle_overlaps_sorted", text, lmin)


def contained(text) -> np.ndarray:
    t = _text(text)
    toff = read_offsets(t)
    out = np.empty(max(toff.size - 1, 1), dtype=np.uint8)
    rc = _load().oracle_contained(_ptr(t), _ptr(toff), toff.size - 1, _ptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle_contained failed ({rc})")
    return out[: toff.size - 1].copy()


def layout(text, edges, contained_flags):
    """Greedy layout; returns (contig bytes concatenated as uint8, int64 offsets)."""
    t = _text(text)
    toff = read_offsets(t)
    nr = toff.size - 1
    ej, ek, eL = (np.ascontiguousarray(e, dtype=np.int32) for e in edges)
    c = np.ascontiguousarray(contained_flags, dtype=np.uint8)
    lib = _load()
    nc = ctypes.c_int64(0)
    nb = ctypes.c_int64(0)
    cap = t.size
    out = np.empty(max(cap, 1), dtype=np.uint8)
    off = np.empty(nr + 2, dtype=np.int64)
    rc = lib.oracle_layout(_ptr(t), _ptr(toff), nr, _ptr(ej), _ptr(ek), _ptr(eL), ej.size,
                           _ptr(c), _ptr(out), cap, _ptr(off), off.size,
                           ctypes.byref(nc), ctypes.byref(nb))
    if rc != 0:
        raise RuntimeError(f"oracle_layout failed ({rc})")
    return out[: nb.value].copy(), off[: nc.value + 1].copy()


def assemble(text, lmin: int, overlap_fn=overlaps_sorted):
    """Whole method on one fragment set: overlaps -> containment -> layout -> contigs."""
    edges = overlap_fn(text, lmin)
    c = contained(text)
    return layout(text, edges, c)


def contigs_as_list(buf: np.ndarray, off: np.ndarray):
    return [bytes(buf[off[i]: off[i + 1]]) for i in range(off.size - 1)]


FIR_SOLVED, FIR_NONE, FIR_GAVE_UP = 0, 1, 2


def fir_reconstruct(text, max_steps: int = 1 << 40):
    """Sec. III two-cut reconstruction.  Returns (status, frag_start, rs, steps):
    status 0 solved / 1 none exists / 2 gave up after max_steps placed fragments;
    frag_start[r] = offset of fragment r in the result RS (-1 unless solved);
    rs = the reconstructed sequence (bytes, empty unless solved)."""
    t = _text(text)
    toff = read_offsets(t)
    nr = toff.size - 1
    start = np.empty(max(nr, 1), dtype=np.int64)
    st = ctypes.c_int32(0)
    rl = ctypes.c_int64(0)
    steps = _load().oracle_fir_reconstruct(_ptr(t), _ptr(toff), nr, int(max_steps), _ptr(start),
                                           ctypes.byref(st), ctypes.byref(rl))
    if steps < 0:
        raise RuntimeError(f"oracle_fir_reconstruct failed ({steps})")
    start = start[:nr].copy()
    rs = b""
    if st.value == FIR_SOLVED:
        buf = np.zeros(rl.value, dtype=np.uint8)
        for r in range(nr):
            buf[start[r]: start[r] + toff[r + 1] - 1 - toff[r]] = t[toff[r]: toff[r + 1] - 1]
        rs = buf.tobytes()
    return int(st.value), start, rs, int(steps)


def overlaps_approx(text, lmin: int, mu_num: int = 0, mu_den: int = 1, rc: bool = False):
    """Edges (a, b, L, mismatches) between oriented fragments (2r = fragment r,
    2r + 1 = its reverse complement when rc), the largest L per ordered pair with
    at most floor(L * mu_num / mu_den) substitutions; (a, b) order."""
    t = _text(text)
    toff = read_offsets(t)
    nr = toff.size - 1
    f = _load().oracle_overlaps_approx
    n = f(_ptr(t), _ptr(toff), nr, lmin, mu_num, mu_den, int(rc), None, None, None, None, 0)
    if n < 0:
        raise RuntimeError(f"oracle_overlaps_approx failed ({n})")
    out = [np.empty(max(n, 1), dtype=np.int32) for _ in range(4)]
    n2 = f(_ptr(t), _ptr(toff), nr, lmin, mu_num, mu_den, int(rc), *(_ptr(o) for o in out), n)
    assert n2 == n
    return tuple(o[:n].copy() for o in out)
