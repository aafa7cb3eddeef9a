"""Served: jobs submitted while others run are batched and overlapped; each
result must be, byte for byte, the job assembled alone (tolerance zero)."""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1404_3456_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def B():
    from paper_1404_3456_gb300 import binding

    return binding


def jobs(n, seed=3):
    out = []
    for i in range(n):
        j = synth.served_job(seed, i, g_lo=5_000, g_hi=60_000)
        out.append(j)
    return out


def test_server_results_equal_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    js = jobs(24)
    ctx = B().Context(0)
    alone = [B().assemble_text(ctx, torch.from_numpy(j["text"]).cuda(), j["min_overlap"]) for j in js]
    ctx.close()
    srv = B().Server(0, slots=2, max_batch=8)
    got = {}
    # submit from another thread at staggered times, so that jobs arrive while
    # earlier batches are on the GPU
    def feed():
        for i, j in enumerate(js):
            srv.submit(j["text"], j["min_overlap"], i)
            time.sleep(0.002 * (i % 3))
    th = threading.Thread(target=feed)
    th.start()
    deadline = time.time() + 120
    while len(got) < len(js) and time.time() < deadline:
        for r in srv.poll(64, wait_ms=200):
            assert r["status"] == 0
            got[r["id"]] = r
    th.join()
    srv.close()
    assert len(got) == len(js)
    for i in range(len(js)):
        assert got[i]["contigs"] == alone[i], i
        assert got[i]["t_submit_ms"] <= got[i]["t_start_ms"] <= got[i]["t_done_ms"]
    # and against the oracle for a few
    for i in (0, 5, 11):
        buf, off = oracle.assemble(js[i]["text"], js[i]["min_overlap"])
        assert got[i]["contigs"] == oracle.contigs_as_list(buf, off)


def test_server_admission_by_budget():
    """A budget that fits one job at a time still finishes every job (one by one)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    js = jobs(5, seed=4)
    srv = B().Server(0, hbm_budget=1, slots=2, max_batch=8)   # nothing fits: each runs alone
    for i, j in enumerate(js):
        srv.submit(j["text"], j["min_overlap"], i)
    got = {}
    deadline = time.time() + 60
    while len(got) < len(js) and time.time() < deadline:
        for r in srv.poll(64, wait_ms=200):
            got[r["id"]] = r
    srv.close()
    assert sorted(got) == list(range(5))
    # alone in the GPU: no two jobs' [start, done] windows overlap
    spans = sorted((r["t_start_ms"], r["t_done_ms"]) for r in got.values())
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 1e-6


def test_server_refuses_malformed_jobs_and_keeps_serving():
    """A malformed text is refused at submit (bad byte, empty fragment, missing
    final '$', leading '$'); the jobs around it are served as if it never came."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    js = jobs(3, seed=6)
    srv = B().Server(0, slots=2, max_batch=8)
    bad = [b"ACGTN$", b"ACG$$TTA$", b"ACGT", b"$ACGT$"]
    srv.submit(js[0]["text"], js[0]["min_overlap"], 0)
    for t in bad:
        with pytest.raises(B().DnasaError) as e:
            srv.submit(np.frombuffer(t, dtype=np.uint8), 31, 99)
        assert e.value.status == B().BAD_ALPHABET
    srv.submit(js[1]["text"], js[1]["min_overlap"], 1)
    srv.submit(js[2]["text"], js[2]["min_overlap"], 2)
    got = {}
    deadline = time.time() + 60
    while len(got) < 3 and time.time() < deadline:
        for r in srv.poll(64, wait_ms=200):
            got[r["id"]] = r
    srv.close()
    assert sorted(got) == [0, 1, 2]
    for i in range(3):
        assert got[i]["status"] == 0
        buf, off = oracle.assemble(js[i]["text"], js[i]["min_overlap"])
        assert got[i]["contigs"] == oracle.contigs_as_list(buf, off)


def test_server_budget_for_two_jobs_never_runs_three():
    """With a budget that holds exactly two jobs' estimates (and 3 slots that
    could run more), at no moment are three jobs on the GPU: admission counts
    each job at dnasa_server_job_bytes."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    js = [synth.served_job(8, i, g_lo=40_000, g_hi=40_000) for i in range(9)]
    sizes = {(j["text"].size, int((j["text"] == ord("$")).sum())) for j in js}
    assert len(sizes) == 1
    N, nr = sizes.pop()
    jb = B().Server.job_bytes(N, nr)
    assert jb > 95 * N   # the suffix-array workspace alone is ~95 bytes per symbol
    srv = B().Server(0, hbm_budget=2 * jb + jb // 2, slots=3, max_batch=8)
    for i, j in enumerate(js):
        srv.submit(j["text"], j["min_overlap"], i)
    got = {}
    deadline = time.time() + 120
    while len(got) < len(js) and time.time() < deadline:
        for r in srv.poll(64, wait_ms=200):
            assert r["status"] == 0
            got[r["id"]] = r
    srv.close()
    assert sorted(got) == list(range(len(js)))
    events = sorted([(r["t_start_ms"], 1) for r in got.values()] +
                    [(r["t_done_ms"], -1) for r in got.values()])   # ends sort before starts
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 2, f"{peak} jobs in flight at once"
    assert peak == 2   # and the budget is used: two run together
    for i in (0, 4):
        buf, off = oracle.assemble(js[i]["text"], js[i]["min_overlap"])
        assert got[i]["contigs"] == oracle.contigs_as_list(buf, off)
