#!/usr/bin/env python
"""Benchmark: suffix-array build (+ LCP) of a 64 Mbp synthetic genome on one GB300.

Workload ("sa64m"): a seeded 64,000,000 bp genome -- 90 % i.i.d. uniform ACGT,
5 % tandem arrays (period U{2..50}, U{10..200} copies), 5 % copies of one
300 bp element with 1 % substitutions -- as one '$'-terminated fragment
(N = 64,000,001 suffixes), 2-bit packed and resident in HBM before timing.
One step = sa_build (int32 SA) + lcp_build (int32 LCP) through the C ABI.
The working set (keys, values, ranks: ~3.5 GB) is far larger than the 129 MB
L2, so no flush is needed between steps.

Metric: Msuffix/s = N * ranks / (max-over-ranks seconds per step) / 1e6.
The single-instance path does not shard across GPUs: with --gpus N every rank
runs its own replica (weak scaling, no collective on the data path).

Extra keys: roofline (the dominant kernel's algorithmic GB/s, timed live with
CUDA events on its stream, against the measured HBM copy peak), cpu_baseline
(the oracle on a bounded prefix of the same genome, single thread), e2e (the
same step with host buffers: H2D of the packed text, D2H of SA + LCP), clocks
sampled by nvidia-smi during the timed region, gpu_launches.

--impl reference times the oracle (plain C, single thread) on a bounded prefix
of the same genome, per step, and prints the same JSON line with
"impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SA build Msuffix/s (suffix array + LCP, 64 Mbp genome)"
UNIT = "Msuffix/s"
SAMPLE_CPU = 16_000_000   # oracle sample for cpu_baseline (~10-20 s single-threaded)
SAMPLE_REF = 4_000_000    # oracle sample per --impl reference step (~3 s)
G = 64_000_000
TUNE_CACHE = os.path.join(ROOT, "paper_1404_3456_gb300", "_build", "tune_cache.tsv")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dnasa", choices=["dnasa", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--genome", type=int, default=G, help="genome length (default 64,000,000)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="sa64m",
                    choices=["sa64m", "large", "batched", "served", "fir", "approx"])
    ap.add_argument("--instances", type=int, default=4096, help="batched: fragment sets per batch")
    ap.add_argument("--solo-sample", type=int, default=256,
                    help="batched: instances timed one job per launch")
    ap.add_argument("--jobs", type=int, default=48, help="served: jobs in the trace")
    ap.add_argument("--distinct", type=int, default=0,
                    help="served: distinct generated jobs the trace cycles through (0 = all distinct)")
    ap.add_argument("--lambdas", default="0.25,0.5,0.75,0.9,1.0,1.25",
                    help="served: arrival rates as multiples of one-job-per-launch capacity")
    ap.add_argument("--no-tune", action="store_true", help="skip the build-option autotuner")
    ap.add_argument("--separate", action="store_true",
                    help="build the SA and the LCP with two calls (sa_build, lcp_build) instead of sa_lcp_build")
    ap.add_argument("--host-rounds", action="store_true",
                    help="run the doubling rounds from the host instead of the captured graph")
    ap.add_argument("--builder", default="doubling", choices=["doubling", "dc3"],
                    help="sa64m / large: suffix-array builder (dc3: the difference-cover algorithm)")
    ap.add_argument("--slots", type=int, default=2)
    ap.add_argument("--max-batch", type=int, default=16)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def rank_setup(local_rank: int, world: int, backend: str = "nccl"):
    """One process per GPU: joins the process group (NCCL between GPUs; gloo for
    the CPU tests of this logic) when there is more than one rank."""
    if world > 1:
        import torch
        import torch.distributed as dist

        if backend == "nccl":
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        else:
            dist.init_process_group(backend)


def rank_barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def over_ranks(values, world: int, op: str = "max", device=None):
    """values reduced over the ranks (max or sum); the values themselves at one rank."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()]


def rank_teardown(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def genome_text(seed: int, size: int):
    from paper_1404_3456_gb300 import synth

    g = synth.sa64m_genome(seed, G)
    if size < G:
        g = g[:size]
    return synth.genome_text(g)


def cpu_oracle_rate(text: np.ndarray):
    """Oracle SA + Kasai LCP of `text` on one host core; returns (Msuffix/s, seconds)."""
    import oracle

    t0 = time.perf_counter()
    sa = oracle.suffix_array(text)
    oracle.lcp_kasai(text, sa)
    dt = time.perf_counter() - t0
    return text.size / dt / 1e6, dt


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    sample = genome_text(args.seed, SAMPLE_REF)
    for _ in range(args.warmup):
        cpu_oracle_rate(sample)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_rate(sample)
        times.append(dt)
    ms = 1000.0 * sum(times) / len(times)
    value = sample.size / (ms / 1000.0) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32", "data": "synthetic",
        "config": {"workload": f"sa64m prefix: oracle SA + Kasai LCP of the first {SAMPLE_REF:,} "
                               "bases of the 64 Mbp genome (bounded sample)",
                   "genome_bp": SAMPLE_REF, "seed": args.seed},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {SAMPLE_REF:,} bp of the sa64m genome, per step; "
                                   f"its Msuffix/s is extrapolated to the {G:,} bp workload "
                                   "(a direct-comparison sort slows as the text grows, so the "
                                   "true full-size rate is lower)",
                         "extrapolated": True},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def pctl(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


ROOF_TIMING = ("per-launch CUDA events on the launching stream, second pass of the same K steps "
               "(with per-launch events the doubling rounds run from the host, not inside the "
               "captured graph the timed steps use)")


def traffic_ratio(kind: str):
    """DRAM bytes (ncu dram__bytes_read + write) per algorithmic byte of a kernel
    class, from profiles/traffic.json -- only while the class's kernel source is the
    one the counters were taken on (sha1 pinned there), else None."""
    import hashlib

    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tj = json.load(open(tfile)).get(kind)
        if not tj or not tj.get("valid"):
            return None
        src = os.path.join(ROOT, tj["source"])
        if hashlib.sha1(open(src, "rb").read()).hexdigest() != tj["source_sha1"]:
            return None
        return float(tj["dram_per_algorithmic_byte"])
    except Exception:
        return None


def roofline_of(prof, peak, peak_src, steps):
    if not prof:
        return None, {}
    name, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    achieved = d["bytes"] / (d["ms"] / 1000.0) / 1e9 if d["ms"] > 0 else 0.0
    total = sum(x["ms"] for x in prof.values())
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / steps, "share": v["ms"] / total}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    return ({"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
             "frac": achieved / peak, "peak_source": peak_src, "traffic": None,
             "launches": d["launches"], "timing": ROOF_TIMING}, kernels)


def _oracle_assemble(text):
    """Pool worker: the oracle's whole method on one fragment set (host only)."""
    import oracle

    oracle.assemble(text, 31)
    return int(text.size)


def oracle_all_cores(texts):
    """The oracle, unchanged, on every host core at once: one instance per worker
    process (spawned, so that no worker inherits the GPU context)."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_assemble, texts[:1])   # workers up and the library loaded
        t0 = time.perf_counter()
        pool.map(_oracle_assemble, texts, chunksize=1)
        dt = time.perf_counter() - t0
    return len(texts) / dt, cores, dt


def large_reads_stage(args, ctx, binding, genome_np, dev, min_overlap=31, n_reads=10_000_000,
                      read_len=150):
    """Overlap search over 10 M reads of 150 bp drawn from the 1.5 Gbp genome (1x):
    SA (int32) and LCP of the reads' text, then every suffix of every read with at
    least min_overlap bases queried against the read starts.  One warm-up run,
    then one timed run per stage (CUDA events)."""
    import torch

    from paper_1404_3456_gb300 import synth

    text_np, _ = synth.large_reads(args.seed, genome_np, n_reads, read_len)
    N = int(text_np.size)
    text = torch.from_numpy(text_np).to(dev)
    packed, toff, nr = binding.pack_text(ctx, text)
    del text
    sa = torch.empty(N, dtype=torch.int32, device=dev)
    lcp = torch.empty(N, dtype=torch.int32, device=dev)
    edges = torch.empty((64 << 20, 3), dtype=torch.int32, device=dev)   # first 64 M edges kept
    contained = torch.empty(nr, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ne = 0
    for rep in range(2):
        ev[0].record(stream)
        binding.sa_build(ctx, packed, toff, nr, N, sa)
        ev[1].record(stream)
        binding.lcp_build(ctx, packed, toff, nr, N, sa, lcp)
        ev[2].record(stream)
        ne = binding.overlap_search(ctx, packed, toff, nr, N, sa, lcp, min_overlap, edges, contained,
                                    count_only_past_cap=True)
        ev[3].record(stream)
        torch.cuda.synchronize()
    sa_ms, lcp_ms, ovl_ms = (ev[i].elapsed_time(ev[i + 1]) for i in range(3))
    queries = nr * max(0, read_len - min_overlap)   # suffixes r_j[o..], o >= 1, >= min_overlap bases
    return {"workload": f"{nr:,} reads x {read_len} bp from the same genome (1x), min overlap "
                        f"{min_overlap}; N = {N:,}", "sa_ms": sa_ms, "lcp_ms": lcp_ms,
            "overlap_ms": ovl_ms, "queries": queries,
            "overlap_queries_per_s": queries / (ovl_ms / 1000.0), "edges": int(ne),
            "edges_stored": int(min(ne, edges.shape[0])),
            "contained": int(contained.sum().item()),
            "sa_msuffix_per_s": N / (sa_ms / 1000.0) / 1e6}


def run_batched(args):
    """Batched workload: independent fragment sets (genome log-uniform 2-200 kbp,
    reads U{100..1000} at 8x, min overlap 31) assembled by one assemble_batched
    call per step, against one assemble() call per instance."""
    import torch

    import oracle
    from paper_1404_3456_gb300 import binding, synth

    rank, local_rank, world = dist_env()
    rank_setup(local_rank, world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # instances shard by rank: each rank draws its own fragment sets
    insts = [synth.batched_instance(args.seed + 1000 * rank, i) for i in range(args.instances)]
    texts = [x["text"] for x in insts]
    inst_off = np.concatenate([[0], np.cumsum([t.size for t in texts])]).astype(np.int64)
    N = int(inst_off[-1])
    ctx = binding.Context(local_rank)
    h_text = torch.from_numpy(np.concatenate(texts)).pin_memory()
    d_text = h_text.cuda()
    contigs = torch.empty(N, dtype=torch.uint8, device="cuda")
    off = torch.empty(N // 2 + 2, dtype=torch.int64, device="cuda")
    ioff = torch.empty(len(texts) + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    opts, tuned = None, None
    if not args.no_tune:
        packed, toff, nr = binding.pack_text(ctx, d_text)
        opts, tms = binding.dnasa_autotune(ctx, packed, toff, nr, N, inst_off, cache_path=TUNE_CACHE)
        tuned = {"tile_items": opts.tile_items, "finish_threshold": opts.finish_threshold,
                 "lookback": opts.lookback, "sa_ms": tms}
        del packed, toff

    def step(t=d_text):
        return binding.assemble_batched(ctx, t, inst_off, 31, contigs, off, ioff, opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    trace = ctx.trace()
    l0 = ctx.launch_count()
    clocks = ClockSampler(local_rank)
    rank_barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        nc, nb = step()
    e1.record(stream)
    torch.cuda.synchronize()
    rank_barrier(world)
    clk = clocks.stop()
    launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    # per-kernel durations for the roofline: the same steps with per-launch events
    ctx.profile(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    # end to end: text from pinned host memory, contigs and offsets back
    h_contigs = torch.empty(N, dtype=torch.uint8).pin_memory()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d2 = torch.empty_like(d_text)
    x0.record(stream)
    for _ in range(args.steps):
        d2.copy_(h_text, non_blocking=True)
        nc, nb = step(d2)
        h_contigs[:nb].copy_(contigs[:nb], non_blocking=True)
        ho = off[: nc + 1].cpu()
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = x0.elapsed_time(x1) / args.steps
    ms, e2e_ms = over_ranks([ms, e2e_ms], world, "max", dev)
    launches = int(over_ranks([launches], world, "sum", dev)[0])
    # one job per launch on the first M instances, and the batch of the same M
    M = min(args.solo_sample, len(texts))
    d_solo = [torch.from_numpy(t).cuda() for t in texts[:M]]
    for t in d_solo[:4]:
        binding.assemble_text(ctx, t, 31)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in d_solo:
        binding.assemble_text(ctx, t, 31)
    torch.cuda.synchronize()
    solo_s = time.perf_counter() - t0
    sub_off = inst_off[: M + 1]
    d_sub = d_text[: int(sub_off[-1])]
    sub_opts = None
    if not args.no_tune:   # the switch point depends on N: tune the subset on its own
        packed, toff, nr = binding.pack_text(ctx, d_sub)
        sub_opts, _ = binding.dnasa_autotune(ctx, packed, toff, nr, int(sub_off[-1]), sub_off,
                                             cache_path=TUNE_CACHE)
        del packed, toff
    binding.assemble_batched(ctx, d_sub, sub_off, 31, contigs, off, ioff[: M + 1], sub_opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    binding.assemble_batched(ctx, d_sub, sub_off, 31, contigs, off, ioff[: M + 1], sub_opts)
    torch.cuda.synchronize()
    sub_s = time.perf_counter() - t0
    cpu, cpu_all = None, None
    if not args.no_cpu_baseline and world == 1:
        sample = texts[:4]
        t0 = time.perf_counter()
        for t in sample:
            oracle.assemble(t, 31)
        dt = time.perf_counter() - t0
        cpu = {"value": len(sample) / dt, "unit": "assemblies/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle assemble of the first {len(sample)} instances "
                         f"({sum(t.size for t in sample):,} symbols), {dt:.1f} s"}
        many = texts[: 4 * (os.cpu_count() or 1)]
        rate, cores, dt = oracle_all_cores(many)
        cpu_all = {"value": rate, "unit": "assemblies/s", "cores": cores, "kind": "oracle",
                   "sample": f"oracle assemble of the first {len(many)} instances, one per worker "
                             f"process, {dt:.1f} s"}
    peak, src = measured_peak()
    roof, kernels = roofline_of(prof, peak, src, args.steps)
    value = len(texts) * world / (ms / 1000.0)
    line = {
        "metric": "batched assemblies/s (assemble_batched, 4096 fragment sets)", "value": value,
        "unit": "assemblies/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8/int32", "data": "synthetic",
        "config": {"workload": f"batched: {len(texts)} instances, {N:,} symbols, genome log-uniform "
                               "2-200 kbp, reads U{100..1000} at 8x, min overlap 31",
                   "msuffix_per_s": N * world / (ms / 1000.0) / 1e6,
                   "one_job_per_launch": {"instances": M, "s": solo_s, "assemblies_per_s": M / solo_s},
                   "batched_same_instances": {"instances": M, "s": sub_s, "assemblies_per_s": M / sub_s},
                   "oracle_all_cores": cpu_all,
                   "sa_rounds": trace["rounds"], "active_per_round": trace["active"],
                   "autotuned": tuned},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": len(texts) / (e2e_ms / 1000.0), "unit": "assemblies/s",
                "h2d_bytes_per_step": N, "d2h_bytes_per_step": int(nb) + 8 * (int(nc) + 1),
                "ms_per_step": e2e_ms},
        "gpu_launches": launches, "clocks": clk, "kernels": kernels,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rank_teardown(world)
    return 0


def run_fir(args):
    """Two-cut workload (Sec. III, Fig. 2): independent genomes log-uniform
    2-200 kbp, each cut by two shotguns into pieces of mean 500 bp (every break
    different, at least 24 bp apart), the pieces of both shuffled; one
    fir_reconstruct_batched call per step rebuilds every genome by the fir
    search with back-tracking."""
    import torch

    import oracle
    from paper_1404_3456_gb300 import binding, synth

    rank, local_rank, world = dist_env()
    rank_setup(local_rank, world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n_inst = args.instances
    texts, genomes = [], []
    for i in range(n_inst):   # instances shard by rank: each rank draws its own
        rng = synth.rng_for(args.seed * 1_000_003 + 1000 * rank + i, 8)
        G = synth.log_uniform(rng, 2_000, 200_000)
        d = synth.two_cut(args.seed * 1_000_003 + 1000 * rank + i, G, mean_len=500)
        texts.append(d["text"])
        genomes.append(d["genome"])
    inst_off = np.concatenate([[0], np.cumsum([t.size for t in texts])]).astype(np.int64)
    N = int(inst_off[-1])
    nf = int(sum(int((t == ord("$")).sum()) for t in texts))
    ctx = binding.Context(local_rank)
    h_text = torch.from_numpy(np.concatenate(texts)).pin_memory()
    d_text = h_text.cuda()
    start = torch.empty(nf, dtype=torch.int64, device=dev)
    rs = torch.empty(N, dtype=torch.uint8, device=dev)
    rs_off = torch.empty(n_inst + 1, dtype=torch.int64, device=dev)
    status = torch.empty(n_inst, dtype=torch.int32, device=dev)
    steps_d = torch.empty(n_inst, dtype=torch.int64, device=dev)
    max_steps = 1 << 20
    stream = torch.cuda.current_stream()

    def step(t=d_text):
        return binding.fir_reconstruct_batched_into(ctx, t, inst_off, max_steps, start, rs, rs_off,
                                                    status, steps_d)

    for _ in range(args.warmup):
        total = step()
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    so = rs_off.cpu().numpy()
    buf = rs[:total].cpu().numpy()
    solved = int((st == 0).sum())
    exact = sum(1 for i in range(n_inst)
                if st[i] == 0 and np.array_equal(buf[so[i]: so[i + 1]], genomes[i]))
    l0 = ctx.launch_count()
    clocks = ClockSampler(local_rank)
    rank_barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        total = step()
    e1.record(stream)
    torch.cuda.synchronize()
    rank_barrier(world)
    clk = clocks.stop()
    launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    ctx.profile(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    h_rs = torch.empty(N, dtype=torch.uint8).pin_memory()
    d2 = torch.empty_like(d_text)
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    for _ in range(args.steps):
        d2.copy_(h_text, non_blocking=True)
        total = step(d2)
        h_rs[:total].copy_(rs[:total], non_blocking=True)
        h_off = rs_off.cpu()
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = x0.elapsed_time(x1) / args.steps
    ms, e2e_ms = over_ranks([ms, e2e_ms], world, "max", dev)
    launches = int(over_ranks([launches], world, "sum", dev)[0])
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        sample = texts[: min(256, n_inst)]
        t0 = time.perf_counter()
        for t in sample:
            oracle.fir_reconstruct(t, max_steps)
        dt = time.perf_counter() - t0
        cpu = {"value": len(sample) / dt, "unit": "reconstructions/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle fir search (direct string comparison, no suffix array) on the "
                         f"first {len(sample)} instances, {dt:.1f} s"}
    peak, src = measured_peak()
    roof, kernels = roofline_of(prof, peak, src, args.steps)
    line = {
        "metric": f"two-cut fir reconstructions/s (fir_reconstruct_batched, {n_inst} genomes)",
        "value": n_inst * world / (ms / 1000.0), "unit": "reconstructions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32", "data": "synthetic",
        "config": {"workload": f"fir: {n_inst} genomes log-uniform 2-200 kbp, each cut twice into "
                               f"pieces of mean 500 bp ({nf:,} fragments, {N:,} symbols)",
                   "solved": solved, "recovered_exactly": exact,
                   "msuffix_per_s": N * world / (ms / 1000.0) / 1e6},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": n_inst * world / (e2e_ms / 1000.0), "unit": "reconstructions/s",
                "h2d_bytes_per_step": N, "d2h_bytes_per_step": int(total) + 8 * (n_inst + 1),
                "ms_per_step": e2e_ms},
        "gpu_launches": launches, "clocks": clk, "kernels": kernels,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rank_teardown(world)
    return 0


def approx_reads(seed: int, G: int, coverage: float = 10.0, read_len: int = 150, subs: float = 0.01):
    """Reads of a G-base i.i.d. genome at uniform starts, each from a random strand
    (reverse complemented with probability 1/2) and with each base substituted
    with probability subs."""
    from paper_1404_3456_gb300 import synth

    rng = synth.rng_for(seed, 10)
    genome = synth.iid(rng, G)
    text, starts = synth.shotgun_fixed_text(rng, genome, coverage, read_len)
    m = text.reshape(-1, read_len + 1)[:, :read_len]
    codes = np.searchsorted(synth.BASES, m).astype(np.uint8)
    hit = rng.random(m.shape) < subs
    codes = np.where(hit, (codes + rng.integers(1, 4, size=m.shape, dtype=np.uint8)) % 4, codes)
    rev = rng.random(m.shape[0]) < 0.5
    codes[rev] = (3 - codes[rev])[:, ::-1]            # reverse complement (A<->T, C<->G)
    m[:] = synth.BASES[codes]
    return text


def run_approx(args):
    """Overlaps on both strands with substitutions (Sec. III DEFINITION): reads of
    150 bp at 10x from a 1 Mbp genome, half of them reverse complemented, 1 %
    substitutions; overlap_search_approx with both strands, min overlap 40, at
    most one mismatch per 30 bases."""
    import torch

    import oracle
    from paper_1404_3456_gb300 import binding

    rank, local_rank, world = dist_env()
    rank_setup(local_rank, world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    G = 1_000_000
    text_np = approx_reads(args.seed + 1000 * rank, G)
    N = int(text_np.size)
    nr = int((text_np == ord("$")).sum())
    ctx = binding.Context(local_rank)
    h_text = torch.from_numpy(text_np).pin_memory()
    d_text = h_text.cuda()
    edges, _ = binding.overlap_search_approx(ctx, d_text, 40, 1, 30, True)   # sizes the edge buffer
    cap = int(edges.shape[0]) + 1024
    buf = torch.empty((cap, 4), dtype=torch.int32, device=dev)
    import ctypes

    n_e, n_o = ctypes.c_int64(0), ctypes.c_int64(0)
    stream = torch.cuda.current_stream()

    def step(t=d_text):
        ctx.check(binding.lib().overlap_search_approx(ctx.handle, ctypes.c_void_p(t.data_ptr()), N, 40, 1, 30,
                                                      1, ctypes.c_void_p(buf.data_ptr()), cap,
                                                      ctypes.byref(n_e), ctypes.byref(n_o), None))
        return n_e.value

    for _ in range(args.warmup):
        ne = step()
    l0 = ctx.launch_count()
    clocks = ClockSampler(local_rank)
    rank_barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ne = step()
    e1.record(stream)
    torch.cuda.synchronize()
    rank_barrier(world)
    clk = clocks.stop()
    launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    ctx.profile(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    h_edges = torch.empty((cap, 4), dtype=torch.int32).pin_memory()
    d2 = torch.empty_like(d_text)
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    for _ in range(args.steps):
        d2.copy_(h_text, non_blocking=True)
        ne = step(d2)
        h_edges[:ne].copy_(buf[:ne], non_blocking=True)
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = x0.elapsed_time(x1) / args.steps
    ms, e2e_ms = over_ranks([ms, e2e_ms], world, "max", dev)
    launches = int(over_ranks([launches], world, "sum", dev)[0])
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        sample = approx_reads(args.seed, 15_000)
        t0 = time.perf_counter()
        oracle.overlaps_approx(sample, 40, 1, 30, True)
        dt = time.perf_counter() - t0
        cpu = {"value": sample.size / dt / 1e6, "unit": "Msymbol/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle all-pairs approximate overlaps of the reads of a 15 kbp genome "
                         f"({sample.size:,} symbols), {dt:.1f} s; all pairs: its rate falls as the "
                         "read set grows"}
    peak, src = measured_peak()
    roof, kernels = roofline_of(prof, peak, src, args.steps)
    line = {
        "metric": "approximate two-strand overlap search Msymbol/s (overlap_search_approx)",
        "value": N * world / (ms / 1000.0) / 1e6, "unit": "Msymbol/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32", "data": "synthetic",
        "config": {"workload": f"approx: {nr:,} reads x 150 bp at 10x of a {G:,} bp genome, half reverse "
                               "complemented, 1 % substitutions; both strands, min overlap 40, mu = 1/30",
                   "edges": int(ne)},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": N * world / (e2e_ms / 1000.0) / 1e6, "unit": "Msymbol/s", "h2d_bytes_per_step": N,
                "d2h_bytes_per_step": 16 * int(ne), "ms_per_step": e2e_ms},
        "gpu_launches": launches, "clocks": clk, "kernels": kernels,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rank_teardown(world)
    return 0


def run_served(args):
    """Served workload: jobs with genome log-uniform 5 kbp - 5 Mbp (2 % tandem
    arrays), 150 bp reads at 10x, min overlap 41, arriving as a Poisson process at
    several multiples of the one-job-per-launch capacity.  The server (continuous
    batching) and a FIFO one-job-per-launch loop see the identical trace."""
    import threading

    import torch

    from paper_1404_3456_gb300 import binding, synth

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    n_pool = args.distinct if 0 < args.distinct < args.jobs else args.jobs
    pool = [synth.served_job(args.seed + 1000 * rank, i) for i in range(n_pool)]
    pool_pinned = [torch.from_numpy(j["text"]).pin_memory() for j in pool]
    jobs = [pool[i % n_pool] for i in range(args.jobs)]          # the trace's jobs
    pinned = [pool_pinned[i % n_pool] for i in range(args.jobs)]
    ctx = binding.Context(local_rank)

    def solo(i):  # one job per launch: upload, assemble, contigs back
        t = pinned[i].cuda(non_blocking=True)
        return binding.assemble_text(ctx, t, jobs[i]["min_overlap"])

    for i in range(min(3, len(jobs))):
        solo(i)
    t0 = time.perf_counter()
    for i in range(n_pool):   # capacity: every distinct job once
        solo(i)
    cap_s = time.perf_counter() - t0
    capacity = n_pool / cap_s
    rng = np.random.default_rng(args.seed)
    results = []
    srv = binding.Server(local_rank, slots=args.slots, max_batch=args.max_batch)
    clocks = ClockSampler(local_rank)
    clocks.start()
    for f in [float(x) for x in args.lambdas.split(",")]:
        lam = f * capacity
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(jobs)))
        # FIFO one job per launch on the trace
        lat = []
        t0 = time.perf_counter()
        for i, a in enumerate(arrivals):
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            solo(i)
            lat.append(1000.0 * (time.perf_counter() - t0 - a))
        fifo_span = time.perf_counter() - t0 - arrivals[0]
        # served, same trace
        done = {}
        t0 = time.perf_counter()

        def feed():
            for i, a in enumerate(arrivals):
                now = time.perf_counter() - t0
                if now < a:
                    time.sleep(a - now)
                srv.submit(jobs[i]["text"], jobs[i]["min_overlap"], i)
        th = threading.Thread(target=feed)
        th.start()
        while len(done) < len(jobs):
            for r in srv.poll(256, wait_ms=50):
                done[r["id"]] = (time.perf_counter() - t0, r)
        th.join()
        s_lat = [1000.0 * (done[i][0] - arrivals[i]) for i in range(len(jobs))]
        s_span = max(v[0] for v in done.values()) - arrivals[0]
        results.append({"lambda_x_capacity": f, "arrival_rate_jobs_per_s": lam,
                        "served": {"jobs_per_s": len(jobs) / s_span, "p50_ms": pctl(s_lat, 50),
                                   "p99_ms": pctl(s_lat, 99)},
                        "one_job_per_launch": {"jobs_per_s": len(jobs) / fifo_span,
                                               "p50_ms": pctl(lat, 50), "p99_ms": pctl(lat, 99)}})
    srv.close()
    clk = clocks.stop()
    top = results[-1]
    line = {
        "metric": "served jobs/s and p99 latency vs one-job-per-launch (continuous batching)",
        "value": top["served"]["jobs_per_s"], "unit": "jobs/s", "n_gpus": world,
        "steps": len(jobs), "warmup": 3, "ms_per_step": 1000.0 / top["served"]["jobs_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32",
        "data": "synthetic",
        "config": {"workload": f"served: {len(jobs)} jobs (genome log-uniform 5 kbp-5 Mbp, 2% tandem, "
                               "150 bp reads at 10x, min overlap 41), Poisson arrivals"
                               + (f"; the trace cycles through {n_pool} distinct generated jobs"
                                  if n_pool < len(jobs) else ""),
                   "one_job_per_launch_capacity_jobs_per_s": capacity,
                   "mean_job_symbols": float(np.mean([j["text"].size for j in jobs])),
                   "distinct_jobs": n_pool,
                   "slots": args.slots, "max_batch": args.max_batch, "sweep": results},
        "e2e": {"value": top["served"]["jobs_per_s"], "unit": "jobs/s",
                "h2d_bytes_per_step": float(np.mean([j["text"].size for j in jobs])),
                "d2h_bytes_per_step": None},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "fir":
        return run_fir(args)
    if args.workload == "approx":
        return run_approx(args)
    if args.workload == "served":
        return run_served(args)
    import torch

    rank, local_rank, world = dist_env()
    rank_setup(local_rank, world)
    torch.cuda.set_device(local_rank)
    from paper_1404_3456_gb300 import binding

    dev = torch.device("cuda", local_rank)
    large = args.workload == "large"
    if large:   # 1.5 Gbp, int64 SA (85 % i.i.d., 10 % tandem, 5 % copies of a 6 kbp element)
        from paper_1404_3456_gb300 import synth

        genome_np = synth.large_genome(args.seed)
        text_np = synth.genome_text(genome_np)
        args.no_e2e = True
    else:
        text_np = genome_text(args.seed, args.genome)
    N = int(text_np.size)
    idx_dtype = torch.int64 if large else torch.int32
    ctx = binding.Context(local_rank)
    stream = torch.cuda.current_stream()
    text = torch.from_numpy(text_np).to(dev)
    packed, toff, nr = binding.pack_text(ctx, text)
    del text
    sa = torch.empty(N, dtype=idx_dtype, device=dev)
    lcp = torch.empty(N, dtype=torch.int32, device=dev)
    opts, tuned = None, None
    if args.builder == "dc3":
        opts = binding.make_opts(builder=1)
    elif not args.no_tune:
        opts, tms = binding.dnasa_autotune(ctx, packed, toff, nr, N, cache_path=TUNE_CACHE)
        tuned = {"tile_items": opts.tile_items, "finish_threshold": opts.finish_threshold,
                 "lookback": opts.lookback, "sa_ms": tms}
    if args.host_rounds:
        opts = opts or binding.make_opts()
        opts.rounds_on_host = 1

    def step():
        if args.separate:
            binding.sa_build(ctx, packed, toff, nr, N, sa, opts)
            binding.lcp_build(ctx, packed, toff, nr, N, sa, lcp)
        else:   # one call: round 0 of the build writes the LCPs its initial keys decide
            binding.sa_lcp_build(ctx, packed, toff, nr, N, sa, lcp, opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    trace = ctx.trace()

    # ---- timed region (device): K steps between two events on the stream
    def barrier():
        rank_barrier(world)
        torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    barrier()
    clocks.start()
    l0 = ctx.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # the same K steps again with an event pair around every kernel launch: the
    # per-kernel durations of the roofline (kept out of the step time above,
    # which the per-launch events would lengthen by a few percent)
    ctx.profile(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)

    # SA-only time of one more step, for information
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    binding.sa_build(ctx, packed, toff, nr, N, sa, opts)
    s1.record(stream)
    torch.cuda.synchronize()
    sa_only_ms = s0.elapsed_time(s1)

    # ---- end to end: host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_packed = packed.cpu().pin_memory()
        h_toff = toff.cpu().pin_memory()
        h_sa = torch.empty(N, dtype=torch.int32).pin_memory()
        h_lcp = torch.empty(N, dtype=torch.int32).pin_memory()
        d_packed = torch.empty_like(packed)
        d_toff = torch.empty_like(toff)

        copy_stream = torch.cuda.Stream(device=dev)

        # one sa_lcp_build per step into alternating output buffers: a step's two
        # read-backs overlap the next step's build, and a buffer set is overwritten
        # only after its own read-backs (two steps earlier) are done.  Every copy is
        # inside the timed region.
        sa_bufs = [sa, torch.empty_like(sa)]
        lcp_bufs = [lcp, torch.empty_like(lcp)]
        read_done = [torch.cuda.Event(), torch.cuda.Event()]
        for ev in read_done:
            ev.record(copy_stream)
        turn = [0]

        def e2e_step():
            k = turn[0]
            turn[0] ^= 1
            d_packed.copy_(h_packed, non_blocking=True)
            d_toff.copy_(h_toff, non_blocking=True)
            stream.wait_event(read_done[k])
            binding.sa_lcp_build(ctx, d_packed, d_toff, nr, N, sa_bufs[k], lcp_bufs[k], opts)
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                h_sa.copy_(sa_bufs[k], non_blocking=True)
                h_lcp.copy_(lcp_bufs[k], non_blocking=True)
                read_done[k].record(copy_stream)

        for _ in range(4):   # two builds per buffer set: each set's graph is captured on its second
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        x0 = torch.cuda.Event(enable_timing=True)
        x1 = torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        stream.wait_stream(copy_stream)
        x1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = x0.elapsed_time(x1) / args.steps
        e2e = {"ms": e2e_ms, "h2d": h_packed.numel() * 8 + h_toff.numel() * 8, "d2h": 8 * N,
               "calls": ("sa_lcp_build into alternating output buffers; each step's read-backs overlap the "
                         "next step's build")}

    reads_info = None
    if large:   # the 10 M x 150 bp reads of the same genome: their own SA, LCP, overlap search
        del sa, lcp, packed, toff
        torch.cuda.empty_cache()
        reads_info = large_reads_stage(args, ctx, binding, genome_np, dev)
    ms, e2e_max = over_ranks([ms, e2e["ms"] if e2e else 0.0], world, "max", dev)
    if e2e:
        e2e["ms"] = e2e_max
    launches = int(over_ranks([launches], world, "sum", dev)[0])
    value = N * world / (ms / 1000.0) / 1e6

    if rank != 0:
        rank_teardown(world)
        return 0
    # ---- roofline of the dominant kernel class
    peak, peak_src = measured_peak()
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else None
    roofline = None
    if dom:
        name, d = dom
        achieved = d["bytes"] / (d["ms"] / 1000.0) / 1e9
        ratio = traffic_ratio(name)
        traffic = ratio * d["bytes"] / d["launches"] if ratio is not None else None
        all_bytes = sum(v["bytes"] for v in prof.values())
        all_ms = sum(v["ms"] for v in prof.values())
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                    "whole_path_frac": all_bytes / (all_ms / 1000.0) / 1e9 / peak if all_ms else None,
                    "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                    "traffic": traffic, "launches": d["launches"],
                    "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                    "avg_launch_ms": d["ms"] / d["launches"], "timing": ROOF_TIMING}
    breakdown = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                     "share": v["ms"] / max(1e-9, sum(x["ms"] for x in prof.values())),
                     "algorithmic_gbs": v["bytes"] / (v["ms"] / 1000.0) / 1e9 if v["ms"] else None,
                     "algorithmic_bytes_per_step": v["bytes"] / args.steps,
                     "dram_per_algorithmic_byte": traffic_ratio(k)}
                 for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    cpu = None
    if not args.no_cpu_baseline and world == 1:   # the oracle's baseline: rank 0 at N = 1 only
        if large:
            from paper_1404_3456_gb300 import synth

            sample = synth.genome_text(text_np[:SAMPLE_CPU].copy())
        else:
            sample = genome_text(args.seed, SAMPLE_CPU)
        rate, dt = cpu_oracle_rate(sample)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle SA + Kasai LCP of the first {SAMPLE_CPU:,} bp of the same "
                         f"genome, one run, {dt:.1f} s; the rate is extrapolated to the "
                         f"{N:,}-suffix workload (the oracle's direct-comparison sort slows as "
                         "the text grows, so the full-size rate would be lower)",
               "extrapolated": True}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/int32", "data": "synthetic",
        "config": {"workload": (f"large: suffix array + LCP of a {N - 1:,} bp genome, int64 SA, "
                                "int32 LCP" if large else
                                f"sa64m: suffix array + LCP of a {args.genome:,} bp genome "
                                f"(N = {N:,} suffixes), int32 SA and LCP"),
                   "calls": "sa_build, lcp_build" if args.separate else "sa_lcp_build",
                   "genome_bp": N - 1, "seed": args.seed, "parallelism": f"replicas{world}",
                   "l2": "working set >> L2 (no flush needed)",
                   "rounds": trace["rounds"], "graph_rounds": trace.get("graph_rounds", 0),
                   "finished_direct": trace["finished_direct"],
                   "active_per_round": trace["active"], "sa_only_ms": sa_only_ms,
                   "autotuned": tuned, "builder": args.builder,
                   **({"dc3_levels": trace["rounds"]} if args.builder == "dc3" else {}),
                   **({"reads": reads_info} if reads_info else {})},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": ({"value": N * world / (e2e["ms"] / 1000.0) / 1e6, "unit": UNIT,
                 "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                 "ms_per_step": e2e["ms"], "calls": e2e["calls"]} if e2e else None),
        "gpu_launches": launches,
        "clocks": clk,
        "kernels": breakdown,
    }
    print(json.dumps(line), flush=True)
    rank_teardown(world)
    return 0


if __name__ == "__main__":
    sys.exit(main())
