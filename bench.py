"""Benchmark: all-neighbour self-search of 1,000,000 synthetic CDR3 sequences
at Levenshtein distance <= 2 (Appendix A, XTNeighbor steps 0-7) on one GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

A step is one xtn_search_self call over the resident 1M-sequence input
(encode, expand, sort, group, emit, pair sort, dedup + verify, count readback).
`value` is verified pairs per second with inputs already in HBM; `e2e` is the
same metric through the C ABI with pinned host buffers (host->device copy of
the sequences and device->host copy of the result rows inside every step).
Under torchrun each rank runs an independent replica (the search has no
exchange step on one GPU), the slowest rank's time is used and `value` counts
the pairs of all ranks.  `--impl reference` times the CPU oracle instead, on
every host core, on a bounded prefix of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import cdr3_synth as gen  # noqa: E402

WORKLOAD = gen.SELF_1M
METRIC = "1M-seq d≤2 all-neighbour search time (s), verified pairs/s; query p50/p99 ms"
UNIT = "verified pairs/s"
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE_N = 100_000
ROOFLINE_KERNEL = "k_onesweep_records"
ROOFLINE_SOURCE = os.path.join(ROOT, "paper_2403_09010_gb300", "csrc", "k_radix.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_onesweep_records_traffic.txt")


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce(x: float, op: str) -> float:
    """x reduced over the ranks ("max" or "sum"); x itself in one process.
    NCCL reduces on the device, gloo on the host."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(units: float, seconds: float) -> float:
    """Whole-job rate of independent replicas: the units of all ranks over
    the slowest rank's time."""
    return _reduce(units, "sum") / _reduce(seconds, "max")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic_per_record():
    """DRAM bytes per sorted record from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    kv = dict(l.split("=", 1) for l in text.splitlines() if "=" in l and not l.startswith("#"))
    src_hash = hashlib.sha256(open(ROOFLINE_SOURCE, "rb").read()).hexdigest()[:16]
    if kv.get("source_sha256_16", "").strip() != src_hash:
        return None
    try:
        return float(kv["dram_bytes_per_record"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi samples (SM clock, throttle reasons) while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_oracle_arm(args):
    """--impl reference: the CPU oracle, as it stands, on every host core (its
    variant keys split over threads by hash), each step a bounded prefix of
    the same workload sized so that warm-up plus timed steps take about three
    minutes."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    seqs, off = gen.workload(WORKLOAD)
    cores = os.cpu_count() or 1
    probe = 20_000
    t0 = time.perf_counter()
    oracle.symdel_self_sharded(seqs[: off[probe]], off[: probe + 1], WORKLOAD.d, threads=cores)
    per_seq = max((time.perf_counter() - t0) / probe, 1e-8)
    budget = 170.0 / max(1, args.steps + args.warmup)
    n_s = int(min(WORKLOAD.n, max(probe, budget / per_seq)))
    s_seqs, s_off = seqs[: off[n_s]], off[: n_s + 1]
    for _ in range(args.warmup):
        oracle.symdel_self_sharded(s_seqs, s_off, WORKLOAD.d, threads=cores)
    times, pairs = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rows = oracle.symdel_self_sharded(s_seqs, s_off, WORKLOAD.d, threads=cores)
        times.append(time.perf_counter() - t0)
        pairs = rows.shape[0]
    total = sum(times)
    value = pairs * args.steps / total
    sample = (f"first {n_s:,} sequences of the {WORKLOAD.n:,}-sequence d={WORKLOAD.d} workload, "
              f"{cores} threads, {pairs:,} pairs per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD.name, "n": WORKLOAD.n, "d": WORKLOAD.d,
                   "sample_n": n_s, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle, keys partitioned by hash over threads",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def cpu_baseline():
    """The oracle on every host core (variant keys split over threads by
    hash) on the whole benchmarked workload: all 1,000,000 sequences."""
    import oracle
    oracle.build()
    seqs, off = gen.workload(WORKLOAD)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    rows = oracle.symdel_self_sharded(seqs, off, WORKLOAD.d, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": rows.shape[0] / dt, "unit": UNIT, "cores": cores,
            "kind": "oracle, keys partitioned by hash over threads",
            "sample": f"the whole {WORKLOAD.n:,}-sequence d={WORKLOAD.d} workload (n = "
                      f"{off.size - 1:,}), {cores} threads, {dt:.1f} s, "
                      f"{rows.shape[0]:,} pairs", "seconds": dt, "pairs": int(rows.shape[0])}


def cpu_single_thread_prefix():
    """The single-thread oracle on the first 100,000 sequences: a labelled
    extra beside the all-core baseline (pairs grow faster than the work with
    the prefix length, so this rate is not the rate on the whole workload)."""
    import oracle
    oracle.build()
    seqs, off = gen.workload(WORKLOAD, CPU_SAMPLE_N)
    t0 = time.perf_counter()
    rows = oracle.symdel_self(seqs, off, WORKLOAD.d)
    dt = time.perf_counter() - t0
    return {"value": rows.shape[0] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {CPU_SAMPLE_N:,} sequences of the {WORKLOAD.n:,}-sequence "
                      f"d={WORKLOAD.d} workload, single thread, {dt:.1f} s, "
                      f"{rows.shape[0]:,} pairs"}


def _events_ms(fn, reps, stream):
    import torch
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return float(np.median(times))


def run_batched(reps: int = 5):
    """256 repertoires (log-uniform sizes 1e3..2e5), d=2: one autotuned plan
    replayed as a CUDA graph vs one xtn_search_self call per repertoire."""
    import torch
    import paper_2403_09010_gb300 as xtn
    from paper_2403_09010_gb300 import autotune
    seqs, off, rep = gen.batched()
    ds = torch.from_numpy(seqs).cuda()
    do = torch.from_numpy(off).cuda()
    tuned = autotune.tune(ds, off, gen.BATCH_D, rep_offsets=rep, use_cache=False)
    plan = xtn.Plan(off, gen.BATCH_D, rep_offsets=rep, tuning=tuned)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        plan.run(ds)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            plan.run(ds)
        graph_ms = _events_ms(g.replay, reps, stream)
        rows = plan.result(like=ds)
        eager_ms = _events_ms(lambda: plan.run(ds), reps, stream)
    stats = plan.stats()
    # the plain path: one call per repertoire on the same resident data
    rep_rows = []

    def per_rep():
        rep_rows.clear()
        for r in range(rep.size - 1):
            a, b = int(rep[r]), int(rep[r + 1])
            o = do[a:b + 1] - do[a]
            part = xtn.search_self(ds[int(off[a]):int(off[b])], o, gen.BATCH_D)
            rep_rows.append((a, part))
    cur = torch.cuda.current_stream()
    per_rep()
    per_rep_ms = _events_ms(per_rep, max(1, reps // 2), cur)
    merged = torch.cat([p + torch.tensor([a, a, 0], dtype=torch.int32, device=p.device)
                        for a, p in rep_rows])
    identical = bool(torch.equal(merged, rows))
    plan.free()
    return {"workload": "batched_256reps_d2", "n": int(off.size - 1), "repertoires": int(rep.size - 1),
            "graph_ms": graph_ms, "plan_eager_ms": eager_ms, "per_repertoire_ms": per_rep_ms,
            "speedup_vs_per_repertoire": per_rep_ms / graph_ms, "pairs": int(rows.shape[0]),
            "identical_output": identical, "autotune": tuned, "counts": stats}


def run_served(speed: float = 1.0):
    """10M-sequence resident index (d=2), 2,000 requests of 1..10,000 queries
    arriving as a Poisson process at 200/s: continuous batching vs a plain
    one-request-at-a-time queue on the same arrivals."""
    import torch
    import paper_2403_09010_gb300 as xtn
    from paper_2403_09010_gb300 import serve
    rs, ro, reqs = gen.served()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx = xtn.index_build(rs, ro, 2)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = idx.info()
    out = {"workload": "served_ref1e7_2000req_d2", "index_build_s": build_s,
           "index_records": info["n_records"], "index_device_bytes": info["device_bytes"]}
    # warm the query path; every server also warms its streams with the
    # largest request before the replay starts
    xtn.search_query(idx, reqs[0].seqs, reqs[0].offsets)
    big = max(reqs, key=lambda r: r.offsets.size)
    # the nominal arrival rate, then the same requests arriving 4x and 16x
    # faster, and all at once (capacity): continuous batching vs a plain queue
    ref_rows = None
    identical = True
    # One pause of the process can set a replay's p99, so every rate is
    # replayed five times (all at once: three) and the run with the median
    # p99 is reported, with every run's p50 and p99 beside it.
    for label, sp, reps in [("rate_200", speed, 5), ("rate_800", 4 * speed, 5),
                            ("rate_3200", 16 * speed, 5), ("all_at_once", 1e9, 3)]:
        res = {}
        for name, kw in [("continuous", dict(slots=4)),
                         ("plain_queue", dict(slots=1, max_batch_queries=1))]:
            runs = []
            for _ in range(reps):
                srv = serve.Server(idx, **kw)
                srv.warm(big.seqs, big.offsets)
                pend = serve.replay(srv, reqs, speed=sp)
                srv.close()
                runs.append(srv.stats(pend))
                rows = [p.rows for p in pend]
                if ref_rows is None:
                    ref_rows = rows
                else:
                    identical &= all(np.array_equal(a, b) for a, b in zip(rows, ref_rows))
            runs.sort(key=lambda r: r["p99_ms"])
            res[name] = dict(runs[len(runs) // 2], replays=reps,
                             p99_ms_runs=[r["p99_ms"] for r in runs],
                             p50_ms_runs=sorted(r["p50_ms"] for r in runs))
        out[label] = res
    out["identical_output"] = bool(identical)
    idx.free()
    return out


def run_tcrdist(reps: int = 10):
    """TCRdist post-filter (score <= 24) of the d=2 neighbours of 1M sequences."""
    import torch
    import paper_2403_09010_gb300 as xtn
    seqs, off = gen.workload(gen.TCRDIST_1M)
    ds, do = torch.from_numpy(seqs).cuda(), torch.from_numpy(off).cuda()
    cur = torch.cuda.current_stream()
    rows = xtn.search_self(ds, do, 2)
    kept = xtn.tcrdist_filter(ds, do, rows, 24)
    search_ms = _events_ms(lambda: xtn.search_self(ds, do, 2), reps, cur)
    filter_ms = _events_ms(lambda: xtn.tcrdist_filter(ds, do, rows, 24), reps, cur)
    return {"workload": "tcrdist_n1e6_d2_score24", "lev2_pairs": int(rows.shape[0]),
            "kept_pairs": int(kept.shape[0]), "search_ms": search_ms, "filter_ms": filter_ms}


def run_retention(n_sub: int = 5000, thresholds=(12, 18, 24, 30, 36)):
    """TCRdist retention of the SymDel prefilter (the paper's TCRdist figure,
    panel B) on the first n_sub sequences: of the pairs within each TCRdist
    threshold (every pair filtered by the library's TCRdist kernel), the
    share that SymDel(d) + filter keeps, for d = 2 and 3; and the time of the
    exhaustive filter against SymDel(d) + filter (panel A)."""
    import torch
    import paper_2403_09010_gb300 as xtn
    seqs, off = gen.workload(gen.TCRDIST_1M, n_sub)
    ds, do = torch.from_numpy(seqs).cuda(), torch.from_numpy(off).cuda()
    cur = torch.cuda.current_stream()
    ii, jj = np.triu_indices(n_sub, 1)
    every = torch.from_numpy(np.stack([ii, jj, np.zeros_like(ii)], 1).astype(np.int32)).cuda()
    lev = {d: xtn.search_self(ds, do, d) for d in (2, 3)}
    curve = []
    for t in thresholds:
        exh = int(xtn.tcrdist_filter(ds, do, every, t).shape[0])
        row = {"tcrdist_max": t, "exhaustive_pairs": exh}
        for d in (2, 3):
            kept = int(xtn.tcrdist_filter(ds, do, lev[d], t).shape[0])
            row[f"kept_d{d}"] = kept
            row[f"retention_d{d}"] = kept / exh if exh else None
        curve.append(row)
    t = 24
    exh_ms = _events_ms(lambda: xtn.tcrdist_filter(ds, do, every, t), 5, cur)
    sym_ms = {f"symdel_d{d}_plus_filter_ms": _events_ms(
        lambda d=d: xtn.tcrdist_filter(ds, do, xtn.search_self(ds, do, d), t), 5, cur)
        for d in (2, 3)}
    return {"workload": f"tcrdist_retention_n{n_sub}", "all_pairs": int(ii.size),
            "curve": curve, "exhaustive_filter_ms": exh_ms, **sym_ms}


def run_d3(reps: int = 3):
    """The 1M search at d <= 3 (about 560 deletion subsets per sequence)."""
    import torch
    import paper_2403_09010_gb300 as xtn
    seqs, off = gen.workload(WORKLOAD)
    ds, do = torch.from_numpy(seqs).cuda(), torch.from_numpy(off).cuda()
    cur = torch.cuda.current_stream()
    rows = xtn.search_self(ds, do, 3)
    ms = _events_ms(lambda: xtn.search_self(ds, do, 3), reps, cur)
    return {"workload": "selfsearch_n1e6_d3", "verified_pairs": int(rows.shape[0]),
            "search_ms": ms, "pairs_per_s": rows.shape[0] / (ms / 1e3)}


def run_hamming(reps: int = 10):
    """The Hamming variant (same candidates, Hamming filter) of the 1M d<=2
    self-search: time per search and pairs, next to the Levenshtein search."""
    import torch
    import paper_2403_09010_gb300 as xtn
    seqs, off = gen.workload(WORKLOAD)
    ds, do = torch.from_numpy(seqs).cuda(), torch.from_numpy(off).cuda()
    cur = torch.cuda.current_stream()
    ham = xtn.search_self(ds, do, 2, metric="hamming")
    ms = _events_ms(lambda: xtn.search_self(ds, do, 2, metric="hamming"), reps, cur)
    return {"workload": "selfsearch_n1e6_d2_hamming", "hamming_pairs": int(ham.shape[0]),
            "search_ms": ms, "pairs_per_s": ham.shape[0] / (ms / 1e3)}


def run_between(reps: int = 10, n_rep: int = 8):
    """Repertoire overlap: the 1M set as eight repertoires of equal size, the
    pairs between different repertoires at d<=2 (Levenshtein and Hamming)."""
    import torch
    import paper_2403_09010_gb300 as xtn
    seqs, off = gen.workload(WORKLOAD)
    n = off.size - 1
    rep = (np.arange(n_rep + 1, dtype=np.int64) * n) // n_rep
    ds, do = torch.from_numpy(seqs).cuda(), torch.from_numpy(off).cuda()
    cur = torch.cuda.current_stream()
    out = {"workload": f"between_n1e6_{n_rep}reps_d2"}
    for metric in ("levenshtein", "hamming"):
        rows = xtn.search_between(ds, do, 2, rep, metric=metric)
        ms = _events_ms(lambda: xtn.search_between(ds, do, 2, rep, metric=metric), reps, cur)
        out[metric] = {"pairs": int(rows.shape[0]), "search_ms": ms}
    return out


def run_paired(reps: int = 5, n: int = 1_000_000):
    """Paired chains (alpha + token + beta, the token never edited), d<=2:
    1M synthetic receptors, time per search and pairs."""
    import torch
    import paper_2403_09010_gb300 as xtn
    a, ao, b, bo = gen.paired(n, 6)
    da, dao = torch.from_numpy(a).cuda(), torch.from_numpy(ao).cuda()
    db, dbo = torch.from_numpy(b).cuda(), torch.from_numpy(bo).cuda()
    cur = torch.cuda.current_stream()
    rows = xtn.search_paired(da, dao, db, dbo, 2)
    ms = _events_ms(lambda: xtn.search_paired(da, dao, db, dbo, 2), reps, cur)
    La, Lb = np.diff(ao), np.diff(bo)
    return {"workload": "paired_n1e6_d2", "receptors": n,
            "mean_len_alpha": float(La.mean()), "mean_len_beta": float(Lb.mean()),
            "pairs": int(rows.shape[0]), "search_ms": ms,
            "pairs_per_s": rows.shape[0] / (ms / 1e3)}


def run_streaming(reps: int = 3):
    """Searches in passes over fingerprint bins: the 1M d<=2 search forced into
    four passes (against its one-pass time), and 9M sequences at d<=3 (about
    5e9 variant records, past what one pass indexes) with the default budget."""
    import torch
    import paper_2403_09010_gb300 as xtn
    cur = torch.cuda.current_stream()
    seqs, off = gen.workload(WORKLOAD)
    ds, do = torch.from_numpy(seqs).cuda(), torch.from_numpy(off).cuda()
    out = {}
    rows, passes = xtn.search_self_streaming(ds, do, 2, max_pass_records=30_000_000)
    ms = _events_ms(lambda: xtn.search_self_streaming(ds, do, 2, max_pass_records=30_000_000),
                    reps, cur)
    out["n1e6_d2_4passes"] = {"passes": passes, "pairs": int(rows.shape[0]), "search_ms": ms}
    n = 9_000_000
    seqs, off = gen.generate(n, 17, 0.15, 0.01)
    ds, do = torch.from_numpy(seqs).cuda(), torch.from_numpy(off).cuda()
    L = np.diff(off).astype(np.int64)
    subsets = int((1 + L + L * (L - 1) // 2 + L * (L - 1) * (L - 2) // 6).sum())
    rows, passes = xtn.search_self_streaming(ds, do, 3)
    ms = _events_ms(lambda: xtn.search_self_streaming(ds, do, 3), reps, cur)
    out["n9e6_d3"] = {"passes": passes, "deletion_subsets": subsets, "pairs": int(rows.shape[0]),
                      "search_ms": ms, "pairs_per_s": rows.shape[0] / (ms / 1e3)}
    del ds, do
    xtn.scratch_trim()
    return out


def run_profile_case(args):
    """Small cases of the query search (a resident index of n reference
    sequences, default 2,000,000, and one request of 20,000 queries, half of
    them one-deletion mutants of reference entries), of the TCRdist filter (the d<=2 rows of the
    first n sequences of the TCRdist workload, default 1,000,000) and of the
    paired-chain search (n receptors, default 400,000), run warm-up plus
    `steps` times; for ncu captures of their kernels."""
    import torch
    import paper_2403_09010_gb300 as xtn
    xtn.build()
    cur = torch.cuda.current_stream()
    if args.case == "query":
        rs, ro = gen.generate(args.n or 2_000_000, 41, 0.15, 0.01)
        qs, qo = gen.generate(10_000, 42, 0.0, 0.0)
        strs = gen.to_strings(rs[: ro[10_000]], ro[: 10_001])
        rng = np.random.default_rng(43)
        mut = [s[:k] + s[k + 1:] for s, k in zip(strs, rng.integers(0, 8, len(strs)))]
        qs, qo = gen.from_strings(gen.to_strings(qs, qo) + mut)
        idx = xtn.index_build(rs, ro, 2)
        dq, dqo = torch.from_numpy(qs).cuda(), torch.from_numpy(qo).cuda()
        rows = xtn.search_query(idx, dq, dqo)
        ms_q = _events_ms(lambda: xtn.search_query(idx, dq, dqo),
                          args.warmup + args.steps, cur)
        out = {"case": "query", "ref_n": int(ro.size - 1), "queries": int(qo.size - 1),
               "rows": int(rows.shape[0]), "search_ms": ms_q}
        idx.free()
    elif args.case == "paired":
        a, ao, b, bo = gen.paired(args.n or 400_000, 6)
        da, dao = torch.from_numpy(a).cuda(), torch.from_numpy(ao).cuda()
        db, dbo = torch.from_numpy(b).cuda(), torch.from_numpy(bo).cuda()
        rows = xtn.search_paired(da, dao, db, dbo, 2)
        ms_p = _events_ms(lambda: xtn.search_paired(da, dao, db, dbo, 2),
                          args.warmup + args.steps, cur)
        out = {"case": "paired", "receptors": int(ao.size - 1), "rows": int(rows.shape[0]),
               "search_ms": ms_p}
    else:
        seqs, off = gen.workload(gen.TCRDIST_1M, args.n)
        ds, do = torch.from_numpy(seqs).cuda(), torch.from_numpy(off).cuda()
        rows = xtn.search_self(ds, do, 2)
        ms_f = _events_ms(lambda: xtn.tcrdist_filter(ds, do, rows, 24),
                          args.warmup + args.steps, cur)
        out = {"case": "tcrdist", "n": int(off.size - 1), "rows": int(rows.shape[0]),
               "filter_ms": ms_f}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="xtn", choices=["xtn", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched / served / TCRdist / Hamming / overlap / "
                         "streaming side measurements")
    ap.add_argument("--n", type=int, default=None,
                    help="use only the first n sequences (small cases for profiling)")
    ap.add_argument("--case", default="self", choices=["self", "query", "tcrdist", "paired"],
                    help="query / tcrdist / paired: a small case of the query search, the "
                         "TCRdist filter or the paired-chain search (default 400,000 "
                         "receptors), for profiling (prints one JSON line of timings)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_oracle_arm(args)
    if args.case != "self":
        return run_profile_case(args)

    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2403_09010_gb300 as xtn
    from paper_2403_09010_gb300 import native
    xtn.build()
    lib = native.lib()

    seqs, off = gen.workload(WORKLOAD, args.n)
    n = off.size - 1
    d_seqs = torch.from_numpy(seqs).cuda()
    d_off = torch.from_numpy(off).cuda()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(d_seqs.data_ptr())
    op = ctypes.c_void_p(d_off.data_ptr())
    st = ctypes.c_void_p(stream.cuda_stream)
    n_out = ctypes.c_int64(0)

    # size the output once (a user would keep this buffer too)
    rc = lib.xtn_search_self(sp, op, n, WORKLOAD.d, None, 0, None, 0, ctypes.byref(n_out), st)
    assert rc in (0, native.XTN_ERR_BUFFER_TOO_SMALL), native.status_string(rc)
    cap = int(n_out.value * 1.1) + 1024
    out = torch.empty((cap, 3), dtype=torch.int32, device="cuda")
    outp = ctypes.c_void_p(out.data_ptr())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step():
        r = lib.xtn_search_self(sp, op, n, WORKLOAD.d, None, 0, outp, cap, ctypes.byref(n_out), st)
        if r != 0:
            raise native.XtnError(r, "xtn_search_self")
        return n_out.value

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # the timed region: events bracket only the dominant kernel's launches
    # (two event records per launch would otherwise add ~2% to the step)
    xtn.profile_report()          # clear
    xtn.profile_only(ROOFLINE_KERNEL)
    xtn.profile_enable(True)
    pairs = 0
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k)                       # L2 flush outside the timed events
            ev[k][0].record(stream)
            pairs = step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    xtn.profile_enable(False)
    xtn.profile_only(None)
    prof_main = {k: v for k, v in xtn.profile_report().items() if not k.startswith("host_")}
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1000.0
    value = replica_throughput(pairs * args.steps, total_s)
    total_s = _reduce(total_s, "max")
    if world > 1:
        torch.distributed.barrier()

    # the same steps again with every launch bracketed: the per-kernel table
    xtn.profile_enable(True)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k)
        step()
    torch.cuda.synchronize()
    xtn.profile_enable(False)
    prof = xtn.profile_report()
    # host-side spans (whole calls, scratch allocations, stream waits) apart
    host = {k: v for k, v in prof.items() if k.startswith("host_")}
    prof = {k: v for k, v in prof.items() if not k.startswith("host_")}
    launches = sum(v[0] for v in prof.values())

    # end to end through the C ABI with pinned host buffers
    h_seqs = torch.from_numpy(seqs).pin_memory()
    h_off = torch.from_numpy(off).pin_memory()
    h_out = torch.empty((cap, 3), dtype=torch.int32).pin_memory()
    hsp, hop, hout = (ctypes.c_void_p(t.data_ptr()) for t in (h_seqs, h_off, h_out))
    e2e_steps = max(3, min(args.steps, 20))
    lib.xtn_search_self(hsp, hop, n, WORKLOAD.d, None, 0, hout, cap, ctypes.byref(n_out), st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = lib.xtn_search_self(hsp, hop, n, WORKLOAD.d, None, 0, hout, cap,
                                 ctypes.byref(n_out), st)
        assert rc == 0, native.status_string(rc)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = replica_throughput(pairs, e2e_s)
    e2e_s = _reduce(e2e_s, "max")

    # roofline of the dominant kernel, from the timed region
    peak, peak_kind = _peaks()
    top = (ROOFLINE_KERNEL, prof_main[ROOFLINE_KERNEL]) if ROOFLINE_KERNEL in prof_main else None
    roofline = None
    if top:
        name, (nl, ms, nbytes) = top
        achieved = nbytes / (ms / 1000.0) / 1e9
        tpr = _traffic_per_record() if name == ROOFLINE_KERNEL else None
        n_rec_per_launch = nbytes / nl / 16.0 if name == ROOFLINE_KERNEL else None
        roofline = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": (tpr * n_rec_per_launch) if tpr and n_rec_per_launch else None,
                    "algorithmic_bytes_per_launch": nbytes / nl,
                    "launches_in_timed_region": nl, "avg_launch_ms": ms / nl}
    kernels = {k: {"launches": v[0], "ms": v[1],
                   "GBps": (v[2] / (v[1] / 1e3) / 1e9) if v[1] else None,
                   "frac": (v[2] / (v[1] / 1e3) / 1e9 / peak) if v[1] else None,
                   "share": v[1] / sum(x[1] for x in prof.values())} for k, v in prof.items()}

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": (WORKLOAD.name if args.n is None
                                else f"prefix_n{n}_of_{WORKLOAD.name}"),
                   "n": n, "d": WORKLOAD.d,
                   "mean_len": float(np.diff(off).mean()),
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": f"replicas x{world}"},
        "search_time_s": total_s / args.steps,
        "verified_pairs": pairs,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(seqs.nbytes + off.nbytes),
                "d2h_bytes_per_step": int(pairs * 12), "search_time_s": e2e_s},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "kernels": kernels,
        "host_per_step": {k: {"count": v[0] / args.steps, "ms": v[1] / args.steps}
                          for k, v in host.items()},
        "clocks": clk.summary(),
    }
    if not args.no_extras and world == 1 and args.n is None:
        line["batched"] = run_batched()
        line["served"] = run_served()
        line["tcrdist"] = run_tcrdist()
        line["hamming"] = run_hamming()
        line["tcrdist_retention"] = run_retention()
        line["d3"] = run_d3()
        line["between"] = run_between()
        line["streaming"] = run_streaming()
        line["paired"] = run_paired()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_single_thread_prefix"] = cpu_single_thread_prefix()
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
