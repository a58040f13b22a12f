"""Autotuner for the planned (batched) self-search.

Picks, by timing on the caller's own data, how records are grouped (global
radix passes on the top bits plus a shared-memory bucket pass, or global
passes on every bit plus a flag pass), where the record sort's digit counts
are taken (in the expand kernel, or one pass ahead in each sort pass),
the tile configuration of each radix sort (variant records and verified
pairs; see xtn_tune_set) and a
candidate-pair capacity for the plan (measured candidates x 1.25, so a plan
holds no more pair memory than it needs).  The pipeline splits large buckets
of shared variants at the granularity of its emit tiles whatever their size,
so there is no bucket-split threshold to tune.  Results are cached as JSON,
keyed by GPU name, workload size and d.  The process-wide knobs are put
back as they were when tuning ends: pass the result to ``xtn.Plan(...,
tuning=r)`` to build a plan with it.
"""
from __future__ import annotations

import json
import os

from . import native, xtn


def _cache_file():
    return os.environ.get("XTN_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "xtn_tune.json"))


def _key(n, n_rep, d):
    try:
        import torch
        gpu = torch.cuda.get_device_name()
    except Exception:
        gpu = "unknown"
    return f"{gpu}|n={n}|reps={n_rep}|d={d}"


def tune(seqs_dev, offsets, d: int, rep_offsets=None, configs=None, repeats: int = 2,
         use_cache: bool = True) -> dict:
    """Time every sort configuration on this workload and return the fastest:
    {"grouping", "record_hist", "records_cfg", "pairs_cfg", "pair_capacity",
    "sort_ms": {...}}.  The knobs hold their previous values afterwards."""
    n = int(offsets.shape[0]) - 1
    n_rep = 0 if rep_offsets is None else int(rep_offsets.shape[0]) - 1
    key = _key(n, n_rep, d)
    path = _cache_file()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        return cache[key]
    current = {name: xtn.tune_get(knob) for name, knob in xtn._TUNING_KNOBS}
    with xtn.tuning_applied(current):  # puts them back when tuning ends
        r = _tune(seqs_dev, offsets, d, rep_offsets, configs, repeats)
    if use_cache:
        cache[key] = r
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            json.dump(cache, open(path, "w"), indent=1)
        except OSError:
            pass
    return r


def _tune(seqs_dev, offsets, d, rep_offsets, configs, repeats):
    import torch
    R, P, H, GR = (native.XTN_TUNE_SORT_RECORDS, native.XTN_TUNE_SORT_PAIRS,
                   native.XTN_TUNE_RECORD_HISTOGRAM, native.XTN_TUNE_GROUPING)
    # the grouping stage: expand, record sort passes, bucket or flag pass
    group_kernels = ("k_expand", "k_onesweep_records", "k_bucket_group", "k_group_flags")
    configs = list(range(xtn.tune_count(R))) if configs is None else list(configs)

    def measure(*kernels):
        plan = xtn.Plan(offsets, d, rep_offsets=rep_offsets)
        plan.run(seqs_dev)                       # warm-up
        torch.cuda.synchronize()
        xtn.profile_report()
        xtn.profile_enable(True)
        for _ in range(repeats):
            plan.run(seqs_dev)
        torch.cuda.synchronize()
        xtn.profile_enable(False)
        prof = xtn.profile_report()
        stats = plan.stats()
        plan.free()
        # kernels a mode does not launch count as zero time
        ms = sum(prof[k][1] for k in kernels if k in prof)
        if not any(k in prof for k in kernels):
            ms = float("inf")
        return ms / repeats, stats

    group_ms = {}
    for gm in (0, 1):  # mode 2 only shrinks the shared-memory segments
        xtn.tune_set(GR, gm)
        group_ms[gm], _ = measure(*group_kernels)
    best_g = min(group_ms, key=group_ms.get)
    xtn.tune_set(GR, best_g)
    hist_ms = {}
    for h in range(xtn.tune_count(H)):
        xtn.tune_set(H, h)
        hist_ms[h], _ = measure(*group_kernels)
    best_h = min(hist_ms, key=hist_ms.get)
    xtn.tune_set(H, best_h)
    rec_ms, pair_ms = {}, {}
    cands = 0
    for c in configs:
        xtn.tune_set(R, c)
        rec_ms[c], st = measure("k_onesweep_records")
        cands = max(cands, st["candidates"])
    best_r = min(rec_ms, key=rec_ms.get)
    xtn.tune_set(R, best_r)
    for c in configs:
        xtn.tune_set(P, c)
        pair_ms[c], _ = measure("k_onesweep_pairs")
    best_p = min(pair_ms, key=pair_ms.get)
    xtn.tune_set(P, best_p)
    return {"grouping": best_g, "record_hist": best_h, "records_cfg": best_r,
            "pairs_cfg": best_p, "pair_capacity": max(65536, int(cands * 1.25)),
            "sort_ms": {"records": rec_ms[best_r], "pairs": pair_ms[best_p]}}
