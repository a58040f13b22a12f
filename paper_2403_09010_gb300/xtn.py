"""Python entry points with the names of the C ABI (include/xtn.h).

Inputs may be numpy arrays (host) or CUDA ``torch.Tensor`` s (device); the
library copies host data itself.  Results come back on the side the sequences
came from: a ``(rows, 3)`` numpy ``uint32`` array for host input, a
``(rows, 3)`` ``torch.int32`` CUDA tensor for device input (columns i, j,
dist; indices < 2^31 in every supported workload).  Device work runs on the
current torch stream of the input's device.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native
from .native import XtnError, check

_ROW = 3


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=None):
    """(pointer, keep-alive object, on_device) for a numpy array or torch tensor."""
    if x is None:
        return None, None, False
    if _is_torch(x):
        if not x.is_contiguous():
            x = x.contiguous()
        return ctypes.c_void_p(x.data_ptr()), x, bool(x.is_cuda)
    a = np.ascontiguousarray(x, dtype=dtype)
    if a.size == 0:
        a = np.zeros(1, dtype=dtype or a.dtype)
    return a.ctypes.data_as(ctypes.c_void_p), a, False


def _stream(x):
    if x is not None and _is_torch(x) and x.is_cuda:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return ctypes.c_void_p(0)


def _alloc_rows(cap: int, like):
    cap = max(int(cap), 1)
    if like is not None and _is_torch(like) and like.is_cuda:
        import torch
        t = torch.empty((cap, _ROW), dtype=torch.int32, device=like.device)
        return t, ctypes.c_void_p(t.data_ptr())
    a = np.empty((cap, _ROW), dtype=np.uint32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _n_items(offsets) -> int:
    return int(offsets.shape[0]) - 1


def _call_with_rows(fn, cap, like, where):
    """fn(out_ptr, cap, n_out_ref) -> status; grows the buffer once if needed."""
    n_out = ctypes.c_int64(0)
    out, optr = _alloc_rows(cap, like)
    rc = fn(optr, max(int(cap), 1), ctypes.byref(n_out))
    if rc == native.XTN_ERR_BUFFER_TOO_SMALL:
        out, optr = _alloc_rows(n_out.value, like)
        rc = fn(optr, max(n_out.value, 1), ctypes.byref(n_out))
    check(rc, where)
    return out[: n_out.value]


_METRICS = {"levenshtein": 0, "hamming": 1}


def search_self(seqs, offsets, d: int, rep_offsets=None, cap: int | None = None,
                metric: str = "levenshtein"):
    """All pairs (i < j) within distance d; see xtn_search_self.  metric
    "hamming" calls xtn_search_self_hamming (equal lengths, substitutions)."""
    if metric not in ("levenshtein", "hamming"):
        raise ValueError(f"unknown metric {metric!r}")
    entry = "xtn_search_self_hamming" if metric == "hamming" else "xtn_search_self"
    n = _n_items(offsets)
    sp, sk, _ = _ptr(seqs, np.uint8)
    op, ok, _ = _ptr(offsets, np.int64)
    rp, rk, _ = _ptr(rep_offsets, np.int64)
    n_rep = 0 if rep_offsets is None else int(rep_offsets.shape[0]) - 1
    stream = _stream(seqs)
    if cap is None:
        cap = 4 * n + 4096

    def fn(optr, c, nref):
        return getattr(native.lib(), entry)(sp, op, n, int(d), rp, n_rep, optr, c, nref, stream)

    return _call_with_rows(fn, cap, seqs, entry)


def search_paired(a_seqs, a_offsets, b_seqs, b_offsets, d: int, cap: int | None = None):
    """All receptor pairs (i < j) whose chains are within d edits in all:
    Lev(alpha_i, alpha_j) + Lev(beta_i, beta_j) <= d; see xtn_search_paired."""
    n = _n_items(a_offsets)
    if _n_items(b_offsets) != n:
        raise ValueError("both chains need one offset per receptor")
    ap, ak, _ = _ptr(a_seqs, np.uint8)
    aop, aok, _ = _ptr(a_offsets, np.int64)
    bp, bk, _ = _ptr(b_seqs, np.uint8)
    bop, bok, _ = _ptr(b_offsets, np.int64)
    stream = _stream(a_seqs)
    if cap is None:
        cap = 4 * n + 4096

    def fn(optr, c, nref):
        return native.lib().xtn_search_paired(ap, aop, bp, bop, n, int(d), optr, c, nref, stream)

    return _call_with_rows(fn, cap, a_seqs, "xtn_search_paired")


def search_between(seqs, offsets, d: int, rep_offsets, cap: int | None = None,
                   metric: str = "levenshtein"):
    """All pairs (i < j) within distance d whose sequences lie in different
    repertoires; see xtn_search_between."""
    if metric not in _METRICS:
        raise ValueError(f"unknown metric {metric!r}")
    if rep_offsets is None:
        raise ValueError("search_between needs rep_offsets")
    n = _n_items(offsets)
    sp, sk, _ = _ptr(seqs, np.uint8)
    op, ok, _ = _ptr(offsets, np.int64)
    rp, rk, _ = _ptr(rep_offsets, np.int64)
    n_rep = int(rep_offsets.shape[0]) - 1
    stream = _stream(seqs)
    if cap is None:
        cap = 4 * n + 4096

    def fn(optr, c, nref):
        return native.lib().xtn_search_between(sp, op, n, int(d), rp, n_rep, _METRICS[metric],
                                               optr, c, nref, stream)

    return _call_with_rows(fn, cap, seqs, "xtn_search_between")


def search_self_streaming(seqs, offsets, d: int, rep_offsets=None, metric: str = "levenshtein",
                          between: bool = False, max_pass_records: int = 0,
                          cap: int | None = None):
    """The self-search in passes over fingerprint bins (xtn_search_self_streaming).
    Returns (rows, passes run)."""
    if metric not in _METRICS:
        raise ValueError(f"unknown metric {metric!r}")
    if between and rep_offsets is None:
        raise ValueError("between needs rep_offsets")
    n = _n_items(offsets)
    sp, sk, _ = _ptr(seqs, np.uint8)
    op, ok, _ = _ptr(offsets, np.int64)
    rp, rk, _ = _ptr(rep_offsets, np.int64)
    n_rep = 0 if rep_offsets is None else int(rep_offsets.shape[0]) - 1
    stream = _stream(seqs)
    if cap is None:
        cap = 4 * n + 4096
    passes = ctypes.c_int64(0)

    def fn(optr, c, nref):
        return native.lib().xtn_search_self_streaming(
            sp, op, n, int(d), rp, n_rep, _METRICS[metric], int(bool(between)),
            int(max_pass_records), optr, c, nref, ctypes.byref(passes), stream)

    rows = _call_with_rows(fn, cap, seqs, "xtn_search_self_streaming")
    return rows, int(passes.value)


class Index:
    """Device-resident deletion-variant index of a reference set."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self):
        n, nr, nb = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        d = ctypes.c_int(0)
        check(native.lib().xtn_index_info(self._h, ctypes.byref(n), ctypes.byref(d),
                                          ctypes.byref(nr), ctypes.byref(nb)), "xtn_index_info")
        return {"n": n.value, "d": d.value, "n_records": nr.value, "device_bytes": nb.value}

    def scratch_bytes(self, q_offsets) -> int:
        """Device scratch a query search of these queries takes (an estimate for
        admission control; see xtn_search_query_scratch).  q_offsets: host."""
        o = np.ascontiguousarray(q_offsets, dtype=np.int64)
        out = ctypes.c_int64(0)
        check(native.lib().xtn_search_query_scratch(self._h, o.ctypes.data_as(ctypes.c_void_p),
                                                    o.size - 1, ctypes.byref(out)),
              "xtn_search_query_scratch")
        return int(out.value)

    def free(self):
        if self._h:
            native.lib().xtn_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


_TUNING_KNOBS = (("grouping", native.XTN_TUNE_GROUPING),
                 ("record_hist", native.XTN_TUNE_RECORD_HISTOGRAM),
                 ("records_cfg", native.XTN_TUNE_SORT_RECORDS),
                 ("pairs_cfg", native.XTN_TUNE_SORT_PAIRS))


class tuning_applied:
    """Context manager: set the knobs named in a tuning dict (keys grouping,
    record_hist, records_cfg, pairs_cfg; missing keys are left alone) and put
    the previous values back on exit."""

    def __init__(self, tuning: dict | None):
        self.tuning = tuning or {}

    def __enter__(self):
        self.saved = [(knob, tune_get(knob)) for name, knob in _TUNING_KNOBS
                      if name in self.tuning]
        for name, knob in _TUNING_KNOBS:
            if name in self.tuning:
                tune_set(knob, int(self.tuning[name]))
        return self

    def __exit__(self, *exc):
        for knob, value in self.saved:
            tune_set(knob, value)
        return False


class Plan:
    """Planned self-search (see xtn_plan_create): device memory allocated once,
    `run` only queues kernels on the current stream (CUDA-graph capturable),
    `result` waits and returns the rows of the last run.  The tuning knobs are
    read when the plan is created; `tuning` (a dict as returned by
    autotune.tune) applies to this plan only, and its pair_capacity is used
    when `pair_capacity` is 0."""

    def __init__(self, offsets, d: int, rep_offsets=None, pair_capacity: int = 0,
                 tuning: dict | None = None):
        n = _n_items(offsets)
        op, ok, _ = _ptr(offsets, np.int64)
        rp, rk, _ = _ptr(rep_offsets, np.int64)
        n_rep = 0 if rep_offsets is None else int(rep_offsets.shape[0]) - 1
        if not pair_capacity and tuning:
            pair_capacity = int(tuning.get("pair_capacity", 0))
        h = ctypes.c_void_p(0)
        with tuning_applied(tuning):
            check(native.lib().xtn_plan_create(op, n, int(d), rp, n_rep, int(pair_capacity),
                                               ctypes.byref(h)), "xtn_plan_create")
        self._h = h
        self.n = n
        self.d = int(d)

    def info(self):
        rc, pc, nb = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        check(native.lib().xtn_plan_info(self._h, ctypes.byref(rc), ctypes.byref(pc),
                                         ctypes.byref(nb)), "xtn_plan_info")
        return {"record_capacity": rc.value, "pair_capacity": pc.value, "device_bytes": nb.value}

    def stats(self, stream=None):
        """Counts of the last run: records, groups, candidates, survivors."""
        v = [ctypes.c_int64(0) for _ in range(4)]
        st = ctypes.c_void_p(stream) if stream is not None else _stream(None)
        check(native.lib().xtn_plan_stats(self._h, *[ctypes.byref(x) for x in v], st),
              "xtn_plan_stats")
        return dict(zip(["records", "groups", "candidates", "survivors"], [x.value for x in v]))

    def run(self, seqs, stream=None) -> None:
        """Queue a search over device-resident `seqs` (torch CUDA tensor)."""
        sp, sk, on_dev = _ptr(seqs, np.uint8)
        if not on_dev:
            raise ValueError("Plan.run needs the sequences in device memory")
        st = ctypes.c_void_p(stream) if stream is not None else _stream(seqs)
        check(native.lib().xtn_plan_run(self._h, sp, st), "xtn_plan_run")
        self._keep = sk

    def result(self, cap: int | None = None, like=None, stream=None):
        """Rows of the last run (raises XtnError with XTN_ERR_CAPACITY if the
        plan's pair capacity was too small; .needed holds the capacity needed)."""
        st = ctypes.c_void_p(stream) if stream is not None else _stream(like)
        if cap is None:
            cap = self.info()["pair_capacity"]
        out, optr = _alloc_rows(cap, like)
        n_out = ctypes.c_int64(0)
        rc = native.lib().xtn_plan_result(self._h, optr, int(cap), ctypes.byref(n_out), st)
        if rc != native.XTN_OK:
            e = XtnError(rc, "xtn_plan_result")
            e.needed = n_out.value
            raise e
        return out[: n_out.value]

    def free(self):
        if getattr(self, "_h", None):
            native.lib().xtn_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def index_build(seqs, offsets, d: int) -> Index:
    n = _n_items(offsets)
    sp, sk, _ = _ptr(seqs, np.uint8)
    op, ok, _ = _ptr(offsets, np.int64)
    h = ctypes.c_void_p(0)
    check(native.lib().xtn_index_build(sp, op, n, int(d), _stream(seqs), ctypes.byref(h)),
          "xtn_index_build")
    return Index(h)


def search_query(index: Index, q_seqs, q_offsets, cap: int | None = None, stream=None,
                 metric: str = "levenshtein"):
    """All (q, r) with Lev(query q, reference r) <= d; see xtn_search_query.
    metric "hamming" calls xtn_search_query_hamming (equal lengths)."""
    if metric not in _METRICS:
        raise ValueError(f"unknown metric {metric!r}")
    entry = "xtn_search_query_hamming" if metric == "hamming" else "xtn_search_query"
    n_q = _n_items(q_offsets)
    sp, sk, _ = _ptr(q_seqs, np.uint8)
    op, ok, _ = _ptr(q_offsets, np.int64)
    st = ctypes.c_void_p(stream) if stream is not None else _stream(q_seqs)
    if cap is None:
        cap = 8 * n_q + 1024

    def fn(optr, c, nref):
        return getattr(native.lib(), entry)(index.handle, sp, op, n_q, optr, c, nref, st)

    return _call_with_rows(fn, cap, q_seqs, entry)


def tcrdist_filter(seqs, offsets, rows, max_score: int = 24):
    """Rows of `rows` whose TCRdist score is <= max_score; see xtn_tcrdist_filter."""
    n = _n_items(offsets)
    n_in = int(rows.shape[0])
    sp, sk, _ = _ptr(seqs, np.uint8)
    op, ok, _ = _ptr(offsets, np.int64)
    if _is_torch(rows):
        rp, rk, _ = _ptr(rows)
    else:
        rp, rk, _ = _ptr(np.ascontiguousarray(rows, dtype=np.uint32).reshape(-1, 3), np.uint32)
    out, optr = _alloc_rows(n_in, rows if _is_torch(rows) else seqs)
    n_out = ctypes.c_int64(0)
    check(native.lib().xtn_tcrdist_filter(sp, op, n, rp, n_in, int(max_score), optr,
                                          ctypes.byref(n_out), _stream(seqs)),
          "xtn_tcrdist_filter")
    return out[: n_out.value]


def scratch_trim() -> None:
    """Free the cached scratch blocks of the current device (xtn_scratch_trim)."""
    check(native.lib().xtn_scratch_trim(), "xtn_scratch_trim")


def set_wait_limit(polls: int) -> None:
    """Poll limit of bounded device waits for later calls (0 = the default);
    see xtn_set_wait_limit."""
    check(native.lib().xtn_set_wait_limit(int(polls)), "xtn_set_wait_limit")


def profile_enable(on: bool = True) -> None:
    native.lib().xtn_profile_enable(1 if on else 0)


def profile_only(name: str | None = None) -> None:
    """Time only the launches named `name` (None: all); see xtn_profile_only."""
    check(native.lib().xtn_profile_only(name.encode() if name else None), "xtn_profile_only")


def profile_report() -> dict:
    """{kernel name: (launches, total_ms, algorithmic_bytes)} since the last report."""
    buf = ctypes.create_string_buffer(1 << 16)
    native.lib().xtn_profile_report(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, launches, ms, nbytes = line.split()
        out[name] = (int(launches), float(ms), float(nbytes))
    return out


def tune_set(knob: int, value: int) -> None:
    """Select a tile configuration for one of the radix sorts (see xtn_tune_set)."""
    check(native.lib().xtn_tune_set(int(knob), int(value)), "xtn_tune_set")


def tune_get(knob: int) -> int:
    return int(native.lib().xtn_tune_get(int(knob)))


def tune_count(knob: int) -> int:
    return int(native.lib().xtn_tune_count(int(knob)))
