"""Query serving over a device-resident reference index, with continuous
batching (the fuzzy database lookup of the paper's Discussion, served).

Requests (each a packed batch of query sequences) arrive over time.  A
scheduler thread keeps up to `slots` micro-batches on the GPU at once.  Each
slot has its own CUDA stream, its own worker thread (started once; the C ABI
releases the GIL, so the searches overlap on the device) and its own pinned
host buffers: the batch's queries are concatenated straight into pinned
memory and the rows come back into pinned memory, so the library's
host<->device copies are asynchronous DMA.  Whenever a slot is free, every
request that has arrived and fits the memory budget is merged into one
micro-batch: one xtn_search_query call against the resident index, rows split
back per request (query indices local to the request).  Requests that arrive
while others are running join the next micro-batch as soon as a slot and
memory free up -- batching is continuous, not a fixed queue drain.

Admission is by device memory: each request's scratch is the library's own
estimate for its queries (xtn_search_query_scratch: exact in the queries'
lengths, the candidate part from the index's candidates per query variant so
far), and a micro-batch is admitted only while the scratch of everything in
flight stays within `memory_budget` bytes (by default half of the device
memory free when the server starts, capped at 16 GiB).  A request larger
than the whole budget is admitted alone.

Latency is measured from a request's scheduled arrival to the moment its rows
are ready on the host; `stats()` reports p50 / p99 latency, requests/s,
queries/s and verified pairs/s.
"""
from __future__ import annotations

import ctypes
import dataclasses
import queue
import threading
import time

import numpy as np

from . import native
from .native import check

# Scratch estimate used only without an index (a stand-in search in tests):
# per query sequence and per micro-batch.
BYTES_PER_QUERY = 8 * 1024
BYTES_PER_BATCH = 8 << 20


@dataclasses.dataclass
class _Pending:
    rid: int
    seqs: np.ndarray
    offsets: np.ndarray
    arrival: float               # scheduled arrival (time.perf_counter() clock)
    need: int = 0                # admitted device scratch (bytes)
    done: threading.Event = dataclasses.field(default_factory=threading.Event)
    rows: np.ndarray | None = None
    error: BaseException | None = None
    finished: float = 0.0
    batch_id: int = -1
    cancelled: bool = False


def estimate_bytes(n_queries: int) -> int:
    return BYTES_PER_BATCH + BYTES_PER_QUERY * int(n_queries)


class _Staging:
    """Host buffers of one slot, pinned when torch can pin them, grown to the
    largest batch seen (doubling)."""

    def __init__(self, pinned: bool):
        self.pinned = pinned
        self.bufs = {}

    def array(self, name: str, n: int, dtype) -> np.ndarray:
        n = max(int(n), 1)
        a = self.bufs.get(name)
        if a is None or a.size < n or a.dtype != np.dtype(dtype):
            size = max(n, 2 * (a.size if a is not None else 0))
            if self.pinned:
                import torch
                t = torch.empty(size * np.dtype(dtype).itemsize, dtype=torch.uint8,
                                pin_memory=True)
                a = t.numpy().view(dtype)
                self.bufs[name + "_keep"] = t
            else:
                a = np.empty(size, dtype=dtype)
            self.bufs[name] = a
        return a[:n]


class Server:
    """Continuous-batching query server for one xtn index.

    search_fn(seqs, offsets, stream) -> (rows (k, 3) uint32, sorted by query)
    defaults to xtn_search_query on `index`; tests may pass a stand-in.
    scratch_fn(offsets) -> bytes is the admission estimate of one request;
    by default the index's own (xtn_search_query_scratch), or estimate_bytes
    without an index.
    """

    def __init__(self, index=None, slots: int = 3, memory_budget: int | None = None,
                 max_batch_queries: int = 65536, search_fn=None, device_streams: bool = True,
                 scratch_fn=None):
        self.index = index
        self.slots = max(1, int(slots))
        self.max_batch_queries = int(max_batch_queries)
        if memory_budget is None:
            memory_budget = 16 << 30
            try:
                import torch
                free = torch.cuda.mem_get_info()[0]
                memory_budget = min(memory_budget, free // 2)
            except Exception:
                pass
        self.memory_budget = int(memory_budget)
        self._search = search_fn or self._xtn_search
        if scratch_fn is None:
            if index is not None and search_fn is None:
                scratch_fn = index.scratch_bytes
            else:
                scratch_fn = lambda offsets: estimate_bytes(np.asarray(offsets).size - 1)
        self._scratch = scratch_fn
        self._device_streams = device_streams
        self._waiting: list[_Pending] = []
        self._cv = threading.Condition()
        self._in_flight_bytes = 0
        self._free_slots = queue.SimpleQueue()
        self._streams = []
        self._staging = []
        self._work = []
        for k in range(self.slots):
            self._free_slots.put(k)
            self._streams.append(self._make_stream())
            self._staging.append(_Staging(pinned=device_streams))
            self._work.append(queue.SimpleQueue())
        self._stop = False
        self._batches: list[tuple[int, int, int]] = []   # (batch id, requests, queries)
        self._peak_in_flight = 0
        self._in_flight = 0
        self._peak_bytes = 0
        self._done: list[_Pending] = []
        self._next_batch = 0
        # one worker per slot for the server's life, and the scheduler
        self._workers = [threading.Thread(target=self._worker, args=(k,), daemon=True)
                         for k in range(self.slots)]
        for t in self._workers:
            t.start()
        self._scheduler = threading.Thread(target=self._schedule, daemon=True)
        self._scheduler.start()

    # ------------------------------------------------------------ plumbing
    def _make_stream(self):
        if not self._device_streams:
            return None
        import torch
        return torch.cuda.Stream()

    def _xtn_search(self, seqs, offsets, stream, slot=None):
        s = np.ascontiguousarray(seqs, dtype=np.uint8)
        if s.size == 0:
            s = np.zeros(1, np.uint8)
        o = np.ascontiguousarray(offsets, dtype=np.int64)
        n_q = o.size - 1
        st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        staging = self._staging[slot] if slot is not None else _Staging(False)
        cap = 8 * n_q + 1024
        while True:
            out = staging.array("rows", 3 * cap, np.uint32).reshape(cap, 3)
            n_out = ctypes.c_int64(0)
            rc = native.lib().xtn_search_query(self.index.handle, s.ctypes.data, o.ctypes.data,
                                               n_q, out.ctypes.data, cap, ctypes.byref(n_out), st)
            if rc == native.XTN_ERR_BUFFER_TOO_SMALL:
                cap = n_out.value
                continue
            check(rc, "xtn_search_query")
            return out[: n_out.value]

    def _run_search(self, seqs, offsets, slot):
        if self._search == self._xtn_search:
            return self._xtn_search(seqs, offsets, self._streams[slot], slot)
        return self._search(seqs, offsets, self._streams[slot])

    # ------------------------------------------------------------- public
    def warm(self, seqs, offsets):
        """Run one search on every slot's stream before serving, so that no
        request pays first-use costs (pool growth on a new stream, pinned
        buffers)."""
        s = np.asarray(seqs, np.uint8)
        o = np.asarray(offsets, np.int64)
        for k in range(self.slots):
            st = self._staging[k]
            ss = st.array("seqs", s.size, np.uint8)
            ss[:] = s
            oo = st.array("offs", o.size, np.int64)
            oo[:] = o
            self._run_search(ss, oo, k)
        if self._device_streams:
            import torch
            torch.cuda.synchronize()

    def submit(self, rid: int, seqs, offsets, arrival: float | None = None) -> _Pending:
        offsets = np.asarray(offsets, np.int64)
        p = _Pending(rid, np.asarray(seqs, np.uint8), offsets,
                     time.perf_counter() if arrival is None else arrival,
                     need=int(self._scratch(offsets)))
        with self._cv:
            self._waiting.append(p)
            self._cv.notify_all()
        return p

    def cancel(self, p: _Pending) -> bool:
        """Withdraw a request that has not been dispatched yet."""
        with self._cv:
            if p in self._waiting:
                self._waiting.remove(p)
                p.cancelled = True
                p.done.set()
                return True
        return False

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._scheduler.join(timeout=60)
        for q in self._work:
            q.put(None)
        for t in self._workers:
            t.join(timeout=60)

    # ---------------------------------------------------------- scheduling
    def _take_batch(self):
        """Waiting requests that fit the memory budget, oldest first."""
        batch, queries, need = [], 0, 0
        for p in list(self._waiting):
            nq = p.offsets.size - 1
            fits = self._in_flight_bytes + need + p.need <= self.memory_budget
            alone = not batch and self._in_flight_bytes == 0
            if batch and (queries + nq > self.max_batch_queries or not fits):
                break
            if not batch and not fits and not alone:
                break
            batch.append(p)
            queries += nq
            need += p.need
        for p in batch:
            self._waiting.remove(p)
        return batch, queries, need

    def _schedule(self):
        while True:
            slot = self._free_slots.get()
            with self._cv:
                while True:
                    if self._stop and not self._waiting:
                        self._free_slots.put(slot)
                        return
                    batch, queries, need = self._take_batch() if self._waiting else ([], 0, 0)
                    if batch:
                        break
                    self._cv.wait(timeout=0.05)
                self._in_flight_bytes += need
                self._in_flight += 1
                self._peak_in_flight = max(self._peak_in_flight, self._in_flight)
                self._peak_bytes = max(self._peak_bytes, self._in_flight_bytes)
                bid = self._next_batch
                self._next_batch += 1
                self._batches.append((bid, len(batch), queries))
            self._work[slot].put((bid, batch, need))

    def _worker(self, slot):
        while True:
            item = self._work[slot].get()
            if item is None:
                return
            self._run_batch(slot, *item)

    def _run_batch(self, slot, bid, batch, need):
        try:
            st = self._staging[slot]
            lens = [p.offsets.size - 1 for p in batch]
            q_base = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
            n_q = int(q_base[-1])
            byte_base = np.concatenate([[0], np.cumsum([p.offsets[-1] for p in batch])])
            seqs = st.array("seqs", int(byte_base[-1]), np.uint8)
            offsets = st.array("offs", n_q + 1, np.int64)
            offsets[0] = 0
            for k, p in enumerate(batch):
                seqs[byte_base[k]:byte_base[k + 1]] = p.seqs[: p.offsets[-1]]
                offsets[q_base[k] + 1:q_base[k + 1] + 1] = p.offsets[1:] + byte_base[k]
            rows = self._run_search(seqs[: int(byte_base[-1])], offsets, slot)
            q = rows[:, 0].astype(np.int64) if rows.size else np.zeros(0, np.int64)
            cut = np.searchsorted(q, q_base)
            now = time.perf_counter()
            for k, p in enumerate(batch):
                part = np.array(rows[cut[k]:cut[k + 1]], dtype=np.uint32, copy=True)
                part[:, 0] -= np.uint32(q_base[k])
                p.rows = part
                p.finished = now
                p.batch_id = bid
                p.done.set()
        except BaseException as e:  # surfaced to the caller of wait()
            for p in batch:
                p.error = e
                p.finished = time.perf_counter()
                p.done.set()
        finally:
            with self._cv:
                self._in_flight_bytes -= need
                self._in_flight -= 1
                self._done.extend(batch)
                self._cv.notify_all()
            self._free_slots.put(slot)

    # -------------------------------------------------------------- report
    def stats(self, pending=None):
        reqs = pending if pending is not None else self._done
        reqs = [p for p in reqs if not p.cancelled and p.error is None]
        if not reqs:
            return {}
        lat = np.array([p.finished - p.arrival for p in reqs]) * 1e3
        t0 = min(p.arrival for p in reqs)
        t1 = max(p.finished for p in reqs)
        queries = sum(p.offsets.size - 1 for p in reqs)
        pairs = sum(p.rows.shape[0] for p in reqs)
        sizes = [b[1] for b in self._batches]
        return {
            "requests": len(reqs),
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()),
            "requests_per_s": len(reqs) / (t1 - t0),
            "queries_per_s": queries / (t1 - t0),
            "pairs_per_s": pairs / (t1 - t0),
            "batches": len(sizes),
            "mean_requests_per_batch": float(np.mean(sizes)) if sizes else 0.0,
            "max_requests_per_batch": int(max(sizes)) if sizes else 0,
            "peak_batches_in_flight": self._peak_in_flight,
            "peak_admitted_bytes": self._peak_bytes,
            "memory_budget": self.memory_budget,
        }


def replay(server: Server, requests, speed: float = 1.0):
    """Submit requests at their arrival times (seconds from the first one,
    divided by `speed`) and wait for all results; returns the pending list."""
    t0 = time.perf_counter()
    base = requests[0].arrival_s if requests else 0.0
    pending = []
    for r in requests:
        due = t0 + (r.arrival_s - base) / speed
        delay = due - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        pending.append(server.submit(r.rid, r.seqs, r.offsets, arrival=due))
    for p in pending:
        p.done.wait()
        if p.error is not None:
            raise p.error
    return pending
