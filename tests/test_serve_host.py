"""Host logic of the continuous-batching server, with a stand-in search (no
GPU): results split back per request, concurrent arrivals merged into one
micro-batch, the memory budget respected, cancellation before dispatch."""
import threading
import time

import numpy as np

import cdr3_synth as gen
from paper_2403_09010_gb300 import serve


def fake_search(delay=0.0, log=None):
    """rows (q, r, dist) depending on each query alone: r = sum of letters % 97."""
    def fn(seqs, offsets, stream):
        if log is not None:
            log.append(offsets.size - 1)
        time.sleep(delay)
        rows = []
        for q in range(offsets.size - 1):
            s = int(seqs[offsets[q]:offsets[q + 1]].astype(np.int64).sum())
            for r in sorted({s % 97, (s * 7) % 97}):
                rows.append((q, r, s % 3))
        return np.array(rows, np.uint32).reshape(-1, 3)
    return fn


def alone(seqs, offsets):
    return fake_search()(seqs, offsets, None)


def _requests(k, seed):
    out = []
    for r in range(k):
        s, o = gen.generate(1 + (r * 37) % 50, seed + r, 0.2, 0.0)
        out.append((r, s, o))
    return out


def test_results_split_per_request_and_batches_merge():
    log = []
    srv = serve.Server(slots=1, memory_budget=1 << 40, search_fn=fake_search(0.05, log),
                       device_streams=False)
    reqs = _requests(30, 1)
    pend = [srv.submit(r, s, o) for r, s, o in reqs]
    for p in pend:
        assert p.done.wait(30)
    srv.close()
    for (r, s, o), p in zip(reqs, pend):
        assert np.array_equal(p.rows, alone(s, o)), r
    st = srv.stats()
    assert st["requests"] == 30
    # with one slot busy for 50 ms, later arrivals were merged
    assert st["max_requests_per_batch"] > 1
    assert sum(log) == sum(o.size - 1 for _, _, o in reqs)


def test_memory_budget_bounds_what_is_in_flight():
    budget = serve.estimate_bytes(120)
    srv = serve.Server(slots=4, memory_budget=budget, search_fn=fake_search(0.02),
                       device_streams=False)
    reqs = _requests(40, 2)
    pend = [srv.submit(r, s, o) for r, s, o in reqs]
    for p in pend:
        assert p.done.wait(30)
    srv.close()
    st = srv.stats()
    assert st["peak_admitted_bytes"] <= budget
    for (r, s, o), p in zip(reqs, pend):
        assert np.array_equal(p.rows, alone(s, o))


def test_oversized_request_runs_alone():
    budget = serve.estimate_bytes(5)
    srv = serve.Server(slots=2, memory_budget=budget, search_fn=fake_search(0.0),
                       device_streams=False)
    s, o = gen.generate(400, 3, 0.2, 0.0)
    p = srv.submit(0, s, o)
    assert p.done.wait(30) and p.error is None
    srv.close()
    assert np.array_equal(p.rows, alone(s, o))


def test_cancel_before_dispatch():
    gate = threading.Event()

    def blocking(seqs, offsets, stream):
        gate.wait(10)
        return alone(seqs, offsets)

    srv = serve.Server(slots=1, memory_budget=1 << 40, search_fn=blocking, device_streams=False)
    s, o = gen.generate(10, 4, 0.2, 0.0)
    first = srv.submit(0, s, o)
    time.sleep(0.1)                 # first is now running and holds the only slot
    second = srv.submit(1, s, o)
    assert srv.cancel(second) and second.cancelled
    gate.set()
    assert first.done.wait(10)
    srv.close()
    assert np.array_equal(first.rows, alone(s, o))
    assert srv.stats()["requests"] == 1


def test_warm_runs_one_search_per_slot():
    calls = []

    def fake(seqs, offsets, stream):
        calls.append(stream)
        return np.zeros((0, 3), np.uint32)

    srv = serve.Server(None, slots=3, memory_budget=1 << 30, search_fn=fake, device_streams=False)
    seqs, off = gen.from_strings(["CASSLG", "CASSF"])
    srv.warm(seqs, off)
    srv.close()
    assert len(calls) == 3


def test_slot_workers_are_started_once():
    srv = serve.Server(slots=3, memory_budget=1 << 40, search_fn=fake_search(0.002),
                       device_streams=False)
    before = threading.active_count()
    reqs = _requests(60, 5)
    pend = []
    for r, s, o in reqs:
        pend.append(srv.submit(r, s, o))
        time.sleep(0.001)
    for p in pend:
        assert p.done.wait(30)
    during = threading.active_count()
    srv.close()
    assert srv.stats()["batches"] > 3
    assert during == before          # no thread per micro-batch
    for (r, s, o), p in zip(reqs, pend):
        assert np.array_equal(p.rows, alone(s, o))


def test_admission_by_scratch_estimate():
    # each request's scratch comes from scratch_fn; what is in flight never
    # exceeds the budget, and a request alone may exceed it
    per_query = 1000
    budget = 30 * per_query
    srv = serve.Server(slots=4, memory_budget=budget, search_fn=fake_search(0.01),
                       device_streams=False,
                       scratch_fn=lambda o: per_query * (np.asarray(o).size - 1))
    reqs = _requests(30, 6)
    pend = [srv.submit(r, s, o) for r, s, o in reqs]
    for p in pend:
        assert p.done.wait(30)
    srv.close()
    st = srv.stats()
    big = max(per_query * (o.size - 1) for _, _, o in reqs)
    assert st["peak_admitted_bytes"] <= max(budget, big)
    assert all(p.need == per_query * (o.size - 1) for (_, _, o), p in zip(reqs, pend))
