"""CUDA path vs the CPU oracle, element by element (bit-exact integer rows).

Every case calls the C ABI through the thin binding.  Outputs are the sorted
(i, j, dist) rows; the oracle computes the same rows from strings with full
dynamic programming (oracle/xtn_oracle.cpp).
"""
import functools

import numpy as np
import pytest

import cdr3_synth as gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def xtn():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2403_09010_gb300 as pkg
    pkg.build()
    return pkg


def _rows(x):
    if isinstance(x, np.ndarray):
        return x.astype(np.uint32)
    return x.cpu().numpy().astype(np.uint32)


def _dev(seqs, off):
    return (torch.from_numpy(np.ascontiguousarray(seqs)).cuda(),
            torch.from_numpy(np.ascontiguousarray(off)).cuda())


def _rand_strings(rng, n, alphabet, lmin, lmax):
    L = rng.integers(lmin, lmax + 1, n)
    return ["".join(rng.choice(list(alphabet), size=l)) for l in L]


# ------------------------------------------------------------ self search ---
def test_pinned_host_buffers_read_and_written_in_place(xtn):
    """Pinned host letters, offsets and rows (read and written by the kernels
    in place) give the oracle's rows, as pageable and device buffers do; a
    short pinned output gets the first rows and the full count."""
    import ctypes
    from paper_2403_09010_gb300 import native
    seqs, off = gen.workload(gen.SELF_1M, 30_000)
    n = off.size - 1
    want = oracle.symdel_self(seqs, off, 2)
    hs = torch.from_numpy(seqs).pin_memory()
    ho = torch.from_numpy(off).pin_memory()
    lib = native.lib()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    for cap in (len(want) + 16, 5):
        out = torch.full((cap, 3), -1, dtype=torch.int32).pin_memory()
        n_out = ctypes.c_int64(0)
        rc = lib.xtn_search_self(ptr(hs), ptr(ho), n, 2, None, 0, ptr(out), cap,
                                 ctypes.byref(n_out), None)
        assert n_out.value == len(want)
        w = min(cap, len(want))
        assert rc == (native.XTN_OK if cap >= len(want) else native.XTN_ERR_BUFFER_TOO_SMALL)
        assert np.array_equal(out[:w].numpy().astype(np.uint32), want[:w])
    assert np.array_equal(_rows(xtn.search_self(seqs, off, 2)), want)          # pageable
    ds, do = _dev(seqs, off)
    assert np.array_equal(_rows(xtn.search_self(ds, do, 2)), want)             # device
    # queries from pinned memory against a resident index
    idx = xtn.index_build(seqs[: off[20_000]], off[: 20_001], 2)
    q_off = off[20_000:22_001] - off[20_000]
    q = seqs[off[20_000]:off[22_000]]
    qw = oracle.bruteforce_query(seqs[: off[20_000]], off[: 20_001], q, q_off, 2, threads=0)
    got = _rows(xtn.search_query(idx, torch.from_numpy(q).pin_memory(),
                                 torch.from_numpy(q_off).pin_memory()))
    idx.free()
    assert np.array_equal(got, qw)


def test_selfsearch_n1e4_d1_full(xtn):
    seqs, off = gen.workload(gen.SELF_SMALL)
    want = oracle.symdel_self(seqs, off, 1)
    got = _rows(xtn.search_self(seqs, off, 1))
    assert got.shape == want.shape and np.array_equal(got, want)


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_selfsearch_generator_slice(xtn, d):
    n = {0: 20_000, 1: 20_000, 2: 20_000, 3: 3_000}[d]
    seqs, off = gen.workload(gen.SELF_1M, n)
    want = oracle.symdel_self(seqs, off, d)
    got = _rows(xtn.search_self(seqs, off, d))
    assert np.array_equal(got, want)


def test_device_inputs_match_host_inputs(xtn):
    seqs, off = gen.generate(30_000, 77, 0.2, 0.01)
    host = _rows(xtn.search_self(seqs, off, 2))
    ds, do = _dev(seqs, off)
    dev_out = xtn.search_self(ds, do, 2)
    assert dev_out.is_cuda
    assert np.array_equal(_rows(dev_out), host)
    assert np.array_equal(host, oracle.symdel_self(seqs, off, 2))


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_small_alphabet_collisions(xtn, d):
    rng = np.random.default_rng(100 + d)
    strs = _rand_strings(rng, 400, "AC", 0, 9)
    seqs, off = gen.from_strings(strs)
    want = oracle.bruteforce_self(seqs, off, d)
    got = _rows(xtn.search_self(seqs, off, d))
    assert np.array_equal(got, want)


def test_edge_cases(xtn):
    # empty input
    seqs, off = gen.from_strings([])
    assert xtn.search_self(seqs, off, 2).shape[0] == 0
    # one sequence, empty strings, maximum length, repeats
    for strs, d in [(["CASSF"], 2), (["", "", "A"], 1), (["W" * 25, "W" * 24, "Y" * 25], 1),
                    (["AAAAAAAAAAAAAAAAAAAAAAAAA", "AAAAAAAAAAAAAAAAAAAAAAAA"], 3),
                    (["ACDEFGHIKLMNPQRSTVWYACDEF", "CDEFGHIKLMNPQRSTVWYACDEFA"], 2)]:
        seqs, off = gen.from_strings(strs)
        assert np.array_equal(_rows(xtn.search_self(seqs, off, d)),
                              oracle.bruteforce_self(seqs, off, d)), strs


def test_identical_sequences_one_giant_bucket(xtn):
    n = 700
    seqs, off = gen.from_strings(["CASSLGQETQYF"] * n)
    got = _rows(xtn.search_self(seqs, off, 2))
    assert got.shape[0] == n * (n - 1) // 2
    assert np.all(got[:, 2] == 0)
    ii, jj = np.triu_indices(n, 1)
    assert np.array_equal(got[:, 0], ii) and np.array_equal(got[:, 1], jj)


def test_d_covers_every_length(xtn):
    rng = np.random.default_rng(5)
    strs = _rand_strings(rng, 150, "ACDEFG", 0, 3)
    seqs, off = gen.from_strings(strs)
    got = _rows(xtn.search_self(seqs, off, 3))
    assert got.shape[0] == 150 * 149 // 2
    assert np.array_equal(got, oracle.bruteforce_self(seqs, off, 3))


def test_buffer_too_small_reports_count(xtn):
    import ctypes
    from paper_2403_09010_gb300 import native
    seqs, off = gen.workload(gen.SELF_SMALL)
    want = oracle.symdel_self(seqs, off, 1)
    cap = 10
    out = np.zeros((cap, 3), np.uint32)
    n_out = ctypes.c_int64(0)
    s = np.ascontiguousarray(seqs)
    o = np.ascontiguousarray(off)
    rc = native.lib().xtn_search_self(s.ctypes.data, o.ctypes.data, o.size - 1, 1, None, 0,
                                      out.ctypes.data, cap, ctypes.byref(n_out), None)
    assert rc == native.XTN_ERR_BUFFER_TOO_SMALL
    assert n_out.value == want.shape[0]
    assert np.array_equal(out, want[:cap])


def test_input_errors(xtn):
    from paper_2403_09010_gb300 import native
    for strs, code in [(["CASSF", "CAXSF"], native.XTN_ERR_BAD_RESIDUE),
                       (["CASSF", "cassf"], native.XTN_ERR_BAD_RESIDUE),
                       (["A" * 26], native.XTN_ERR_SEQ_TOO_LONG),
                       (["A" * 26, "", ""], native.XTN_ERR_SEQ_TOO_LONG)]:
        seqs, off = gen.from_strings(strs)
        with pytest.raises(native.XtnError) as ei:
            xtn.search_self(seqs, off, 1)
        assert ei.value.status == code
        # the same checks on device-resident input run in the encode kernel
        ds, do = _dev(seqs, off)
        with pytest.raises(native.XtnError) as ei:
            xtn.search_self(ds, do, 1)
        assert ei.value.status == code


def test_decreasing_offsets_are_rejected(xtn):
    from paper_2403_09010_gb300 import native
    seqs, _ = gen.from_strings(["CASSF", "CASF"])
    off = np.array([0, 5, 3, 9], dtype=np.int64)      # a negative length inside the total
    for s_, o_ in [(seqs, off), _dev(seqs, off)]:
        with pytest.raises(native.XtnError) as ei:
            xtn.search_self(s_, o_, 1)
        assert ei.value.status == native.XTN_ERR_INVALID_ARG


def test_every_sort_configuration(xtn):
    R, P, H = xtn.XTN_TUNE_SORT_RECORDS, xtn.XTN_TUNE_SORT_PAIRS, xtn.XTN_TUNE_RECORD_HISTOGRAM
    default = (xtn.tune_get(R), xtn.tune_get(P), xtn.tune_get(H))
    seqs, off = gen.workload(gen.SELF_1M, 60_000)
    want = oracle.symdel_self(seqs, off, 2)
    small_s, small_o = gen.generate(777, 4, 0.5, 0.1)
    small_want = oracle.symdel_self(small_s, small_o, 2)
    try:
        for h in range(xtn.tune_count(H)):
            xtn.tune_set(H, h)
            for cfg in range(xtn.tune_count(R)):
                xtn.tune_set(R, cfg)
                xtn.tune_set(P, cfg)
                assert np.array_equal(_rows(xtn.search_self(seqs, off, 2)), want), (h, cfg)
                assert np.array_equal(_rows(xtn.search_self(small_s, small_o, 2)),
                                      small_want), (h, cfg)
            # the planned path takes the knobs at plan creation
            plan = xtn.Plan(off, 2)
            plan.run(torch.from_numpy(seqs).cuda())
            assert np.array_equal(_rows(plan.result()), want), h
            plan.free()
    finally:
        xtn.tune_set(R, default[0])
        xtn.tune_set(P, default[1])
        xtn.tune_set(H, default[2])


# -------------------------------------------------------- grouping modes ---
@functools.lru_cache(maxsize=None)
def _case(name):
    """(seqs, offsets, d, expected rows) of a named parity case; expected
    values come from the oracle only."""
    if name == "gen60k_d2":
        seqs, off = gen.workload(gen.SELF_1M, 60_000)
        return seqs, off, 2, oracle.symdel_self(seqs, off, 2)
    if name == "small_d1":
        seqs, off = gen.workload(gen.SELF_SMALL)
        return seqs, off, 1, oracle.symdel_self(seqs, off, 1)
    if name == "tiny_d2":  # one bucket only (no global pass)
        seqs, off = gen.workload(gen.SELF_1M, 20)
        return seqs, off, 2, oracle.bruteforce_self(seqs, off, 2)
    if name == "alphabet_AC_d2":
        strs = _rand_strings(np.random.default_rng(31), 400, "AC", 0, 9)
        seqs, off = gen.from_strings(strs)
        return seqs, off, 2, oracle.bruteforce_self(seqs, off, 2)
    raise KeyError(name)


def _with_copies(base_seqs, base_off, copy, n_copies, d):
    """Input = base sequences followed by n_copies of `copy`, and its rows:
    the oracle on base + one copy, the copy's rows repeated for every copy,
    and every pair of copies at distance 0."""
    base = gen.to_strings(base_seqs, base_off)
    nb = len(base)
    s1, o1 = gen.from_strings(base + [copy])
    one = oracle.symdel_self(s1, o1, d).astype(np.int64)
    keep = one[one[:, 1] < nb]
    to_copy = one[one[:, 1] == nb]
    parts = [keep]
    for k in range(n_copies):
        t = to_copy.copy()
        t[:, 1] = nb + k
        parts.append(t)
    ii, jj = np.triu_indices(n_copies, 1)
    parts.append(np.stack([ii + nb, jj + nb, np.zeros_like(ii)], 1))
    rows = np.concatenate(parts)
    rows = rows[np.lexsort((rows[:, 1], rows[:, 0]))]
    seqs, off = gen.from_strings(base + [copy] * n_copies)
    return seqs, off, rows.astype(np.uint32)


@pytest.fixture
def grouping(xtn):
    G = xtn.XTN_TUNE_GROUPING
    old = xtn.tune_get(G)
    yield lambda mode: xtn.tune_set(G, mode)
    xtn.tune_set(G, old)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_grouping_modes_match_oracle(xtn, grouping, mode):
    grouping(mode)
    for name in ["gen60k_d2", "small_d1", "tiny_d2", "alphabet_AC_d2"]:
        seqs, off, d, want = _case(name)
        assert np.array_equal(_rows(xtn.search_self(seqs, off, d)), want), (mode, name)
    # planned path (device-side counts) and the 700-copy bucket
    seqs, off, d, want = _case("gen60k_d2")
    plan = xtn.Plan(off, d)
    plan.run(torch.from_numpy(seqs).cuda())
    assert np.array_equal(_rows(plan.result()), want), mode
    plan.free()
    n = 700
    seqs, off = gen.from_strings(["CASSLGQETQYF"] * n)
    got = _rows(xtn.search_self(seqs, off, 2))
    ii, jj = np.triu_indices(n, 1)
    assert got.shape[0] == ii.size and np.all(got[:, 2] == 0), mode
    assert np.array_equal(got[:, 0], ii) and np.array_equal(got[:, 1], jj), mode


@pytest.mark.parametrize("mode", [0, 2])
def test_plan_with_buckets_larger_than_shared_memory(xtn, grouping, mode):
    # a plan emits the pairs of small buckets while grouping and those of
    # large ones (here 700 copies, and with 512-record segments also some
    # generator buckets) through the flag route, appended after them
    grouping(mode)
    bs, bo = gen.workload(gen.SELF_1M, 4000)
    seqs, off, want = _with_copies(bs, bo, "CASSLGQETQYF", 700, 2)
    # 700 copies of a 12-residue sequence: about 19.3 M candidate words
    plan = xtn.Plan(off, 2, pair_capacity=30_000_000)
    plan.run(torch.from_numpy(seqs).cuda())
    got = _rows(plan.result())
    plan.free()
    assert got.shape == want.shape and np.array_equal(got, want)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_grouping_modes_query_index(xtn, grouping, mode):
    grouping(mode)
    rs, ro, reqs = gen.served(ref_n=30_000, n_req=3, max_req=2000)
    idx = xtn.index_build(rs, ro, 2)
    for r in reqs:
        want = oracle.symdel_query(rs, ro, r.seqs, r.offsets, 2)
        assert np.array_equal(_rows(xtn.search_query(idx, r.seqs, r.offsets)), want), mode
    idx.free()


@pytest.mark.parametrize("mode", [0, 2])
def test_bucket_larger_than_shared_memory(xtn, grouping, mode):
    # 4,200 copies put more records in one bucket than a block's shared memory
    # holds (2,048 when grouping, 4,096 when sorting): that bucket is sorted
    # in global memory
    grouping(mode)
    bs, bo = gen.workload(gen.SELF_1M, 3000)
    seqs, off, want = _with_copies(bs, bo, "CASS", 4200, 1)
    got = _rows(xtn.search_self(seqs, off, 1))
    assert got.shape == want.shape and np.array_equal(got, want)


# --------------------------------------------------------------- batched ---
def test_batched_matches_oracle(xtn):
    seqs, off, rep = gen.batched(n_rep=12, seed=9, size_min=1, size_max=3000)
    want = oracle.symdel_batched(seqs, off, rep, 2)             # (rep, i_loc, j_loc, dist)
    got = _rows(xtn.search_self(seqs, off, 2, rep_offsets=rep))  # global indices
    rep_of = np.searchsorted(rep, got[:, 0], side="right") - 1
    assert np.all(np.searchsorted(rep, got[:, 1], side="right") - 1 == rep_of)
    local = np.stack([rep_of, got[:, 0] - rep[rep_of], got[:, 1] - rep[rep_of], got[:, 2]], 1)
    assert np.array_equal(local.astype(np.uint32), want)


def test_batched_equals_separate_calls(xtn):
    seqs, off, rep = gen.batched(n_rep=6, seed=10, size_min=500, size_max=4000)
    got = _rows(xtn.search_self(seqs, off, 2, rep_offsets=rep))
    parts = []
    for r in range(6):
        s = seqs[off[rep[r]]:off[rep[r + 1]]]
        o = off[rep[r]:rep[r + 1] + 1] - off[rep[r]]
        g = _rows(xtn.search_self(s, o, 2)).astype(np.int64)
        g[:, :2] += rep[r]
        parts.append(g)
    assert np.array_equal(got, np.concatenate(parts).astype(np.uint32))


# ------------------------------------------------------------------ plans ---
def test_plan_matches_one_shot_and_replays_in_a_graph(xtn):
    seqs, off, rep = gen.batched(n_rep=20, seed=11, size_min=100, size_max=8000)
    want = _rows(xtn.search_self(seqs, off, 2, rep_offsets=rep))
    ds, do = _dev(seqs, off)
    plan = xtn.Plan(off, 2, rep_offsets=rep)
    info = plan.info()
    assert info["record_capacity"] > 0 and info["pair_capacity"] >= 65536
    plan.run(ds)
    assert np.array_equal(_rows(plan.result(like=ds)), want)
    # the run queues only kernels and memsets: capture it and replay
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.run(ds)                       # warm-up on the capture stream
        torch.cuda.current_stream().synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.run(ds)
    for _ in range(3):
        g.replay()
        got = _rows(plan.result(like=ds))
        assert np.array_equal(got, want)
    # new letters, same layout: the graph searches whatever is in the buffer now
    mutated = seqs.copy()
    mutated[::7] = ord("W")
    ds.copy_(torch.from_numpy(mutated))
    g.replay()
    assert np.array_equal(_rows(plan.result(like=ds)),
                          _rows(xtn.search_self(mutated, off, 2, rep_offsets=rep)))
    plan.free()


def test_plan_capacity_is_reported(xtn):
    from paper_2403_09010_gb300 import native
    seqs, off = gen.workload(gen.SELF_1M, 30_000)
    want = oracle.symdel_self(seqs, off, 2)
    ds, do = _dev(seqs, off)
    small = xtn.Plan(do, 2, pair_capacity=1000)
    small.run(ds)
    with pytest.raises(native.XtnError) as ei:
        small.result(like=ds)
    assert ei.value.status == native.XTN_ERR_CAPACITY and ei.value.needed > 1000
    big = xtn.Plan(do, 2, pair_capacity=ei.value.needed)
    big.run(ds)
    assert np.array_equal(_rows(big.result(like=ds)), want)


# --------------------------------------------------------------- Hamming ---
@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_hamming_matches_oracle(xtn, d):
    seqs, off = gen.workload(gen.SELF_1M, 20_000 if d < 3 else 3_000)
    want = oracle.symdel_self(seqs, off, d, "hamming")
    assert np.array_equal(_rows(xtn.search_self(seqs, off, d, metric="hamming")), want)
    # two letters: many equal-length near-copies and repeated residues
    strs = _rand_strings(np.random.default_rng(60 + d), 400, "AC", 0, 9)
    s2, o2 = gen.from_strings(strs)
    assert np.array_equal(_rows(xtn.search_self(s2, o2, d, metric="hamming")),
                          oracle.bruteforce_self(s2, o2, d, "hamming"))


def test_hamming_batched_matches_oracle(xtn):
    seqs, off, rep = gen.batched(n_rep=8, seed=21, size_min=100, size_max=3000)
    want = oracle.symdel_batched(seqs, off, rep, 2, "hamming")
    got = _rows(xtn.search_self(seqs, off, 2, rep_offsets=rep, metric="hamming"))
    rep_of = np.searchsorted(rep, got[:, 0], side="right") - 1
    local = np.stack([rep_of, got[:, 0] - rep[rep_of], got[:, 1] - rep[rep_of], got[:, 2]], 1)
    assert np.array_equal(local.astype(np.uint32), want)


def test_hamming_pairs_are_levenshtein_pairs_1m(xtn):
    # at full size: every Hamming pair is a Levenshtein pair of the same d
    # with no larger distance, and has equal lengths
    seqs, off = gen.workload(gen.SELF_1M)
    ds, do = _dev(seqs, off)
    ham = _rows(xtn.search_self(ds, do, 2, metric="hamming"))
    lev = _rows(xtn.search_self(ds, do, 2))
    assert 0 < ham.shape[0] <= lev.shape[0]
    key = lambda r: r[:, 0].astype(np.uint64) << np.uint64(32) | r[:, 1].astype(np.uint64)
    pos = np.searchsorted(key(lev), key(ham))
    assert np.all(pos < lev.shape[0]) and np.array_equal(key(lev)[pos], key(ham))
    assert np.all(lev[pos, 2] <= ham[:, 2])
    lens = np.diff(off)
    assert np.array_equal(lens[ham[:, 0]], lens[ham[:, 1]])
    # a sample of rows against the plain definition
    strs = gen.to_strings(seqs, off)
    rng = np.random.default_rng(5)
    for r in ham[rng.choice(ham.shape[0], 200, replace=False)]:
        assert oracle.hamming(strs[r[0]], strs[r[1]]) == r[2]


def test_autotuned_plan_matches_oracle_and_leaves_knobs(xtn):
    from paper_2403_09010_gb300 import autotune
    seqs, off, rep = gen.batched(n_rep=8, seed=22, size_min=100, size_max=3000)
    knobs = [k for _, k in xtn.xtn._TUNING_KNOBS]
    before = [xtn.tune_get(k) for k in knobs]
    ds = torch.from_numpy(seqs).cuda()
    r = autotune.tune(ds, off, 2, rep_offsets=rep, configs=[0, 9], repeats=1, use_cache=False)
    assert [xtn.tune_get(k) for k in knobs] == before
    plan = xtn.Plan(off, 2, rep_offsets=rep, tuning=r)
    assert plan.info()["pair_capacity"] >= r["pair_capacity"]
    plan.run(ds)
    got = _rows(plan.result(like=ds))
    want = oracle.symdel_batched(seqs, off, rep, 2)
    rep_of = np.searchsorted(rep, got[:, 0], side="right") - 1
    local = np.stack([rep_of, got[:, 0] - rep[rep_of], got[:, 1] - rep[rep_of], got[:, 2]], 1)
    assert np.array_equal(local.astype(np.uint32), want)
    plan.free()


def test_scratch_cache_reuse_grow_trim_and_threads(xtn):
    # calls carve scratch from cached blocks: repeated calls, a larger call
    # that grows the block, a trim, and calls on two streams from two threads
    import threading
    a_s, a_o = gen.workload(gen.SELF_1M, 20_000)
    b_s, b_o = gen.workload(gen.SELF_1M, 12_000)
    want_a = oracle.symdel_self(a_s, a_o, 2)
    want_b = oracle.symdel_self(b_s, b_o, 2)
    for _ in range(3):
        assert np.array_equal(_rows(xtn.search_self(a_s, a_o, 2)), want_a)
    big_s, big_o = gen.workload(gen.SELF_1M, 200_000)
    big = _rows(xtn.search_self(big_s, big_o, 2))
    assert np.array_equal(_rows(xtn.search_self(big_s, big_o, 2)), big)
    assert np.array_equal(_rows(xtn.search_self(b_s, b_o, 2)), want_b)
    xtn.scratch_trim()
    assert np.array_equal(_rows(xtn.search_self(a_s, a_o, 2)), want_a)
    results, errors = {}, []

    def worker(name, s, o, reps):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                ds, do = _dev(s, o)
                results[name] = [_rows(xtn.search_self(ds, do, 2)) for _ in range(reps)]
        except Exception as e:  # reported below
            errors.append(e)

    ts = [threading.Thread(target=worker, args=("a", a_s, a_o, 6)),
          threading.Thread(target=worker, args=("b", b_s, b_o, 6))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors
    assert all(np.array_equal(r, want_a) for r in results["a"])
    assert all(np.array_equal(r, want_b) for r in results["b"])


# ---------------------------------------------------- between repertoires ---
@pytest.mark.parametrize("d,metric", [(1, "levenshtein"), (2, "levenshtein"),
                                      (3, "levenshtein"), (2, "hamming")])
def test_between_matches_oracle(xtn, d, metric):
    # one generated set cut into eight repertoires at random points: its
    # near-copies land in other repertoires, so there are pairs between them
    n = 20_000 if d < 3 else 3_000
    seqs, off = gen.workload(gen.SELF_1M, n)
    cuts = np.sort(np.random.default_rng(40 + d).choice(np.arange(1, n), 7, replace=False))
    rep = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    want = oracle.symdel_cross(seqs, off, rep, d, metric)
    got = _rows(xtn.search_between(seqs, off, d, rep, metric=metric))
    assert want.shape[0] > 0 and np.array_equal(got, want)


def test_between_independent_repertoires(xtn):
    # repertoires drawn independently share few neighbours
    seqs, off, rep = gen.batched(n_rep=8, seed=33, size_min=100, size_max=3000)
    want = oracle.symdel_cross(seqs, off, rep, 2)
    assert np.array_equal(_rows(xtn.search_between(seqs, off, 2, rep)), want)


def test_between_small_alphabet_and_empty_repertoires(xtn):
    # two letters give many shared variants across repertoires; empty
    # repertoires and a single repertoire are degenerate cases
    rng = np.random.default_rng(70)
    strs = _rand_strings(rng, 500, "AC", 0, 8)
    s2, o2 = gen.from_strings(strs)
    rep = np.array([0, 0, 120, 120, 121, 380, 500, 500], dtype=np.int64)
    for d in (0, 1, 2):
        got = _rows(xtn.search_between(s2, o2, d, rep))
        assert np.array_equal(got, oracle.symdel_cross(s2, o2, rep, d))
    one = np.array([0, 500], dtype=np.int64)
    assert _rows(xtn.search_between(s2, o2, 2, one)).shape[0] == 0


def test_within_and_between_partition_the_1m_search(xtn):
    # at full size: the rows between four repertoires of the 1M set and the
    # rows within them together are the rows of the whole self-search
    seqs, off = gen.workload(gen.SELF_1M)
    n = off.size - 1
    rep = np.array([0, n // 5, n // 2, n - 1000, n], dtype=np.int64)
    ds, do = _dev(seqs, off)
    whole = _rows(xtn.search_self(ds, do, 2))
    between = _rows(xtn.search_between(ds, do, 2, rep))
    within = _rows(xtn.search_self(ds, do, 2, rep_offsets=rep))
    r_of = lambda i: np.searchsorted(rep, i, side="right") - 1
    assert np.all(r_of(between[:, 0]) != r_of(between[:, 1]))
    assert np.all(r_of(within[:, 0]) == r_of(within[:, 1]))
    both = np.concatenate([between, within])
    both = both[np.lexsort((both[:, 1], both[:, 0]))]
    assert np.array_equal(both, whole)


# ----------------------------------------------------------------- query ---
@pytest.mark.parametrize("d", [1, 2])
def test_query_matches_oracle(xtn, d):
    rs, ro, reqs = gen.served(ref_n=40_000, n_req=6, max_req=3000)
    idx = xtn.index_build(rs, ro, d)
    info = idx.info()
    assert info["n"] == 40_000 and info["d"] == d
    for r in reqs:
        want = oracle.symdel_query(rs, ro, r.seqs, r.offsets, d)
        got = _rows(xtn.search_query(idx, r.seqs, r.offsets))
        assert np.array_equal(got, want)
    idx.free()


def test_query_hamming_matches_oracle(xtn):
    rs, ro, reqs = gen.served(ref_n=40_000, n_req=4, max_req=3000)
    idx = xtn.index_build(rs, ro, 2)
    for r in reqs:
        want = oracle.symdel_query(rs, ro, r.seqs, r.offsets, 2, "hamming")
        got = _rows(xtn.search_query(idx, r.seqs, r.offsets, metric="hamming"))
        assert np.array_equal(got, want)
    # two letters: equal-length near-copies and repeated residues
    rng = np.random.default_rng(72)
    ref, qs = _rand_strings(rng, 400, "AC", 0, 9), _rand_strings(rng, 150, "AC", 0, 9)
    (a, ao), (b, bo) = gen.from_strings(ref), gen.from_strings(qs)
    small = xtn.index_build(a, ao, 2)
    assert np.array_equal(_rows(xtn.search_query(small, b, bo, metric="hamming")),
                          oracle.bruteforce_query(a, ao, b, bo, 2, "hamming"))
    small.free()
    idx.free()


def test_query_small_reference_bruteforce(xtn):
    rng = np.random.default_rng(8)
    ref = _rand_strings(rng, 300, "ACD", 0, 7)
    qs = _rand_strings(rng, 120, "ACD", 0, 7)
    rs, ro = gen.from_strings(ref)
    q, qo = gen.from_strings(qs)
    for d in [0, 1, 2, 3]:
        idx = xtn.index_build(rs, ro, d)
        assert np.array_equal(_rows(xtn.search_query(idx, q, qo)),
                              oracle.bruteforce_query(rs, ro, q, qo, d))
        idx.free()


# --------------------------------------------------------------- tcrdist ---
def test_tcrdist_filter_matches_oracle(xtn):
    seqs, off = gen.workload(gen.TCRDIST_1M, 5000)
    lev = _rows(xtn.search_self(seqs, off, 2))
    got = _rows(xtn.tcrdist_filter(seqs, off, lev, 24))
    want = oracle.tcrdist_filter(seqs, off, lev, 24)
    assert np.array_equal(got, want)
    allp = oracle.tcrdist_allpairs(seqs, off, 2, 24)
    assert np.array_equal(got, allp[:, :3])


@pytest.mark.parametrize("d", [2, 3])
def test_tcrdist_thresholds_and_exhaustive_rows(xtn, d):
    # the retention experiment: SymDel(d) rows filtered at several TCRdist
    # thresholds equal the all-pairs scorer restricted to Lev <= d; filtering
    # every pair gives the exhaustive TCRdist neighbours
    seqs, off = gen.workload(gen.TCRDIST_1M, 2000)
    lev = _rows(xtn.search_self(seqs, off, d))
    n = off.size - 1
    ii, jj = np.triu_indices(n, 1)
    every = np.stack([ii, jj, np.zeros_like(ii)], 1).astype(np.uint32)
    for t in (12, 24, 36):
        got = _rows(xtn.tcrdist_filter(seqs, off, lev, t))
        want = oracle.tcrdist_allpairs(seqs, off, d, t)
        assert np.array_equal(got, want[:, :3]), (d, t)
        exh = _rows(xtn.tcrdist_filter(seqs, off, every, t))
        want_exh = oracle.tcrdist_allpairs(seqs, off, 25, t)
        assert np.array_equal(exh[:, :2], want_exh[:, :2]), (d, t)


def test_tcrdist_every_residue_pair(xtn):
    # one pair per ordered residue pair (a, b) at the same position: covers
    # every BLOSUM62 entry the score uses.
    aa = gen.AA
    strs = []
    for a in aa:
        for b in aa:
            strs += ["CAS" + a + "GF", "CAS" + b + "GF"]
    seqs, off = gen.from_strings(strs)
    rows = np.array([[2 * k, 2 * k + 1, 1] for k in range(len(strs) // 2)], np.uint32)
    for thr in [0, 3, 6, 9, 12, 24]:
        got = _rows(xtn.tcrdist_filter(seqs, off, rows, thr))
        assert np.array_equal(got, oracle.tcrdist_filter(seqs, off, rows, thr)), thr


# ------------------------------------------------------ search in passes ---
def _variant_records(off, d):
    # deletion subsets of <= d positions (canonical ones are fewer): budgets
    # below are fractions of this, and each test checks the passes it ran
    L = np.diff(off).astype(np.int64)
    return int((1 + L + (L * (L - 1) // 2 if d >= 2 else 0)).sum())


@pytest.mark.parametrize("d,metric", [(1, "levenshtein"), (2, "levenshtein"), (2, "hamming")])
def test_streaming_matches_oracle(xtn, d, metric):
    seqs, off = gen.workload(gen.SELF_1M, 20_000)
    want = oracle.symdel_self(seqs, off, d, metric)
    budget = _variant_records(off, d) // 12
    rows, passes = xtn.search_self_streaming(seqs, off, d, metric=metric, max_pass_records=budget)
    assert passes >= 4
    assert np.array_equal(_rows(rows), want)


def test_streaming_batched_and_between(xtn):
    n = 20_000
    seqs, off = gen.workload(gen.SELF_1M, n)
    cuts = np.sort(np.random.default_rng(45).choice(np.arange(1, n), 5, replace=False))
    rep = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    budget = _variant_records(off, 2) // 10
    rows, passes = xtn.search_self_streaming(seqs, off, 2, rep_offsets=rep, between=True,
                                             max_pass_records=budget)
    assert passes >= 4
    assert np.array_equal(_rows(rows), oracle.symdel_cross(seqs, off, rep, 2))
    rows, _ = xtn.search_self_streaming(seqs, off, 2, rep_offsets=rep, max_pass_records=budget)
    got = _rows(rows)
    want = oracle.symdel_batched(seqs, off, rep, 2)
    rep_of = np.searchsorted(rep, got[:, 0], side="right") - 1
    local = np.stack([rep_of, got[:, 0] - rep[rep_of], got[:, 1] - rep[rep_of], got[:, 2]], 1)
    assert np.array_equal(local.astype(np.uint32), want)


def test_streaming_d3_and_small_alphabet(xtn):
    seqs, off = gen.workload(gen.SELF_1M, 3_000)
    rows, passes = xtn.search_self_streaming(seqs, off, 3, max_pass_records=200_000)
    assert passes >= 4
    assert np.array_equal(_rows(rows), oracle.symdel_self(seqs, off, 3))
    # two letters: buckets far larger than shared memory, repeated residues,
    # one bin per pass at the smallest budget
    strs = _rand_strings(np.random.default_rng(71), 3000, "AC", 0, 10)
    s2, o2 = gen.from_strings(strs)
    want = oracle.bruteforce_self(s2, o2, 2)
    for budget in (1, 2_000, 10_000):
        rows, passes = xtn.search_self_streaming(s2, o2, 2, max_pass_records=budget)
        assert passes >= 2
        assert np.array_equal(_rows(rows), want)


def test_streaming_edge_cases(xtn):
    # empty input, one sequence, empty strings, maximum length, repeats, and
    # d = 0, each at a budget of one record per pass (one bin per pass)
    seqs, off = gen.from_strings([])
    rows, passes = xtn.search_self_streaming(seqs, off, 2, max_pass_records=1)
    assert rows.shape[0] == 0 and passes == 0
    for strs, d in [(["CASSF"], 2), (["", "", "A"], 1), (["W" * 25, "W" * 24, "Y" * 25], 1),
                    (["A" * 25, "A" * 24], 3), (["CASSF", "CASSF", "CAS", "", ""], 0),
                    (["ACDEFGHIKLMNPQRSTVWYACDEF", "CDEFGHIKLMNPQRSTVWYACDEFA"], 2)]:
        seqs, off = gen.from_strings(strs)
        rows, passes = xtn.search_self_streaming(seqs, off, d, max_pass_records=1)
        assert passes >= 1
        assert np.array_equal(_rows(rows), oracle.bruteforce_self(seqs, off, d)), strs


def test_streaming_1m_equals_one_pass(xtn):
    seqs, off = gen.workload(gen.SELF_1M)
    ds, do = _dev(seqs, off)
    whole = _rows(xtn.search_self(ds, do, 2))
    rows, passes = xtn.search_self_streaming(ds, do, 2, max_pass_records=30_000_000)
    assert passes >= 4
    assert np.array_equal(_rows(rows), whole)
    rows, passes = xtn.search_self_streaming(ds, do, 2)
    assert passes == 1 and np.array_equal(_rows(rows), whole)


# ------------------------------------------------------ bounded waits ---
def test_bounded_wait_gives_up_and_reports(xtn):
    # With a poll limit of one, look-back waits on tiles whose predecessors
    # are still running give up: the call reports XTN_ERR_DEVICE_TIMEOUT
    # instead of waiting (indices computed from the incomplete sums are
    # range-checked, so nothing is written out of bounds).  With the default
    # limit restored, the next calls give the exact rows again.
    from paper_2403_09010_gb300 import native
    seqs, off = gen.workload(gen.SELF_1M)
    ds, do = _dev(seqs, off)
    whole = _rows(xtn.search_self(ds, do, 2))
    statuses = []
    xtn.set_wait_limit(1)
    try:
        for _ in range(3):
            try:
                got = _rows(xtn.search_self(ds, do, 2))
                statuses.append(native.XTN_OK)
                assert np.array_equal(got, whole)     # no wait gave up: exact rows
            except native.XtnError as e:
                statuses.append(e.status)
    finally:
        xtn.set_wait_limit(0)
    assert native.XTN_ERR_DEVICE_TIMEOUT in statuses, statuses
    assert set(statuses) <= {native.XTN_OK, native.XTN_ERR_DEVICE_TIMEOUT}, statuses
    assert np.array_equal(_rows(xtn.search_self(ds, do, 2)), whole)
    small_s, small_o = gen.workload(gen.SELF_1M, 20_000)
    assert np.array_equal(_rows(xtn.search_self(small_s, small_o, 2)),
                          oracle.symdel_self(small_s, small_o, 2))


# --------------------------------------------------------- paired chains ---
@pytest.mark.parametrize("d", [0, 1, 2])
def test_paired_matches_oracle(xtn, d):
    a, ao, b, bo = gen.paired(6_000, 80 + d)
    want = oracle.symdel_paired(a, ao, b, bo, d)
    got = _rows(xtn.search_paired(a, ao, b, bo, d))
    assert got.shape == want.shape and np.array_equal(got, want)
    if d >= 1:
        assert want.shape[0] > 100
    # device inputs give the same rows
    da, dao = _dev(a, ao)
    db, dbo = _dev(b, bo)
    assert np.array_equal(_rows(xtn.search_paired(da, dao, db, dbo, d)), want)


def test_paired_small_alphabet_and_edges(xtn):
    rng = np.random.default_rng(83)
    a = _rand_strings(rng, 700, "AC", 0, 6)
    b = _rand_strings(rng, 700, "AC", 0, 6)
    sa, oa = gen.from_strings(a)
    sb, ob = gen.from_strings(b)
    for d in (0, 1, 2):
        assert np.array_equal(_rows(xtn.search_paired(sa, oa, sb, ob, d)),
                              oracle.bruteforce_paired(sa, oa, sb, ob, d)), d
    # longest chains, empty chains, a receptor repeated many times
    strs_a = ["W" * 25, "W" * 24, "", "", "CASSF"] + ["CAVF"] * 300
    strs_b = ["Y" * 25, "Y" * 25, "", "A", ""] + ["CASSF"] * 300
    sa, oa = gen.from_strings(strs_a)
    sb, ob = gen.from_strings(strs_b)
    for d in (1, 2):
        assert np.array_equal(_rows(xtn.search_paired(sa, oa, sb, ob, d)),
                              oracle.bruteforce_paired(sa, oa, sb, ob, d)), d


def test_paired_with_empty_second_chains_is_the_self_search(xtn):
    seqs, off = gen.workload(gen.SELF_1M, 30_000)
    empty = np.zeros(0, np.uint8)
    zero = np.zeros(off.size, np.int64)
    assert np.array_equal(_rows(xtn.search_paired(seqs, off, empty, zero, 2)),
                          _rows(xtn.search_self(seqs, off, 2)))


def test_paired_rejects_bad_arguments(xtn):
    from paper_2403_09010_gb300 import native
    a, ao, b, bo = gen.paired(50, 9)
    with pytest.raises(native.XtnError) as ei:
        xtn.search_paired(a, ao, b, bo, 3)
    assert ei.value.status == native.XTN_ERR_INVALID_ARG
    bad = b.copy()
    bad[0] = ord("X")
    with pytest.raises(native.XtnError) as ei:
        xtn.search_paired(a, ao, bad, bo, 1)
    assert ei.value.status == native.XTN_ERR_BAD_RESIDUE


# ------------------------------------------------------------- profiler ---
def test_profiler_times_every_kernel_or_only_the_named_one(xtn):
    """xtn_profile_enable brackets every launch with events, tagged with its
    algorithmic bytes; xtn_profile_only restricts that to one kernel name."""
    seqs, off = gen.workload(gen.SELF_1M, 50_000)
    ds, do = _dev(seqs, off)
    want = _rows(xtn.search_self(ds, do, 2))
    xtn.profile_report()
    try:
        xtn.profile_enable(True)
        got = _rows(xtn.search_self(ds, do, 2))
        every = xtn.profile_report()
        xtn.profile_only("k_onesweep_records")
        xtn.search_self(ds, do, 2)
        only = xtn.profile_report()
    finally:
        xtn.profile_enable(False)
        xtn.profile_only(None)
    assert np.array_equal(got, want)
    kernels = {k: v for k, v in every.items() if not k.startswith("host_")}
    for name in ("k_encode", "k_expand", "k_onesweep_records", "k_bucket_filter",
                 "k_verify_candidates", "k_onesweep_pairs", "k_unique_finalize"):
        assert name in kernels, name
        launches, ms, nbytes = kernels[name]
        assert launches >= 1 and ms > 0 and nbytes > 0
    assert "host_call_search_self" in every
    assert set(only) == {"k_onesweep_records"}
    assert only["k_onesweep_records"][0] == kernels["k_onesweep_records"][0]
    # 16 algorithmic bytes per record and pass
    n_rec = only["k_onesweep_records"][2] / 16 / only["k_onesweep_records"][0]
    assert n_rec == int(n_rec) and n_rec > 50_000
