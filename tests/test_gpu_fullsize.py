"""The full-size workloads against the CPU oracle, in the launch configuration
the benchmark uses (device-resident inputs, default or autotuned knobs).

* 1,000,000 sequences at d <= 2: every row against the oracle's SymDel
  search with its variant keys split over all host threads.
* 256 repertoires of log-uniform size (8.96M sequences, d <= 2) through the
  autotuned plan: the rows of five repertoires (the smallest, the largest
  and three others) against the oracle's search of each repertoire alone.
* A 10,000,000-sequence resident reference index (d <= 2): small requests,
  alone and inside a continuous-batching mix, against exhaustive comparison
  with all ten million references.
* 9,000,000 sequences at d <= 3, past 2^32 deletion records (searched in
  passes): the complete neighbour lists of sampled sequences against
  exhaustive comparison with all nine million sequences.

Rows are compared element by element: (i, j, dist) integers, bit-exact.
"""
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
    oracle.build()
    return pkg


def _rows(x):
    if isinstance(x, np.ndarray):
        return x.astype(np.uint32)
    return x.cpu().numpy().astype(np.uint32)


def _dev(seqs, off):
    return (torch.from_numpy(np.ascontiguousarray(seqs)).cuda(),
            torch.from_numpy(np.ascontiguousarray(off)).cuda())


def _neighbour_lists(rows, samples):
    """For each sampled index s, its (other, dist) rows sorted by other."""
    i, j, dist = rows[:, 0], rows[:, 1], rows[:, 2]
    out = {}
    for s in samples:
        m = (i == s) | (j == s)
        other = np.where(i[m] == s, j[m], i[m])
        got = np.stack([other, dist[m]], 1).astype(np.uint32)
        out[int(s)] = got[np.argsort(got[:, 0], kind="stable")]
    return out


def test_selfsearch_n1e6_d2_every_row(xtn):
    seqs, off = gen.workload(gen.SELF_1M)
    ds, do = _dev(seqs, off)
    got = _rows(xtn.search_self(ds, do, 2))
    want = oracle.symdel_self_sharded(seqs, off, 2, threads=0)
    assert want.shape[0] > 250_000
    assert got.shape == want.shape and np.array_equal(got, want)


def test_batched_256_repertoires_sampled_against_oracle(xtn):
    from paper_2403_09010_gb300 import autotune
    seqs, off, rep = gen.batched()
    assert rep.size - 1 == 256
    ds = torch.from_numpy(seqs).cuda()
    tuned = autotune.tune(ds, off, gen.BATCH_D, rep_offsets=rep, repeats=1, use_cache=False)
    plan = xtn.Plan(off, gen.BATCH_D, rep_offsets=rep, tuning=tuned)
    plan.run(ds)
    got = _rows(plan.result(like=ds))
    plan.free()
    sizes = np.diff(rep)
    rng = np.random.default_rng(256)
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    picks |= set(int(r) for r in rng.choice(256, 3, replace=False))
    rep_of = np.searchsorted(rep, got[:, 0], side="right") - 1
    assert np.array_equal(np.searchsorted(rep, got[:, 1], side="right") - 1, rep_of)
    for r in sorted(picks):
        a, b = int(rep[r]), int(rep[r + 1])
        mine = got[rep_of == r].astype(np.int64)
        mine[:, :2] -= a
        want = oracle.symdel_self_sharded(seqs[off[a]:off[b]], off[a:b + 1] - off[a],
                                          gen.BATCH_D, threads=0)
        assert np.array_equal(mine.astype(np.uint32), want), r


def test_served_ref1e7_small_requests_against_oracle(xtn):
    from paper_2403_09010_gb300 import serve
    rs, ro, reqs = gen.served()
    idx = xtn.index_build(rs, ro, 2)
    small = [r for r in reqs if r.offsets.size - 1 <= 20][:6]
    assert len(small) == 6
    # the small requests inside a mix with the requests that arrived first
    mix = sorted({r.rid for r in reqs[:24]} | {r.rid for r in small})
    mix = [reqs[k] for k in mix]
    srv = serve.Server(idx, slots=4)
    pend = serve.replay(srv, mix)
    srv.close()
    in_mix = {r.rid: p.rows for r, p in zip(mix, pend)}
    # one exhaustive pass of all small requests' queries over the reference
    q_s, q_o = gen.concat([r.seqs for r in small], [r.offsets for r in small])
    want = oracle.bruteforce_query(rs, ro, q_s, q_o, 2, threads=0)
    first = np.concatenate([[0], np.cumsum([r.offsets.size - 1 for r in small])])
    for k, r in enumerate(small):
        part = want[(want[:, 0] >= first[k]) & (want[:, 0] < first[k + 1])].copy()
        part[:, 0] -= np.uint32(first[k])
        alone = _rows(xtn.search_query(idx, r.seqs, r.offsets))
        assert np.array_equal(alone, part), r.rid
        assert np.array_equal(_rows(in_mix[r.rid]), part), r.rid
    assert want.shape[0] > 0
    idx.free()


def test_beyond_2_32_records_sampled_against_oracle(xtn):
    # 9M sequences at d <= 3 give about 5e9 deletion records: the search runs
    # in passes.  Sampled sequences' complete neighbour lists are compared
    # with exhaustive comparison against every one of the nine million.
    n = 9_000_000
    seqs, off = gen.generate(n, 17, 0.15, 0.01)
    ds, do = _dev(seqs, off)
    rows, passes = xtn.search_self_streaming(ds, do, 3)
    assert passes >= 2
    got = _rows(rows)
    assert np.all(got[:, 0] < got[:, 1]) and np.all(got[:, 2] <= 3)
    key = got[:, 0].astype(np.uint64) << np.uint64(32) | got[:, 1].astype(np.uint64)
    assert np.all(np.diff(key.astype(np.int64)) > 0)
    rng = np.random.default_rng(6)
    samples = np.sort(rng.choice(n, 8, replace=False))
    q_s, q_o = gen.concat([seqs[off[s]:off[s + 1]] for s in samples],
                          [off[s:s + 2] - off[s] for s in samples])
    want = oracle.bruteforce_query(seqs, off, q_s, q_o, 3, threads=0)
    mine = _neighbour_lists(got, samples)
    total = 0
    for k, s in enumerate(samples):
        w = want[(want[:, 0] == k) & (want[:, 1] != s)][:, 1:]
        assert np.array_equal(mine[int(s)], w), int(s)
        total += w.shape[0]
    assert total > 0
    # rows among the first 1M sequences are those of the one-pass search of
    # that prefix (under 2^32 records)
    m = 1_000_000
    prefix = _rows(xtn.search_self(ds[: int(off[m])], do[: m + 1], 3))
    assert np.array_equal(got[got[:, 1] < m], prefix)
    # the one-shot call takes the same passes past 2^32 records
    assert np.array_equal(_rows(xtn.search_self(ds, do, 3)), got)
