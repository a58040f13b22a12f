"""Served mode on the GPU: a resident reference index, requests replayed on a
Poisson arrival process through the continuous-batching server; every
request's rows are identical alone and in the mix (and to the oracle)."""
import numpy as np
import pytest

import cdr3_synth as gen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_served_results_identical_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2403_09010_gb300 as xtn
    from paper_2403_09010_gb300 import serve
    xtn.build()
    rs, ro, reqs = gen.served(ref_n=60_000, n_req=60, max_req=2000, rate=2000.0, seed=21)
    idx = xtn.index_build(rs, ro, 2)
    srv = serve.Server(idx, slots=3)
    pend = serve.replay(srv, reqs)
    srv.close()
    st = srv.stats(pend)
    assert st["requests"] == len(reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert st["max_requests_per_batch"] > 1        # continuous batching happened
    assert st["peak_batches_in_flight"] > 1        # micro-batches overlapped on the GPU
    for r, p in zip(reqs, pend):
        alone = xtn.search_query(idx, r.seqs, r.offsets).astype(np.uint32)
        assert np.array_equal(p.rows, alone), r.rid
    for r, p in list(zip(reqs, pend))[:4]:
        assert np.array_equal(p.rows, oracle.symdel_query(rs, ro, r.seqs, r.offsets, 2))
    idx.free()
