"""The seeded synthetic inputs have the stated shape and are reproducible."""
import numpy as np

import cdr3_synth as gen


def test_reproducible_and_shaped():
    a = gen.generate(20_000, 9, 0.15, 0.01)
    b = gen.generate(20_000, 9, 0.15, 0.01)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    seqs, off = a
    L = np.diff(off)
    assert L.min() >= 6 and L.max() <= 24
    assert 14.0 < L.mean() < 15.0
    strs = gen.to_strings(seqs, off)
    assert set("".join(strs)) <= set(gen.AA)
    assert 0.85 < np.mean([s[:3] == "CAS" for s in strs]) ** (1 / 3) < 0.95
    assert 0.85 < np.mean([s[-1] == "F" for s in strs]) < 0.95
    # about 1% exact copies of earlier sequences
    dup = len(strs) - len(set(strs))
    assert 0.005 * len(strs) < dup < 0.03 * len(strs)


def test_batched_and_served_shapes():
    seqs, off, rep = gen.batched(n_rep=6, size_min=100, size_max=2000)
    assert rep[0] == 0 and rep[-1] == off.size - 1 and np.all(np.diff(rep) >= 100)
    rs, ro, reqs = gen.served(ref_n=5000, n_req=20, max_req=300)
    assert ro.size == 5001 and len(reqs) == 20
    assert all(1 <= r.offsets.size - 1 <= 300 for r in reqs)
    assert all(reqs[k].arrival_s < reqs[k + 1].arrival_s for k in range(19))


def test_from_to_strings_roundtrip():
    strs = ["", "A", "CASSF", "W" * 25]
    assert gen.to_strings(*gen.from_strings(strs)) == strs
