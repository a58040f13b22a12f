"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* worked numbers printed in the paper (Sec. 2.1, tests/golden/paper_counts.txt);
* textbook edit distances and an exhaustive edit-ball enumeration (BFS over
  single edits, independent of any dynamic programming);
* exhaustive all-pairs search (the plain definition) on many random inputs;
* the SymDel guarantee of Sec. 2.1 (within distance d => a shared deletion
  variant with <= d deletions each) and its converse bound (a shared variant
  => distance <= 2d, Fig. 1D);
* special cases: d = 0 is exact-duplicate grouping, identical inputs give all
  n(n-1)/2 pairs at distance 0, d >= every length gives every pair;
* the bag-of-amino-acids bound of Appendix B on every output pair;
* hand-worked TCRdist scores (tests/golden/tcrdist_hand.txt) and BLOSUM62
  consistency checks;
* paired chains joined by a token no edit may touch (Discussion): hand-worked
  distances (tests/golden/paired_hand.txt), a BFS over the admissible edits,
  the split into the two chains' edit distances, variant counts, SymDel
  against exhaustive search, and the special case of empty second chains.
"""
import itertools
import math
import os
import random

import numpy as np
import pytest

import cdr3_synth as gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
AA = gen.AA


def _edits1(s, alphabet):
    out = set()
    for i in range(len(s) + 1):
        for c in alphabet:
            out.add(s[:i] + c + s[i:])
    for i in range(len(s)):
        out.add(s[:i] + s[i + 1:])
        for c in alphabet:
            if c != s[i]:
                out.add(s[:i] + c + s[i + 1:])
    return out


def _ball_levels(s, radius, alphabet):
    """{t: minimal number of single edits from s to t} for t within radius (BFS)."""
    dist = {s: 0}
    frontier = {s}
    for r in range(1, radius + 1):
        nxt = set()
        for t in frontier:
            nxt |= _edits1(t, alphabet)
        nxt -= dist.keys()
        for t in nxt:
            dist[t] = r
        frontier = nxt
    return dist


def _deletions(s, d):
    out, cur = {s}, {s}
    for _ in range(d):
        cur = {t[:i] + t[i + 1:] for t in cur for i in range(len(t))}
        out |= cur
    return out


def _rand_strings(rng, n, alphabet, lmin, lmax):
    return ["".join(rng.choice(alphabet) for _ in range(rng.randint(lmin, lmax))) for _ in range(n)]


# ------------------------------------------------------------------ paper ---
def test_paper_worked_counts():
    rows = [l.split("#")[0].split() for l in open(os.path.join(GOLDEN, "paper_counts.txt"))]
    rows = [r for r in rows if r]
    assert rows
    for s, d, n_var, n_ball in rows:
        d, n_var, n_ball = int(d), int(n_var), int(n_ball)
        assert oracle.count_variants(s, d) == n_var
        assert len(_deletions(s, d)) == n_var
        ball = _ball_levels(s, d, AA)
        assert len(ball) == n_ball
        # every string of the ball is within d by the oracle's DP, at its BFS level
        sample = random.Random(0).sample(sorted(ball), 3000)
        for t in sample:
            assert oracle.levenshtein(s, t) == ball[t]


def test_repeat_counts_shrink():
    # Sec. 2.1 / Fig. 1C: repeats make deletion variants coincide.
    assert oracle.count_variants("AAAAAAAAAA", 2) == 3
    assert oracle.count_variants("", 2) == 1
    assert oracle.count_variants("AB", 5) == 4          # AB, A, B, ""


# ------------------------------------------------------------ levenshtein ---
@pytest.mark.parametrize("a,b,dist", [
    ("kitten", "sitting", 3), ("flaw", "lawn", 2), ("", "abc", 3), ("abc", "", 3),
    ("", "", 0), ("CASSF", "CASSF", 0), ("intention", "execution", 5),
    ("saturday", "sunday", 3), ("AB", "BA", 2), ("ABC", "CAB", 2),
])
def test_levenshtein_textbook(a, b, dist):
    assert oracle.levenshtein(a, b) == dist
    assert oracle.levenshtein(b, a) == dist


def test_levenshtein_matches_edit_ball():
    rng = random.Random(1)
    for s in ["", "A", "ACA", "CCAD", "DACAC"]:
        ball = _ball_levels(s, 3, "ACD")
        for t, lvl in ball.items():
            assert oracle.levenshtein(s, t) == lvl, (s, t)
        # strings outside the radius-3 ball are farther than 3
        for t in _rand_strings(rng, 200, "ACD", 0, 8):
            if t not in ball:
                assert oracle.levenshtein(s, t) > 3


def test_levenshtein_metric_axioms():
    rng = random.Random(2)
    strs = _rand_strings(rng, 40, "ACDE", 0, 9)
    for a, b, c in itertools.islice(itertools.product(strs, repeat=3), 4000):
        ab, bc, ac = oracle.levenshtein(a, b), oracle.levenshtein(b, c), oracle.levenshtein(a, c)
        assert ac <= ab + bc
        assert abs(len(a) - len(b)) <= ab <= max(len(a), len(b))
        assert (ab == 0) == (a == b)


# ------------------------------------------------- SymDel vs exhaustive ---
def _check_self(strs, d):
    seqs, off = gen.from_strings(strs)
    got = oracle.symdel_self(seqs, off, d)
    ref = oracle.bruteforce_self(seqs, off, d)
    assert np.array_equal(got, ref)
    # independent check of a sample of rows with the pure-Python ball
    return got


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_symdel_equals_bruteforce_small_alphabet(d):
    rng = random.Random(10 + d)
    strs = _rand_strings(rng, 250, "AC", 0, 8)
    _check_self(strs, d)


@pytest.mark.parametrize("d", [1, 2])
def test_symdel_equals_bruteforce_generator(d):
    seqs, off = gen.generate(1500, 100 + d, 0.3, 0.02)
    assert np.array_equal(oracle.symdel_self(seqs, off, d), oracle.bruteforce_self(seqs, off, d))


def test_symdel_rows_are_canonical():
    seqs, off = gen.generate(800, 7, 0.3, 0.05)
    rows = oracle.symdel_self(seqs, off, 2)
    assert rows.shape[1] == 3 and rows.shape[0] > 0
    assert np.all(rows[:, 0] < rows[:, 1])
    keys = rows[:, 0].astype(np.int64) * len(off) + rows[:, 1]
    assert np.all(np.diff(keys) > 0)                      # sorted, unique
    strs = gen.to_strings(seqs, off)
    for i, j, dist in rows[:200]:
        assert oracle.levenshtein(strs[i], strs[j]) == dist <= 2


def test_symdel_guarantee_and_converse():
    rng = random.Random(3)
    for _ in range(300):
        a = "".join(rng.choice("ACDG") for _ in range(rng.randint(1, 10)))
        b = a
        d = rng.randint(0, 3)
        for _ in range(rng.randint(0, d)):
            b = rng.choice(sorted(_edits1(b, "ACDG")))
        lev = oracle.levenshtein(a, b)
        assert lev <= d
        # within d => a shared variant with <= d deletions on each side
        assert _deletions(a, d) & _deletions(b, d)
        # shared variant with k1, k2 <= d deletions => lev <= 2d
        c = "".join(rng.choice("ACDG") for _ in range(rng.randint(1, 10)))
        if _deletions(a, d) & _deletions(c, d):
            assert oracle.levenshtein(a, c) <= 2 * d


def test_special_case_d0_is_duplicate_grouping():
    rng = random.Random(4)
    strs = _rand_strings(rng, 300, "AC", 1, 4)
    seqs, off = gen.from_strings(strs)
    got = oracle.symdel_self(seqs, off, 0)
    want = sorted((i, j, 0) for i in range(len(strs)) for j in range(i + 1, len(strs))
                  if strs[i] == strs[j])
    assert [tuple(r) for r in got.tolist()] == want


def test_special_case_identical_inputs():
    n = 60
    seqs, off = gen.from_strings(["CASSLGQETQYF"] * n)
    got = oracle.symdel_self(seqs, off, 2)
    assert got.shape[0] == n * (n - 1) // 2
    assert np.all(got[:, 2] == 0)


def test_special_case_d_covers_every_length():
    rng = random.Random(5)
    strs = _rand_strings(rng, 40, "ACDEFG", 0, 4)
    seqs, off = gen.from_strings(strs)
    got = oracle.symdel_self(seqs, off, 4)
    assert got.shape[0] == 40 * 39 // 2
    for i, j, dist in got:
        assert dist == oracle.levenshtein(strs[i], strs[j])


def test_bag_of_amino_acids_bound():
    seqs, off = gen.generate(1200, 11, 0.3, 0.02)
    strs = gen.to_strings(seqs, off)
    rows = oracle.symdel_self(seqs, off, 2)
    assert rows.shape[0] > 0
    for i, j, dist in rows:
        ca = np.array([strs[i].count(c) for c in AA])
        cb = np.array([strs[j].count(c) for c in AA])
        assert np.linalg.norm(ca - cb) <= math.sqrt(2) * dist + 1e-12


# ------------------------------------------------------- query / batched ---
@pytest.mark.parametrize("d", [1, 2])
def test_query_equals_bruteforce(d):
    rs, ro = gen.generate(1200, 20 + d, 0.2, 0.01)
    qs, qo = gen.generate(300, 30 + d, 0.2, 0.0)
    # plant some near copies of reference entries among the queries
    strs = gen.to_strings(qs, qo) + gen.to_strings(rs, ro)[:50]
    qs, qo = gen.from_strings(strs)
    got = oracle.symdel_query(rs, ro, qs, qo, d)
    ref = oracle.bruteforce_query(rs, ro, qs, qo, d)
    assert np.array_equal(got, ref)
    assert got.shape[0] >= 50


def test_batched_is_per_repertoire_self_search():
    parts = [gen.generate(n, 40 + k, 0.3, 0.02) for k, n in enumerate([0, 1, 200, 57, 400])]
    seqs, off = gen.concat([p[0] for p in parts], [p[1] for p in parts])
    rep_off = np.concatenate([[0], np.cumsum([p[1].size - 1 for p in parts])])
    got = oracle.symdel_batched(seqs, off, rep_off, 2)
    want = []
    for r, (s, o) in enumerate(parts):
        for row in oracle.bruteforce_self(s, o, 2).tolist():
            want.append([r] + row)
    assert got.tolist() == sorted(want)


# ---------------------------------------------------------------- TCRdist ---
def test_blosum62_consistency():
    for a in AA:
        assert 4 <= oracle.blosum62(a, a) <= 11
        for b in AA:
            assert oracle.blosum62(a, b) == oracle.blosum62(b, a)
            if a != b:
                assert -4 <= oracle.blosum62(a, b) <= 3
    # well-known entries of the published matrix
    assert oracle.blosum62("W", "W") == 11 and oracle.blosum62("C", "C") == 9
    assert oracle.blosum62("I", "V") == 3 and oracle.blosum62("F", "Y") == 3


def test_tcrdist_hand_worked():
    rows = [l.split("#")[0].split() for l in open(os.path.join(GOLDEN, "tcrdist_hand.txt"))]
    rows = [r for r in rows if r]
    assert len(rows) >= 5
    for a, b, score in rows:
        assert oracle.tcrdist(a, b) == int(score), (a, b)
        assert oracle.tcrdist(b, a) == int(score), (b, a)


def test_tcrdist_properties():
    rng = random.Random(6)
    strs = _rand_strings(rng, 60, AA, 4, 12)
    for a in strs:
        assert oracle.tcrdist(a, a) == 0
        for b in strs[:20]:
            s = oracle.tcrdist(a, b)
            assert s % 3 == 0
            g = abs(len(a) - len(b))
            m = min(len(a), len(b))
            assert 12 * g <= s <= 3 * (4 * m + 4 * g)


def test_tcrdist_filter_and_allpairs_agree():
    seqs, off = gen.generate(1000, 12, 0.3, 0.02)
    lev = oracle.symdel_self(seqs, off, 2)
    kept = oracle.tcrdist_filter(seqs, off, lev, 24)
    allp = oracle.tcrdist_allpairs(seqs, off, 2, 24)
    assert np.array_equal(kept, allp[:, :3])
    strs = gen.to_strings(seqs, off)
    for i, j, _, score in allp:
        assert oracle.tcrdist(strs[i], strs[j]) == score <= 24


# ----------------------------------------------------------------- Hamming ---
# The Hamming variant (Results, comparison with CompAIRR): the same SymDel
# steps, with the last one filtering by Hamming distance.
@pytest.mark.parametrize("a, b, dist", [("KAROLIN", "KATHRIN", 3), ("CASSF", "CASSF", 0),
                                        ("ACDE", "WYKL", 4), ("", "", 0)])
def test_hamming_textbook(a, b, dist):
    assert oracle.hamming(a, b) == dist


def test_hamming_unequal_lengths_are_never_neighbours():
    assert oracle.hamming("CASS", "CAS") == -1
    seqs, off = gen.from_strings(["CASS", "CAS", "CASSS"])
    assert oracle.bruteforce_self(seqs, off, 3, "hamming").shape[0] == 0
    assert oracle.symdel_self(seqs, off, 3, "hamming").shape[0] == 0
    # ... while CASS, one deletion from each of the others, has two
    # Levenshtein neighbours at d = 1 (CAS and CASSS are two apart)
    assert oracle.symdel_self(seqs, off, 1).shape[0] == 2


def test_hamming_is_at_least_levenshtein():
    rng = random.Random(77)
    for _ in range(300):
        L = rng.randint(0, 10)
        a = "".join(rng.choice("ACD") for _ in range(L))
        b = "".join(rng.choice("ACD") for _ in range(L))
        h, lev = oracle.hamming(a, b), oracle.levenshtein(a, b)
        assert h == sum(x != y for x, y in zip(a, b))
        assert lev <= h


def test_hamming_ball_closed_form():
    # all strings of length 4 over {A, C, D}: the ball of radius k around one
    # of them holds sum_{i <= k} C(4, i) 2^i strings
    alphabet = "ACD"
    strs = ["".join(t) for t in itertools.product(alphabet, repeat=4)]
    centre = strs.index("ACDA")
    seqs, off = gen.from_strings(strs)
    for d in range(4):
        rows = oracle.bruteforce_self(seqs, off, d, "hamming")
        mine = rows[(rows[:, 0] == centre) | (rows[:, 1] == centre)]
        assert mine.shape[0] == sum(math.comb(4, i) * 2 ** i for i in range(1, d + 1))
        assert np.array_equal(rows, oracle.symdel_self(seqs, off, d, "hamming"))


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_hamming_symdel_equals_bruteforce(d):
    rng = random.Random(40 + d)
    strs = _rand_strings(rng, 300, "AC", 0, 9)
    seqs, off = gen.from_strings(strs)
    want = oracle.bruteforce_self(seqs, off, d, "hamming")
    assert np.array_equal(oracle.symdel_self(seqs, off, d, "hamming"), want)
    g_seqs, g_off = gen.generate(1200, 300 + d, 0.3, 0.02)
    assert np.array_equal(oracle.symdel_self(g_seqs, g_off, d, "hamming"),
                          oracle.bruteforce_self(g_seqs, g_off, d, "hamming"))


def test_hamming_batched_is_per_repertoire():
    seqs, off, rep = gen.batched(n_rep=5, seed=12, size_min=50, size_max=400)
    got = oracle.symdel_batched(seqs, off, rep, 2, "hamming")
    parts = []
    for r in range(rep.size - 1):
        lo, hi = rep[r], rep[r + 1]
        s, o = gen.from_strings(gen.to_strings(seqs, off)[lo:hi])
        rows = oracle.bruteforce_self(s, o, 2, "hamming")
        parts.append(np.column_stack([np.full(rows.shape[0], r, np.uint32), rows]))
    assert np.array_equal(got, np.concatenate(parts))


# ---------------------------------------------------- between repertoires ---
@pytest.mark.parametrize("metric", ["levenshtein", "hamming"])
def test_cross_and_within_partition_the_whole_search(metric):
    # every pair of the concatenation lies within one repertoire or between two
    # one generated set cut into repertoires: its near-copies cross the cuts
    seqs, off = gen.workload(gen.SELF_1M, 1500)
    rep = np.array([0, 200, 210, 700, 1100, 1500], dtype=np.int64)
    whole = oracle.bruteforce_self(seqs, off, 2, metric)
    cross = oracle.symdel_cross(seqs, off, rep, 2, metric)
    within = oracle.symdel_batched(seqs, off, rep, 2, metric)
    glob = np.stack([within[:, 1] + rep[within[:, 0]], within[:, 2] + rep[within[:, 0]],
                     within[:, 3]], 1).astype(np.uint32)
    both = np.concatenate([cross, glob])
    both = both[np.lexsort((both[:, 1], both[:, 0]))]
    assert np.array_equal(both, whole)
    r_of = lambda i: np.searchsorted(rep, i, side="right") - 1
    assert np.all(r_of(cross[:, 0]) != r_of(cross[:, 1]))
    assert cross.shape[0] >= 10 and within.shape[0] >= 10


# ------------------------------------------------------ sharded oracle ---
@pytest.mark.parametrize("metric", ["levenshtein", "hamming"])
def test_sharded_search_is_the_brute_force(metric):
    # keys split over threads: any thread count gives the brute-force rows
    rng = np.random.default_rng(90)
    strs = ["".join(rng.choice(list("ACD"), size=k)) for k in rng.integers(0, 9, 400)]
    seqs, off = gen.from_strings(strs)
    want = oracle.bruteforce_self(seqs, off, 2, metric)
    assert want.shape[0] > 100
    for threads in (1, 2, 3, 7):
        assert np.array_equal(oracle.symdel_self_sharded(seqs, off, 2, metric, threads), want)
    seqs, off = gen.workload(gen.SELF_1M, 2_000)
    assert np.array_equal(oracle.symdel_self_sharded(seqs, off, 2, metric, 4),
                          oracle.bruteforce_self(seqs, off, 2, metric))


@pytest.mark.parametrize("d", [1, 2])
def test_hamming_query_equals_bruteforce(d):
    rs, ro = gen.generate(1200, 60 + d, 0.2, 0.01)
    strs = gen.to_strings(rs, ro)
    # one substitution in 60 reference entries, plus fresh queries
    subst = [s[:2] + ("W" if s[2] != "W" else "Y") + s[3:] for s in strs[:60] if len(s) > 3]
    qs, qo = gen.from_strings(subst + gen.to_strings(*gen.generate(200, 70 + d, 0.0, 0.0)))
    got = oracle.symdel_query(rs, ro, qs, qo, d, "hamming")
    assert np.array_equal(got, oracle.bruteforce_query(rs, ro, qs, qo, d, "hamming"))
    assert got.shape[0] >= len(subst)
    lens_r, lens_q = np.diff(ro), np.diff(qo)
    assert np.array_equal(lens_q[got[:, 0]], lens_r[got[:, 1]])
    lev = oracle.symdel_query(rs, ro, qs, qo, d)
    key = lambda r: r[:, 0].astype(np.int64) << 32 | r[:, 1].astype(np.int64)
    assert np.isin(key(got), key(lev)).all()


# ------------------------------------------- threaded exhaustive query ---
@pytest.mark.parametrize("metric", ["levenshtein", "hamming"])
def test_threaded_bruteforce_query_is_the_brute_force(metric):
    # references split over threads: every thread count, including more
    # threads than references, gives the single-thread exhaustive rows
    rs, ro = gen.generate(700, 81, 0.2, 0.01)
    strs = gen.to_strings(rs, ro)
    qs, qo = gen.from_strings(strs[::97] + strs[-3:] + gen.to_strings(*gen.generate(40, 82)))
    want = oracle.bruteforce_query(rs, ro, qs, qo, 2, metric)
    assert want.shape[0] >= 10
    assert np.array_equal(want, oracle.symdel_query(rs, ro, qs, qo, 2, metric))
    for threads in (2, 3, 7, 0):
        got = oracle.bruteforce_query(rs, ro, qs, qo, 2, metric, threads=threads)
        assert np.array_equal(got, want), threads
    tiny_s, tiny_o = gen.from_strings(["CASSF", "CASF", "CAS"])
    q_s, q_o = gen.from_strings(["CASF", "CAF"])
    want = oracle.bruteforce_query(tiny_s, tiny_o, q_s, q_o, 1, metric)
    for threads in (1, 2, 5, 9):
        assert np.array_equal(
            oracle.bruteforce_query(tiny_s, tiny_o, q_s, q_o, 1, metric, threads=threads), want)


# --------------------------------------------------------- paired chains ---
def test_paired_hand_worked():
    for line in open(os.path.join(GOLDEN, "paired_hand.txt")):
        line = line.split("#")[0].split()
        if line:
            assert oracle.lev_token(line[0], line[1]) == int(line[2]), line


def _token_edits1(s, alphabet):
    # single edits that leave the token '|' alone: residue insertions,
    # deletions and substitutions anywhere else
    out = set()
    for i in range(len(s) + 1):
        for c in alphabet:
            out.add(s[:i] + c + s[i:])
    for i in range(len(s)):
        if s[i] == "|":
            continue
        out.add(s[:i] + s[i + 1:])
        for c in alphabet:
            if c != s[i]:
                out.add(s[:i] + c + s[i + 1:])
    return out


def test_paired_distance_matches_bfs_over_admissible_edits():
    # every string within radius 3 of a receptor, by BFS over token-respecting
    # edits (independent of any DP), has its BFS level as lev_token
    for s in ["AC|C", "|A", "CA|", "A|CA"]:
        dist = {s: 0}
        frontier = {s}
        for r in range(1, 4):
            nxt = set()
            for t in frontier:
                nxt |= _token_edits1(t, "AC")
            nxt -= dist.keys()
            for t in nxt:
                dist[t] = r
            frontier = nxt
        rng = random.Random(len(s))
        for t in rng.sample(sorted(dist), min(300, len(dist))):
            assert oracle.lev_token(s, t) == dist[t], (s, t)
        # strings with one token outside the ball are farther than 3
        far = ["AAAA|CCCC", "|CCCCA", "CCCCAA|"]
        for t in far:
            if t not in dist:
                assert oracle.lev_token(s, t) > 3


def test_paired_distance_is_the_sum_of_chain_distances():
    rng = random.Random(11)
    for _ in range(400):
        a1, b1, a2, b2 = (_rand_strings(rng, 1, "ACD", 0, 6)[0] for _ in range(4))
        want = oracle.levenshtein(a1, a2) + oracle.levenshtein(b1, b2)
        assert oracle.lev_token(a1 + "|" + b1, a2 + "|" + b2) == want


def test_paired_variant_counts():
    # the token is never deleted: distinct residues give sum_k C(L, k) variants
    # over the residues of both chains (Sec. 2.1's 56 for L = 10, d = 2)
    assert oracle.count_variants_token("ACDEFGHIKL|", 2) == 56
    assert oracle.count_variants_token("ACDEF|GHIKL", 2) == 56
    assert oracle.count_variants_token("AC|DE", 2) == 1 + 4 + 6
    assert oracle.count_variants_token("|", 3) == 1


def _paired_set(rng, n, alphabet, lmax):
    a = _rand_strings(rng, n, alphabet, 0, lmax)
    b = _rand_strings(rng, n, alphabet, 0, lmax)
    sa, oa = gen.from_strings(a)
    sb, ob = gen.from_strings(b)
    return sa, oa, sb, ob


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_paired_symdel_equals_bruteforce(d):
    rng = random.Random(30 + d)
    for alphabet, lmax in [("AC", 5), ("ACDE", 7)]:
        sa, oa, sb, ob = _paired_set(rng, 150, alphabet, lmax)
        want = oracle.bruteforce_paired(sa, oa, sb, ob, d)
        got = oracle.symdel_paired(sa, oa, sb, ob, d)
        assert np.array_equal(got, want)
        if d >= 1:
            assert want.shape[0] > 0


def test_paired_with_empty_second_chains_is_the_single_chain_search():
    seqs, off = gen.workload(gen.SELF_1M, 800)
    empty = np.zeros(0, np.uint8)
    zero = np.zeros(off.size, np.int64)
    for d in (1, 2):
        assert np.array_equal(oracle.symdel_paired(seqs, off, empty, zero, d),
                              oracle.bruteforce_self(seqs, off, d))
