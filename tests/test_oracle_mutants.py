"""Planted mistakes in the oracle: each plausible slip in its arithmetic must
fail one of the pin checks below.

Every mutant is a copy of oracle/xtn_oracle.cpp with one edit, built on the
CPU into a temporary library that the oracle module is pointed at.  The
checks restate the pins of test_oracle_pins.py in a compact form: textbook
edit distances, the worked variant count of Sec. 2.1, the special case
d = 0, Hamming textbook values and lengths, the hand-worked TCRdist scores of
tests/golden/tcrdist_hand.txt, the self, query, batched and sharded searches
against exhaustive comparison, the threaded exhaustive query against the
single-thread one, paired chains (hand-worked distances, a variant count and
SymDel against exhaustive search), one sequence's neighbours, the TCRdist filter
against the all-pairs scorer, and the within/between partition of the
batched search.  The unmutated source passes every check.
"""
import concurrent.futures
import os
import subprocess

import numpy as np
import pytest

import cdr3_synth as gen
import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "xtn_oracle.cpp")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tcrdist_hand.txt")

# (what the slip is, text in the source, replacement); every text occurs once
MUTANTS = [
    ("equal letters cost a substitution", "(a[x - 1] == b[y - 1] ? 0 : 1)", "1"),
    ("insertions are free", "int ins = D[x * w + (y - 1)] + 1;", "int ins = D[x * w + (y - 1)] + 0;"),
    ("first DP column left at zero", "for (size_t x = 0; x <= la; ++x) D[x * w] = static_cast<int>(x);",
     "for (size_t x = 0; x <= la; ++x) D[x * w] = 0;"),
    ("one deletion fewer", "for (int k = 1; k <= d; ++k) {\n    std::unordered_set<std::string> next;",
     "for (int k = 1; k < d; ++k) {\n    std::unordered_set<std::string> next;"),
    ("the string itself is not a variant", "std::unordered_set<std::string> all{s};",
     "std::unordered_set<std::string> all;"),
    ("only the first residue is ever deleted", "std::string u = t.substr(0, p) + t.substr(p + 1);",
     "std::string u = t.substr(1);"),
    ("a sequence paired with itself", "    if (c.first >= c.second) continue;",
     "    if (c.first > c.second) continue;"),
    ("the threshold is strict",
     "    if (dist <= d) rows.push_back({c.first, c.second, static_cast<uint32_t>(dist)});",
     "    if (dist < d) rows.push_back({c.first, c.second, static_cast<uint32_t>(dist)});"),
    ("Hamming counts agreeing positions", "h += a[p] != b[p];", "h += a[p] == b[p];"),
    ("Hamming compares unequal lengths by their difference",
     "if (a.size() != b.size()) return NOT_NEIGHBOURS;",
     "if (a.size() != b.size()) return (int)(a.size() > b.size() ? a.size() - b.size() : b.size() - a.size());"),
    ("TCRdist gap costs 3", "sum += 4 * static_cast<int>(g);", "sum += 3 * static_cast<int>(g);"),
    ("TCRdist weight 2", "return 3 * sum;", "return 2 * sum;"),
    ("TCRdist gaps one position later", "const size_t p = m / 2;", "const size_t p = (m + 1) / 2;"),
    ("TCRdist mismatch cost uncapped", "sum += std::min(4, 4 - blosum62(x, y));",
     "sum += 4 - blosum62(x, y);"),
    ("pairs within a repertoire reported as between",
     "if (rep_of(row[0]) != rep_of(row[1])) keep.push_back(row);",
     "if (rep_of(row[0]) == rep_of(row[1])) keep.push_back(row);"),
    ("queries look up one deletion fewer", "for (const std::string& v : deletion_variants(s, d)) {",
     "for (const std::string& v : deletion_variants(s, d > 0 ? d - 1 : 0)) {"),
    ("query threshold strict",
     "if (dist <= d) rows.push_back({static_cast<uint32_t>(q), r, static_cast<uint32_t>(dist)});",
     "if (dist < d) rows.push_back({static_cast<uint32_t>(q), r, static_cast<uint32_t>(dist)});"),
    ("batched rows keep global indices",
     "all.push_back({static_cast<uint32_t>(r), row[0], row[1], row[2]});",
     "all.push_back({static_cast<uint32_t>(r), row[0] + (uint32_t)rep_off[r], "
     "row[1] + (uint32_t)rep_off[r], row[2]});"),
    ("exhaustive search pairs a sequence with itself",
     "for (int64_t j = i + 1; j < n; ++j) {\n      int dist = distance(s[i], s[j], metric);",
     "for (int64_t j = i; j < n; ++j) {\n      int dist = distance(s[i], s[j], metric);"),
    ("exhaustive query threshold strict",
     "      if (dist <= d)\n        rows.push_back({static_cast<uint32_t>(q), static_cast<uint32_t>(r),",
     "      if (dist < d)\n        rows.push_back({static_cast<uint32_t>(q), static_cast<uint32_t>(r),"),
    ("one sequence's neighbours include itself", "    if (j == i) continue;\n", ""),
    ("TCRdist filter threshold strict",
     "seq_at(seqs, off, j)) <= max_score)", "seq_at(seqs, off, j)) < max_score)"),
    ("all-pairs scorer threshold strict", "if (score > max_score) continue;",
     "if (score >= max_score) continue;"),
    ("sharded search pairs an id with itself",
     "for (size_t b = a + 1; b < kv.second.size(); ++b)",
     "for (size_t b = a; b < kv.second.size(); ++b)"),
    ("paired variants delete the token", "        if (t[p] == TOKEN) continue;\n", ""),
    ("paired distance lets the token be substituted",
     "return (x == TOKEN || y == TOKEN) ? FORBIDDEN : 1;", "return 1;"),
    ("paired distance lets the token be deleted or inserted",
     "auto del = [&](char c) { return c == TOKEN ? FORBIDDEN : 1; };",
     "auto del = [&](char c) { return 1; };"),
    ("paired threshold strict",
     "if (dist <= d) rows.push_back({c.first, c.second, (uint32_t)dist});  // paired",
     "if (dist < d) rows.push_back({c.first, c.second, (uint32_t)dist});  // paired"),
    ("threaded exhaustive query skips the last reference of each range",
     "for (int64_t r = lo; r < hi; ++r) {", "for (int64_t r = lo; r + 1 < hi; ++r) {"),
    ("threaded exhaustive query threshold strict",
     "          if (dist <= d)\n            part[t].push_back(",
     "          if (dist < d)\n            part[t].push_back("),
]


# ------------------------------------------------------------- the checks ---
_PREFIX = {}


def _prefix(n):
    """The first n <= 1500 sequences of the 1M workload (generated once)."""
    if not _PREFIX:
        _PREFIX["all"] = gen.workload(gen.SELF_1M, 1500)
    seqs, off = _PREFIX["all"]
    return seqs[: off[n]], off[: n + 1]


def check_textbook_distances():
    for a, b, want in [("kitten", "sitting", 3), ("flaw", "lawn", 2), ("", "CAS", 3),
                       ("CAS", "", 3), ("intention", "execution", 5), ("CASSF", "CASSF", 0)]:
        assert oracle.levenshtein(a, b) == want


def check_worked_variant_count():
    # Sec. 2.1: 56 variants with up to two deletions of a length-10 string
    # of distinct residues; 11 with up to one
    assert oracle.count_variants("ACDEFGHIKL", 2) == 56
    assert oracle.count_variants("ACDEFGHIKL", 1) == 11


def _small_sets():
    rng = np.random.default_rng(5)
    strs = ["".join(rng.choice(list("AC"), size=k)) for k in rng.integers(0, 8, 150)]
    yield gen.from_strings(strs)
    yield _prefix(800)


def check_search_equals_exhaustive():
    for seqs, off in _small_sets():
        for d in (1, 2):
            want = oracle.bruteforce_self(seqs, off, d)
            assert want.shape[0] > 0
            assert np.array_equal(oracle.symdel_self(seqs, off, d), want)


def check_d0_is_duplicate_grouping():
    strs = ["CASSF", "CASSF", "CAS", "", "", "CASSF", "CAT"]
    seqs, off = gen.from_strings(strs)
    want = [[i, j, 0] for i in range(len(strs)) for j in range(i + 1, len(strs))
            if strs[i] == strs[j]]
    assert oracle.symdel_self(seqs, off, 0).tolist() == want


def check_hamming():
    assert oracle.hamming("KAROLIN", "KATHRIN") == 3
    assert oracle.hamming("CASSF", "CASSF") == 0
    seqs, off = gen.from_strings(["CAS", "CASS", "CAT", "CA"])
    # only CAS-CAT has equal lengths
    assert oracle.symdel_self(seqs, off, 2, "hamming").tolist() == [[0, 2, 1]]


def check_tcrdist_hand_worked():
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if line:
            assert oracle.tcrdist(line[0], line[1]) == int(line[2])


def check_between_and_within_partition():
    seqs, off = _prefix(1000)
    rep = np.array([0, 300, 310, 700, 1000], dtype=np.int64)
    whole = oracle.bruteforce_self(seqs, off, 2)
    cross = oracle.symdel_cross(seqs, off, rep, 2)
    within = oracle.symdel_batched(seqs, off, rep, 2)
    glob = np.stack([within[:, 1] + rep[within[:, 0]], within[:, 2] + rep[within[:, 0]],
                     within[:, 3]], 1).astype(np.uint32)
    both = np.concatenate([cross, glob])
    both = both[np.lexsort((both[:, 1], both[:, 0]))]
    assert np.array_equal(both, whole)


def check_query_equals_exhaustive():
    rs, ro = _prefix(600)
    strs = gen.to_strings(rs, ro)
    qs, qo = gen.from_strings(strs[:40] + [s[1:] + "A" for s in strs[40:80]])
    for d in (1, 2):
        want = oracle.bruteforce_query(rs, ro, qs, qo, d)
        assert want.shape[0] > 40
        assert np.array_equal(oracle.symdel_query(rs, ro, qs, qo, d), want)


def check_batched_is_per_repertoire():
    seqs, off = _prefix(600)
    rep = np.array([0, 250, 600], dtype=np.int64)
    want = []
    for r in range(2):
        a, b = int(rep[r]), int(rep[r + 1])
        for row in oracle.bruteforce_self(seqs[off[a]:off[b]], off[a:b + 1] - off[a], 2).tolist():
            want.append([r] + row)
    assert oracle.symdel_batched(seqs, off, rep, 2).tolist() == sorted(want)


def check_neighbours_of_one_sequence():
    seqs, off = _prefix(600)
    rows = oracle.bruteforce_self(seqs, off, 2)
    for i in (int(rows[0, 0]), int(rows[-1, 1])):
        want = sorted([[int(r[1]) if r[0] == i else int(r[0]), int(r[2])]
                       for r in rows if i in (r[0], r[1])])
        assert oracle.neighbors_of(seqs, off, i, 2).tolist() == want


def check_threaded_query_equals_exhaustive():
    rs, ro = _prefix(600)
    strs = gen.to_strings(rs, ro)
    # the last reference of each of the three ranges is some query's neighbour
    qs, qo = gen.from_strings(strs[::37] + [s[1:] for s in strs[::41]]
                              + [strs[199], strs[399], strs[599]])
    want = oracle.bruteforce_query(rs, ro, qs, qo, 2)
    assert want.shape[0] > 20
    assert np.array_equal(oracle.bruteforce_query(rs, ro, qs, qo, 2, threads=3), want)


def check_paired():
    golden = os.path.join(os.path.dirname(__file__), "golden", "paired_hand.txt")
    for line in open(golden):
        line = line.split("#")[0].split()
        if line:
            assert oracle.lev_token(line[0], line[1]) == int(line[2])
    assert oracle.count_variants_token("AC|DE", 2) == 11
    seqs, off = _prefix(300)
    strs = gen.to_strings(seqs, off)
    a_s, a_o = gen.from_strings(strs[:150])
    b_s, b_o = gen.from_strings([s[3:] for s in strs[150:]])
    for d in (1, 2):
        want = oracle.bruteforce_paired(a_s, a_o, b_s, b_o, d)
        assert np.array_equal(oracle.symdel_paired(a_s, a_o, b_s, b_o, d), want)
    # a receptor set with planted one- and two-edit neighbours
    a_s, a_o = gen.from_strings(["CASSF", "CASF", "CAS", "CASSF"])
    b_s, b_o = gen.from_strings(["CAVF", "CAVF", "CAV", "CAIF"])
    assert oracle.symdel_paired(a_s, a_o, b_s, b_o, 2).tolist() == \
        [[0, 1, 1], [0, 3, 1], [1, 2, 2], [1, 3, 2]]


def check_sharded_equals_exhaustive():
    seqs, off = _prefix(600)
    assert np.array_equal(oracle.symdel_self_sharded(seqs, off, 2, threads=3),
                          oracle.bruteforce_self(seqs, off, 2))


def check_tcrdist_filter_and_scorer():
    seqs, off = _prefix(1500)
    lev = oracle.bruteforce_self(seqs, off, 2)
    kept = oracle.tcrdist_filter(seqs, off, lev, 24)
    full = oracle.tcrdist_allpairs(seqs, off, 2, 24)
    assert (full[:, 3] == 24).any()       # a score on the threshold itself
    assert np.array_equal(kept, full[:, :3])


# cheapest first: a mutant stops at its first failing check
CHECKS = [check_textbook_distances, check_worked_variant_count, check_hamming,
          check_tcrdist_hand_worked, check_d0_is_duplicate_grouping,
          check_search_equals_exhaustive, check_query_equals_exhaustive,
          check_batched_is_per_repertoire, check_neighbours_of_one_sequence,
          check_sharded_equals_exhaustive, check_threaded_query_equals_exhaustive, check_paired,
          check_tcrdist_filter_and_scorer,
          check_between_and_within_partition]


def _failing(path, first_only):
    failed = []
    with oracle.built_from(path):
        for check in CHECKS:
            try:
                check()
            except AssertionError:
                failed.append(check.__name__)
                if first_only:
                    break
    return failed


def _build(text, path):
    with open(path + ".cpp", "w") as f:
        f.write(text)
    subprocess.run(["g++", "-O1", "-std=c++17", "-pthread", "-shared", "-fPIC", path + ".cpp",
                    "-o", path], check=True)
    return path


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("mutants")
    jobs = {"original": src}
    for k, (what, old, new) in enumerate(MUTANTS):
        assert src.count(old) == 1, what
        jobs[what] = src.replace(old, new)
    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as pool:
        futs = {what: pool.submit(_build, text, str(d / f"m{k}.so"))
                for k, (what, text) in enumerate(jobs.items())}
        return {what: f.result() for what, f in futs.items()}


def test_unmutated_source_passes_every_check(builds):
    assert _failing(builds["original"], first_only=False) == []


@pytest.mark.parametrize("what", [m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(builds, what):
    assert _failing(builds[what], first_only=True), f"no pin catches: {what}"
