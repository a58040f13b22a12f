// CPU oracle for symmetric-deletion (SymDel) Levenshtein neighbour search
// (and its Hamming variant).
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
// benchmark's CPU-baseline leg may load this library. It shares no code,
// header, table or constant with the CUDA path: it works on std::string, full
// O(La*Lb) dynamic programming and std::unordered_map, and is slow on purpose.
//
// What it computes (the plain definition the GPU path must reproduce):
//   { (i, j, Lev(s_i, s_j)) : i < j, Lev(s_i, s_j) <= d }  sorted by (i, j)
// with unit-cost insertion / deletion / substitution edit distance.
//
// The self-search follows the paper's CPU algorithm in its own order
// (Appendix, "Symmetric deletion lookup step-by-step", steps 0-4):
//   1. generate every deletion variant with up to d deletions (0 deletions,
//      i.e. the string itself, included) of every sequence;
//   2. store them in a multi-value hash map  variant -> indices;
//   3. look every sequence's own variants up again, collecting candidates;
//   4. drop self/duplicate candidates and those with Lev > d.
// Pins (tests/test_oracle_pins.py): brute-force all-pairs Levenshtein, the
// worked counts of Sec. 2.1 (56 variants / 79,746 neighbours), textbook
// distances, exhaustive edit balls, the SymDel guarantee of Sec. 2.1 and the
// bag-of-amino-acids bound of Appendix B.
//
// Paired chains (Discussion): receptors alpha + '|' + beta, the joining token
// never deleted, inserted or substituted (lev_token, deletion_variants_token);
// SymDel and exhaustive searches over them.
//
// TCRdist score (Results, "SymDel lookup can be combined with more advanced
// similarity metrics"; the paper cites TCRdist without defining it; reading
// used here): gaps = |La - Lb| placed in the shorter sequence after its first
// floor(m/2) residues (m = shorter length); each aligned position costs 0 if
// the residues agree, else min(4, 4 - BLOSUM62[a][b]); each gap costs 4; the
// sum is multiplied by 3. BLOSUM62 is the published matrix (Henikoff &
// Henikoff 1992): parity unpinned beyond symmetry/range checks.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

struct Result {
  int width;                    // uint32 fields per record
  std::vector<uint32_t> v;
};

std::string seq_at(const uint8_t* seqs, const int64_t* off, int64_t i) {
  return std::string(reinterpret_cast<const char*>(seqs) + off[i],
                     static_cast<size_t>(off[i + 1] - off[i]));
}

// Wagner-Fischer: D[x][y] = edit distance between a[0:x] and b[0:y].
int lev_full(const std::string& a, const std::string& b) {
  const size_t la = a.size(), lb = b.size();
  const size_t w = lb + 1;                       // D[x][y] stored at D[x * w + y]
  std::vector<int> D((la + 1) * w, 0);
  for (size_t x = 0; x <= la; ++x) D[x * w] = static_cast<int>(x);
  for (size_t y = 0; y <= lb; ++y) D[y] = static_cast<int>(y);
  for (size_t x = 1; x <= la; ++x) {
    for (size_t y = 1; y <= lb; ++y) {
      int del = D[(x - 1) * w + y] + 1;
      int ins = D[x * w + (y - 1)] + 1;
      int sub = D[(x - 1) * w + (y - 1)] + (a[x - 1] == b[y - 1] ? 0 : 1);
      D[x * w + y] = std::min(std::min(del, ins), sub);
    }
  }
  return D[la * w + lb];
}

// Hamming distance (Results, comparison with CompAIRR: the last step filters
// by Hamming instead of Levenshtein distance): the number of positions at
// which two strings of equal length differ; strings of different lengths are
// never Hamming neighbours (returned as a distance no threshold admits).
constexpr int NOT_NEIGHBOURS = 1 << 30;
int hamming(const std::string& a, const std::string& b) {
  if (a.size() != b.size()) return NOT_NEIGHBOURS;
  int h = 0;
  for (size_t p = 0; p < a.size(); ++p) h += a[p] != b[p];
  return h;
}

// The last step's distance: 0 = Levenshtein, 1 = Hamming.
int distance(const std::string& a, const std::string& b, int metric) {
  return metric == 1 ? hamming(a, b) : lev_full(a, b);
}

// Paired chains (Discussion: the CDR3s of both chains concatenated with a
// non-deletable joining token).  A receptor is the string alpha + TOKEN +
// beta.  Reading used here: the token is a character outside the residue
// alphabet that no edit may delete, insert or substitute, so in every
// admissible alignment the two tokens face each other.  The distance is the
// edit distance under that rule (infinite cost for any other operation on
// the token), computed by the same Wagner-Fischer recurrence.
constexpr char TOKEN = '|';
constexpr int FORBIDDEN = 1 << 20;  // cost of an edit that touches the token

int lev_token(const std::string& a, const std::string& b) {
  const size_t la = a.size(), lb = b.size();
  const size_t w = lb + 1;                       // D[x][y] stored at D[x * w + y]
  std::vector<int> D((la + 1) * w, 0);
  auto del = [&](char c) { return c == TOKEN ? FORBIDDEN : 1; };
  auto sub = [&](char x, char y) {
    if (x == y) return 0;
    return (x == TOKEN || y == TOKEN) ? FORBIDDEN : 1;
  };
  for (size_t x = 1; x <= la; ++x) D[x * w] = std::min(FORBIDDEN, D[(x - 1) * w] + del(a[x - 1]));
  for (size_t y = 1; y <= lb; ++y) D[y] = std::min(FORBIDDEN, D[y - 1] + del(b[y - 1]));
  for (size_t x = 1; x <= la; ++x) {
    for (size_t y = 1; y <= lb; ++y) {
      int dl = D[(x - 1) * w + y] + del(a[x - 1]);
      int in = D[x * w + (y - 1)] + del(b[y - 1]);
      int sb = D[(x - 1) * w + (y - 1)] + sub(a[x - 1], b[y - 1]);
      D[x * w + y] = std::min(FORBIDDEN, std::min(std::min(dl, in), sb));
    }
  }
  return D[la * w + lb];
}

// Step 1 for paired chains: every string reachable from s by at most d
// deletions of residues (the token is never deleted).
std::unordered_set<std::string> deletion_variants_token(const std::string& s, int d) {
  std::unordered_set<std::string> found{s};
  std::unordered_set<std::string> level{s};   // strings of exactly r deletions
  for (int r = 1; r <= d; ++r) {
    std::unordered_set<std::string> deeper;
    for (const std::string& t : level)
      for (size_t p = 0; p < t.size(); ++p) {
        if (t[p] == TOKEN) continue;
        deeper.insert(t.substr(0, p) + t.substr(p + 1));
      }
    found.insert(deeper.begin(), deeper.end());
    level.swap(deeper);
  }
  return found;
}

// Step 1: all strings reachable from s by at most d single-character deletions.
std::unordered_set<std::string> deletion_variants(const std::string& s, int d) {
  std::unordered_set<std::string> all{s};
  std::unordered_set<std::string> frontier{s};
  for (int k = 1; k <= d; ++k) {
    std::unordered_set<std::string> next;
    for (const std::string& t : frontier)
      for (size_t p = 0; p < t.size(); ++p) {
        std::string u = t.substr(0, p) + t.substr(p + 1);
        next.insert(u);
      }
    for (const std::string& u : next) all.insert(u);
    frontier.swap(next);
  }
  return all;
}

void sort_unique(std::vector<std::vector<uint32_t>>& rows) {
  std::sort(rows.begin(), rows.end());
  rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
}

Result* pack(std::vector<std::vector<uint32_t>>& rows, int width) {
  Result* r = new Result;
  r->width = width;
  r->v.reserve(rows.size() * width);
  for (auto& row : rows) r->v.insert(r->v.end(), row.begin(), row.end());
  return r;
}

// Self search over sequences [lo, hi) with indices reported relative to lo.
std::vector<std::vector<uint32_t>> symdel_self_range(const uint8_t* seqs, const int64_t* off,
                                                     int64_t lo, int64_t hi, int d,
                                                     int metric = 0) {
  const int64_t n = hi - lo;
  std::vector<std::string> s(n);
  for (int64_t i = 0; i < n; ++i) s[i] = seq_at(seqs, off, lo + i);
  // Steps 1-2: variants x and the multi-value map variant -> ids.
  std::vector<std::unordered_set<std::string>> x(n);
  std::unordered_map<std::string, std::vector<uint32_t>> table;
  for (int64_t i = 0; i < n; ++i) {
    x[i] = deletion_variants(s[i], d);
    for (const std::string& v : x[i]) table[v].push_back(static_cast<uint32_t>(i));
  }
  // Step 3: reuse x to look the table up -> candidates y.
  std::vector<std::pair<uint32_t, uint32_t>> y;
  for (int64_t i = 0; i < n; ++i)
    for (const std::string& v : x[i])
      for (uint32_t j : table[v]) y.emplace_back(static_cast<uint32_t>(i), j);
  // Step 4: keep unordered pairs once (i < j), verify the distance, dedup.
  // Two strings of one length with h <= d differing positions share the
  // string left after deleting those positions from both, so every Hamming
  // neighbour is a candidate too.
  std::vector<std::vector<uint32_t>> rows;
  std::sort(y.begin(), y.end());
  y.erase(std::unique(y.begin(), y.end()), y.end());
  for (auto& c : y) {
    if (c.first >= c.second) continue;
    int dist = distance(s[c.first], s[c.second], metric);
    if (dist <= d) rows.push_back({c.first, c.second, static_cast<uint32_t>(dist)});
  }
  sort_unique(rows);
  return rows;
}

// The same self-search with the variant keys partitioned over T threads by
// a hash of the key: thread t keeps the map of the keys of its part, pairs
// up the ids of every key it holds, and verifies those candidates; the rows
// of all threads are merged and deduplicated.  Only the bookkeeping differs
// from symdel_self_range (equal variants always fall in one part), so the
// rows are the same.  It exists to time the oracle on every host core.
std::vector<std::vector<uint32_t>> symdel_self_sharded(const uint8_t* seqs, const int64_t* off,
                                                       int64_t n, int d, int metric, int T) {
  if (T < 1) T = 1;
  std::vector<std::string> s(n);
  for (int64_t i = 0; i < n; ++i) s[i] = seq_at(seqs, off, i);
  // step 1, every sequence's variants, split over the threads by sequence
  std::vector<std::vector<std::string>> x(n);
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t)
    pool.emplace_back([&, t] {
      for (int64_t i = t; i < n; i += T) {
        auto v = deletion_variants(s[i], d);
        x[i].assign(v.begin(), v.end());
      }
    });
  for (auto& th : pool) th.join();
  pool.clear();
  // steps 2-4 per part of the key space
  std::vector<std::vector<std::vector<uint32_t>>> part(T);
  for (int t = 0; t < T; ++t)
    pool.emplace_back([&, t] {
      std::hash<std::string> h;
      std::unordered_map<std::string, std::vector<uint32_t>> table;
      for (int64_t i = 0; i < n; ++i)
        for (const std::string& v : x[i])
          if ((int)(h(v) % (size_t)T) == t) table[v].push_back(static_cast<uint32_t>(i));
      std::vector<std::pair<uint32_t, uint32_t>> y;
      for (auto& kv : table)
        for (size_t a = 0; a < kv.second.size(); ++a)
          for (size_t b = a + 1; b < kv.second.size(); ++b)
            y.emplace_back(kv.second[a], kv.second[b]);  // ids ascend within a key
      std::sort(y.begin(), y.end());
      y.erase(std::unique(y.begin(), y.end()), y.end());
      for (auto& c : y) {
        const int dist = distance(s[c.first], s[c.second], metric);
        if (dist <= d) part[t].push_back({c.first, c.second, static_cast<uint32_t>(dist)});
      }
    });
  for (auto& th : pool) th.join();
  std::vector<std::vector<uint32_t>> rows;
  for (auto& p : part) rows.insert(rows.end(), p.begin(), p.end());
  sort_unique(rows);
  return rows;
}

// ---- BLOSUM62 (Henikoff & Henikoff 1992), rows/cols in the order below. ----
const char kB62Order[] = "ARNDCQEGHILKMFPSTWYV";
const int kB62[20][20] = {
    /*A*/ {4, -1, -2, -2, 0, -1, -1, 0, -2, -1, -1, -1, -1, -2, -1, 1, 0, -3, -2, 0},
    /*R*/ {-1, 5, 0, -2, -3, 1, 0, -2, 0, -3, -2, 2, -1, -3, -2, -1, -1, -3, -2, -3},
    /*N*/ {-2, 0, 6, 1, -3, 0, 0, 0, 1, -3, -3, 0, -2, -3, -2, 1, 0, -4, -2, -3},
    /*D*/ {-2, -2, 1, 6, -3, 0, 2, -1, -1, -3, -4, -1, -3, -3, -1, 0, -1, -4, -3, -3},
    /*C*/ {0, -3, -3, -3, 9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1},
    /*Q*/ {-1, 1, 0, 0, -3, 5, 2, -2, 0, -3, -2, 1, 0, -3, -1, 0, -1, -2, -1, -2},
    /*E*/ {-1, 0, 0, 2, -4, 2, 5, -2, 0, -3, -3, 1, -2, -3, -1, 0, -1, -3, -2, -2},
    /*G*/ {0, -2, 0, -1, -3, -2, -2, 6, -2, -4, -4, -2, -3, -3, -2, 0, -2, -2, -3, -3},
    /*H*/ {-2, 0, 1, -1, -3, 0, 0, -2, 8, -3, -3, -1, -2, -1, -2, -1, -2, -2, 2, -3},
    /*I*/ {-1, -3, -3, -3, -1, -3, -3, -4, -3, 4, 2, -3, 1, 0, -3, -2, -1, -3, -1, 3},
    /*L*/ {-1, -2, -3, -4, -1, -2, -3, -4, -3, 2, 4, -2, 2, 0, -3, -2, -1, -2, -1, 1},
    /*K*/ {-1, 2, 0, -1, -3, 1, 1, -2, -1, -3, -2, 5, -1, -3, -1, 0, -1, -3, -2, -2},
    /*M*/ {-1, -1, -2, -3, -1, 0, -2, -3, -2, 1, 2, -1, 5, 0, -2, -1, -1, -1, -1, 1},
    /*F*/ {-2, -3, -3, -3, -2, -3, -3, -3, -1, 0, 0, -3, 0, 6, -4, -2, -2, 1, 3, -1},
    /*P*/ {-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4, 7, -1, -1, -4, -3, -2},
    /*S*/ {1, -1, 1, 0, -1, 0, 0, 0, -1, -2, -2, 0, -1, -2, -1, 4, 1, -3, -2, -2},
    /*T*/ {0, -1, 0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1, 1, 5, -2, -2, 0},
    /*W*/ {-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1, 1, -4, -3, -2, 11, 2, -3},
    /*Y*/ {-2, -2, -2, -3, -2, -1, -2, -3, 2, -1, -1, -2, -1, 3, -3, -2, -2, 2, 7, -1},
    /*V*/ {0, -3, -3, -3, -1, -2, -2, -3, -3, 3, 1, -2, 1, -1, -2, -2, 0, -3, -1, 4},
};

int b62_index(char c) {
  const char* p = std::strchr(kB62Order, c);
  return (p && c) ? static_cast<int>(p - kB62Order) : -1;
}

int blosum62(char a, char b) {
  int x = b62_index(a), y = b62_index(b);
  if (x < 0 || y < 0) return -1000;
  return kB62[x][y];
}

int tcrdist_score(const std::string& a, const std::string& b) {
  const std::string& s = a.size() <= b.size() ? a : b;   // shorter
  const std::string& l = a.size() <= b.size() ? b : a;   // longer
  const size_t m = s.size();
  const size_t g = l.size() - m;
  const size_t p = m / 2;                                // gaps after s[0:p]
  int sum = 0;
  for (size_t k = 0; k < m; ++k) {
    char x = s[k];
    char y = (k < p) ? l[k] : l[k + g];
    if (x != y) sum += std::min(4, 4 - blosum62(x, y));
  }
  sum += 4 * static_cast<int>(g);
  return 3 * sum;
}

}  // namespace

extern "C" {

// ---------------- result handles ----------------
int64_t xo_result_rows(void* h) {
  Result* r = static_cast<Result*>(h);
  return static_cast<int64_t>(r->v.size() / r->width);
}
int xo_result_width(void* h) { return static_cast<Result*>(h)->width; }
void xo_result_copy(void* h, uint32_t* dst) {
  Result* r = static_cast<Result*>(h);
  if (!r->v.empty()) std::memcpy(dst, r->v.data(), r->v.size() * sizeof(uint32_t));
}
void xo_result_free(void* h) { delete static_cast<Result*>(h); }

// ---------------- scalar helpers ----------------
int xo_hamming(const uint8_t* a, int la, const uint8_t* b, int lb) {
  const int h = hamming(std::string(reinterpret_cast<const char*>(a), la),
                        std::string(reinterpret_cast<const char*>(b), lb));
  return h == NOT_NEIGHBOURS ? -1 : h;
}

int xo_levenshtein(const uint8_t* a, int la, const uint8_t* b, int lb) {
  return lev_full(std::string(reinterpret_cast<const char*>(a), la),
                  std::string(reinterpret_cast<const char*>(b), lb));
}

int64_t xo_count_variants(const uint8_t* s, int L, int d) {
  return static_cast<int64_t>(
      deletion_variants(std::string(reinterpret_cast<const char*>(s), L), d).size());
}

int xo_blosum62(char a, char b) { return blosum62(a, b); }

int xo_tcrdist(const uint8_t* a, int la, const uint8_t* b, int lb) {
  return tcrdist_score(std::string(reinterpret_cast<const char*>(a), la),
                       std::string(reinterpret_cast<const char*>(b), lb));
}

// ---------------- searches ----------------
// SymDel self-search: rows (i, j, dist), i < j, sorted.
void* xo_symdel_self(const uint8_t* seqs, const int64_t* off, int64_t n, int d) {
  auto rows = symdel_self_range(seqs, off, 0, n, d);
  return pack(rows, 3);
}

// The self-search with its keys partitioned over `threads` threads (0: the
// host's hardware threads).  metric: 0 = Levenshtein, 1 = Hamming.
void* xo_symdel_self_sharded(const uint8_t* seqs, const int64_t* off, int64_t n, int d,
                             int metric, int threads) {
  if (threads <= 0) threads = std::max(1u, std::thread::hardware_concurrency());
  auto rows = symdel_self_sharded(seqs, off, n, d, metric, threads);
  return pack(rows, 3);
}

// The same with the Hamming distance in the last step.
void* xo_symdel_self_hamming(const uint8_t* seqs, const int64_t* off, int64_t n, int d) {
  auto rows = symdel_self_range(seqs, off, 0, n, d, 1);
  return pack(rows, 3);
}

// Independent repertoires: rows (rep, i_local, j_local, dist), sorted.
// metric: 0 = Levenshtein, 1 = Hamming.
void* xo_symdel_batched(const uint8_t* seqs, const int64_t* off, const int64_t* rep_off,
                        int64_t n_rep, int d, int metric) {
  std::vector<std::vector<uint32_t>> all;
  for (int64_t r = 0; r < n_rep; ++r) {
    auto rows = symdel_self_range(seqs, off, rep_off[r], rep_off[r + 1], d, metric);
    for (auto& row : rows)
      all.push_back({static_cast<uint32_t>(r), row[0], row[1], row[2]});
  }
  sort_unique(all);
  return pack(all, 4);
}

// Pairs between repertoires (the repertoire-overlap workload of the CompAIRR
// comparison): the SymDel self-search of the whole concatenation, keeping the
// pairs whose two sequences lie in different repertoires.  Rows (i, j, dist)
// with global indices, sorted.  metric: 0 = Levenshtein, 1 = Hamming.
void* xo_symdel_cross(const uint8_t* seqs, const int64_t* off, const int64_t* rep_off,
                      int64_t n_rep, int d, int metric) {
  const int64_t n = rep_off[n_rep];
  auto rows = symdel_self_range(seqs, off, 0, n, d, metric);
  std::vector<std::vector<uint32_t>> keep;
  auto rep_of = [&](uint32_t i) {
    return std::upper_bound(rep_off, rep_off + n_rep + 1, (int64_t)i) - rep_off - 1;
  };
  for (auto& row : rows)
    if (rep_of(row[0]) != rep_of(row[1])) keep.push_back(row);
  return pack(keep, 3);
}

// SymDel query-vs-reference: rows (q, r, dist) with dist <= d, sorted by
// (q, r).  Steps 1-2 on the reference, step 3 with the queries' own variants.
// metric: 0 = Levenshtein, 1 = Hamming.
void* xo_symdel_query_metric(const uint8_t* ref_seqs, const int64_t* ref_off, int64_t n_ref,
                             const uint8_t* q_seqs, const int64_t* q_off, int64_t n_q, int d,
                             int metric) {
  std::vector<std::string> ref(n_ref);
  std::unordered_map<std::string, std::vector<uint32_t>> table;
  for (int64_t r = 0; r < n_ref; ++r) {
    ref[r] = seq_at(ref_seqs, ref_off, r);
    for (const std::string& v : deletion_variants(ref[r], d))
      table[v].push_back(static_cast<uint32_t>(r));
  }
  std::vector<std::vector<uint32_t>> rows;
  for (int64_t q = 0; q < n_q; ++q) {
    std::string s = seq_at(q_seqs, q_off, q);
    std::vector<uint32_t> cand;
    for (const std::string& v : deletion_variants(s, d)) {
      auto it = table.find(v);
      if (it != table.end()) cand.insert(cand.end(), it->second.begin(), it->second.end());
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (uint32_t r : cand) {
      int dist = distance(s, ref[r], metric);
      if (dist <= d) rows.push_back({static_cast<uint32_t>(q), r, static_cast<uint32_t>(dist)});
    }
  }
  sort_unique(rows);
  return pack(rows, 3);
}

// Exhaustive search over all n(n-1)/2 pairs (the brute-force pin).
// metric: 0 = Levenshtein, 1 = Hamming.
void* xo_bruteforce_self_metric(const uint8_t* seqs, const int64_t* off, int64_t n, int d,
                                int metric) {
  std::vector<std::string> s(n);
  for (int64_t i = 0; i < n; ++i) s[i] = seq_at(seqs, off, i);
  std::vector<std::vector<uint32_t>> rows;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      int dist = distance(s[i], s[j], metric);
      if (dist <= d)
        rows.push_back({static_cast<uint32_t>(i), static_cast<uint32_t>(j),
                        static_cast<uint32_t>(dist)});
    }
  return pack(rows, 3);
}

void* xo_bruteforce_self(const uint8_t* seqs, const int64_t* off, int64_t n, int d) {
  return xo_bruteforce_self_metric(seqs, off, n, d, 0);
}

void* xo_symdel_query(const uint8_t* ref_seqs, const int64_t* ref_off, int64_t n_ref,
                      const uint8_t* q_seqs, const int64_t* q_off, int64_t n_q, int d) {
  return xo_symdel_query_metric(ref_seqs, ref_off, n_ref, q_seqs, q_off, n_q, d, 0);
}

// All (q, r) with dist <= d by exhaustive comparison.  metric: 0 =
// Levenshtein, 1 = Hamming.
void* xo_bruteforce_query_metric(const uint8_t* ref_seqs, const int64_t* ref_off, int64_t n_ref,
                                 const uint8_t* q_seqs, const int64_t* q_off, int64_t n_q, int d,
                                 int metric) {
  std::vector<std::string> ref(n_ref);
  for (int64_t r = 0; r < n_ref; ++r) ref[r] = seq_at(ref_seqs, ref_off, r);
  std::vector<std::vector<uint32_t>> rows;
  for (int64_t q = 0; q < n_q; ++q) {
    std::string s = seq_at(q_seqs, q_off, q);
    for (int64_t r = 0; r < n_ref; ++r) {
      int dist = distance(s, ref[r], metric);
      if (dist <= d)
        rows.push_back({static_cast<uint32_t>(q), static_cast<uint32_t>(r),
                        static_cast<uint32_t>(dist)});
    }
  }
  return pack(rows, 3);
}

void* xo_bruteforce_query(const uint8_t* ref_seqs, const int64_t* ref_off, int64_t n_ref,
                          const uint8_t* q_seqs, const int64_t* q_off, int64_t n_q, int d) {
  return xo_bruteforce_query_metric(ref_seqs, ref_off, n_ref, q_seqs, q_off, n_q, d, 0);
}

// The same exhaustive comparison with the references cut into `threads`
// contiguous ranges (0: the host's hardware threads), one per thread: each
// thread compares every query with every reference of its range.  Only the
// split of the reference loop differs from xo_bruteforce_query_metric, so the
// rows are the same; it lets a test check a few queries against references
// of millions of sequences in seconds.
void* xo_bruteforce_query_threaded(const uint8_t* ref_seqs, const int64_t* ref_off,
                                   int64_t n_ref, const uint8_t* q_seqs, const int64_t* q_off,
                                   int64_t n_q, int d, int metric, int threads) {
  if (threads <= 0) threads = std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::string> q(n_q);
  for (int64_t k = 0; k < n_q; ++k) q[k] = seq_at(q_seqs, q_off, k);
  std::vector<std::vector<std::vector<uint32_t>>> part(threads);
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&, t] {
      const int64_t lo = n_ref * t / threads, hi = n_ref * (t + 1) / threads;
      for (int64_t r = lo; r < hi; ++r) {
        const std::string s = seq_at(ref_seqs, ref_off, r);
        for (int64_t k = 0; k < n_q; ++k) {
          const int dist = distance(q[k], s, metric);
          if (dist <= d)
            part[t].push_back({static_cast<uint32_t>(k), static_cast<uint32_t>(r),
                               static_cast<uint32_t>(dist)});
        }
      }
    });
  for (auto& th : pool) th.join();
  std::vector<std::vector<uint32_t>> rows;
  for (auto& p : part) rows.insert(rows.end(), p.begin(), p.end());
  sort_unique(rows);
  return pack(rows, 3);
}

// Every j != i with Lev(s_i, s_j) <= d: rows (j, dist), sorted by j. This is
// the plain definition evaluated for one sequence, for sampled checks of
// outputs too large to recompute in full.
void* xo_neighbors_of(const uint8_t* seqs, const int64_t* off, int64_t n, int64_t i, int d) {
  std::string a = seq_at(seqs, off, i);
  std::vector<std::vector<uint32_t>> rows;
  for (int64_t j = 0; j < n; ++j) {
    if (j == i) continue;
    int dist = lev_full(a, seq_at(seqs, off, j));
    if (dist <= d) rows.push_back({static_cast<uint32_t>(j), static_cast<uint32_t>(dist)});
  }
  return pack(rows, 2);
}

// ---------------- paired chains ----------------
int xo_lev_token(const uint8_t* a, int la, const uint8_t* b, int lb) {
  return lev_token(std::string(reinterpret_cast<const char*>(a), la),
                   std::string(reinterpret_cast<const char*>(b), lb));
}

int64_t xo_count_variants_token(const uint8_t* s, int L, int d) {
  return static_cast<int64_t>(
      deletion_variants_token(std::string(reinterpret_cast<const char*>(s), L), d).size());
}

// SymDel over receptors alpha + TOKEN + beta (packed as one string each):
// steps 1-4 of the self-search with token-respecting variants and distance.
// Rows (i, j, dist), i < j, dist <= d, sorted.
void* xo_symdel_paired(const uint8_t* seqs, const int64_t* off, int64_t n, int d) {
  std::vector<std::string> s(n);
  for (int64_t i = 0; i < n; ++i) s[i] = seq_at(seqs, off, i);
  std::vector<std::unordered_set<std::string>> x(n);
  std::unordered_map<std::string, std::vector<uint32_t>> table;
  for (int64_t i = 0; i < n; ++i) {
    x[i] = deletion_variants_token(s[i], d);
    for (const std::string& v : x[i]) table[v].push_back(static_cast<uint32_t>(i));
  }
  std::vector<std::pair<uint32_t, uint32_t>> y;
  for (int64_t i = 0; i < n; ++i)
    for (const std::string& v : x[i])
      for (uint32_t j : table[v]) y.emplace_back(static_cast<uint32_t>(i), j);
  std::sort(y.begin(), y.end());
  y.erase(std::unique(y.begin(), y.end()), y.end());
  std::vector<std::vector<uint32_t>> rows;
  for (auto& c : y) {
    if (c.second <= c.first) continue;  // unordered pairs once, no self pairs
    const int dist = lev_token(s[c.first], s[c.second]);
    if (dist <= d) rows.push_back({c.first, c.second, (uint32_t)dist});  // paired
  }
  sort_unique(rows);
  return pack(rows, 3);
}

// Exhaustive paired search over all pairs (the brute-force pin).
void* xo_bruteforce_paired(const uint8_t* seqs, const int64_t* off, int64_t n, int d) {
  std::vector<std::string> s(n);
  for (int64_t i = 0; i < n; ++i) s[i] = seq_at(seqs, off, i);
  std::vector<std::vector<uint32_t>> rows;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      const int dist = lev_token(s[i], s[j]);
      if (dist <= d)
        rows.push_back({static_cast<uint32_t>(i), static_cast<uint32_t>(j),
                        static_cast<uint32_t>(dist)});
    }
  return pack(rows, 3);
}

// TCRdist post-filter over (i, j, dist) rows: keep score <= max_score.
void* xo_tcrdist_filter(const uint8_t* seqs, const int64_t* off, const uint32_t* triples,
                        int64_t n_in, int max_score) {
  std::vector<std::vector<uint32_t>> rows;
  for (int64_t k = 0; k < n_in; ++k) {
    uint32_t i = triples[3 * k], j = triples[3 * k + 1], dist = triples[3 * k + 2];
    if (tcrdist_score(seq_at(seqs, off, i), seq_at(seqs, off, j)) <= max_score)
      rows.push_back({i, j, dist});
  }
  return pack(rows, 3);
}

// All-pairs scorer: every i < j with Lev <= lev_max and TCRdist <= max_score.
// Rows (i, j, lev, score).
void* xo_tcrdist_allpairs(const uint8_t* seqs, const int64_t* off, int64_t n, int lev_max,
                          int max_score) {
  std::vector<std::string> s(n);
  for (int64_t i = 0; i < n; ++i) s[i] = seq_at(seqs, off, i);
  std::vector<std::vector<uint32_t>> rows;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      int score = tcrdist_score(s[i], s[j]);
      if (score > max_score) continue;
      int dist = lev_full(s[i], s[j]);
      if (dist <= lev_max)
        rows.push_back({static_cast<uint32_t>(i), static_cast<uint32_t>(j),
                        static_cast<uint32_t>(dist), static_cast<uint32_t>(score)});
    }
  return pack(rows, 4);
}

}  // extern "C"
