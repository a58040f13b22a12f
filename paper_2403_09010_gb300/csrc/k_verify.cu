// Exact verification and duplicate removal (Appendix A, XTNeighbor steps 6-7:
// `map` + `if` with the edit distance, `sort` + `unique`), and the TCRdist
// post-filter (Results, "SymDel lookup can be combined with more advanced
// similarity metrics").
//
// The paper removes duplicate pairs first and verifies after; here every
// candidate is verified first and only the survivors are sorted: the
// duplicates of Fig. 1C are cheap to verify but costly to sort, and the
// output is the same set either way.
//
//   k_verify_candidates : per candidate (i, j): drop i == j (one sequence
//                         sharing a variant with itself through repeated
//                         residues) and pairs from different repertoires
//                         (from the same one when searching between them),
//                         reject |len_i - len_j| > d, compute the edit
//                         distance bit-parallel, keep it if <= d.  Survivors
//                         are appended with one atomic per warp; their radix
//                         histograms are accumulated on the way.
//   k_unique_finalize   : over the sorted survivors, drop a word equal to its
//                         predecessor (the duplicates of Fig. 1C) and write
//                         {i, j, dist} rows in order (single-pass compaction
//                         with decoupled look-back).
//
// Edit distance: the bit-vector algorithm of Myers (1999) in the global-
// distance form of Hyyro (2001).  Pattern i (<= 25 residues) lives in one
// 32-bit word; its match vectors come from the per-sequence table built by
// k_peq; the text j is streamed from its packed key, 5 bits per step.
#include <algorithm>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

constexpr int VER_THREADS = 256;
constexpr int VER_ITEMS = 8;
constexpr int VER_TILE = VER_THREADS * VER_ITEMS;
static_assert(VER_TILE == VERIFY_TILE, "status sizing in xtn_kernels.h assumes this tile");

// Levenshtein distance between pattern (match vectors peq, length m) and the
// text held in packed key t (length n <= XTN_MAX_LEN).  All match vectors the
// text needs are loaded first (independent loads, one latency), then the
// bit-vector recurrence runs from registers, unrolled over XTN_MAX_LEN steps
// with the steps past n switched off.
__device__ __forceinline__ uint32_t edit_distance(const uint32_t* __restrict__ peq, uint32_t m,
                                                  Key128 t, uint32_t n) {
  uint32_t eqv[XTN_MAX_LEN];
#pragma unroll
  for (int j = 0; j < XTN_MAX_LEN; ++j) {
    const uint32_t c = (uint32_t)(t.lo & 31u);
    t.lo = (t.lo >> 5) | (t.hi << 59);
    t.hi >>= 5;
    eqv[j] = ((uint32_t)j < n && c - 1u < 20u) ? __ldg(peq + (c - 1u)) : 0u;
  }
  if (m == 0) return n;
  uint32_t pv = (m >= 32) ? ~0u : ((1u << m) - 1u);
  uint32_t mv = 0;
  uint32_t score = m;
  const uint32_t hb = 1u << (m - 1);
#pragma unroll
  for (int j = 0; j < XTN_MAX_LEN; ++j) {
    // a lane leaves after its own text, so a warp runs the steps of its
    // longest text, not XTN_MAX_LEN
    if ((uint32_t)j >= n) break;
    {
      const uint32_t eq = eqv[j];
      const uint32_t xv = eq | mv;
      const uint32_t xh = (((eq & pv) + pv) ^ pv) | eq;
      uint32_t ph = mv | ~(xh | pv);
      uint32_t mh = pv & xh;
      score += (ph & hb) ? 1u : 0u;
      score -= (mh & hb) ? 1u : 0u;
      ph = (ph << 1) | 1u;
      mh <<= 1;
      pv = mh | ~(xv | ph);
      mv = ph & xv;
    }
  }
  return score;
}

// Hamming distance (the last step of the Hamming variant, Results) between
// pattern (match vectors peq) and text t of the same length n: the positions
// p whose text residue's match vector lacks bit p.
__device__ __forceinline__ uint32_t hamming_distance(const uint32_t* __restrict__ peq, Key128 t,
                                                     uint32_t n) {
  uint32_t match = 0;
#pragma unroll
  for (int j = 0; j < XTN_MAX_LEN; ++j) {
    const uint32_t c = (uint32_t)(t.lo & 31u);
    t.lo = (t.lo >> 5) | (t.hi << 59);
    t.hi >>= 5;
    if ((uint32_t)j < n && c - 1u < 20u) match |= __ldg(peq + (c - 1u)) & (1u << j);
  }
  return n - (uint32_t)__popc(match);
}

// The distance of the last step: metric 0 = Levenshtein (<= d needs
// |m - n| <= d), 1 = Hamming (equal lengths only).  Returns d + 1 for a pair
// that cannot be within d.
__device__ __forceinline__ uint32_t pair_distance(int metric, int d,
                                                  const uint32_t* __restrict__ peq, uint32_t m,
                                                  Key128 t, uint32_t n) {
  if (metric == 1) return m == n ? hamming_distance(peq, t, n) : (uint32_t)d + 1u;
  if ((m > n ? m - n : n - m) > (uint32_t)d) return (uint32_t)d + 1u;
  return edit_distance(peq, m, t, n);
}

// Distance of candidate (i, j) for the last step: pair_distance of the one
// chain, or for paired receptors (metric 2) the sum of both chains' edit
// distances (a pair with |dLa| + |dLb| > d gets d + 1).  d >= XTN_MAX_LEN
// asks for the exact distance.
__device__ __forceinline__ uint32_t cand_distance(int metric, int d,
                                                  const uint32_t* __restrict__ peq_i,
                                                  const uint8_t* __restrict__ lens_i,
                                                  const Key128* __restrict__ keys_j,
                                                  const uint8_t* __restrict__ lens_j,
                                                  const SecondChain& sc, uint64_t i, uint64_t j) {
  if (metric != 2)
    return pair_distance(metric, d, peq_i + i * PEQ_STRIDE, lens_i[i], keys_j[j], lens_j[j]);
  const uint32_t ma = lens_i[i], na = lens_j[j], mb = sc.lens_i[i], nb = sc.lens_j[j];
  const uint32_t gap = (ma > na ? ma - na : na - ma) + (mb > nb ? mb - nb : nb - mb);
  if (gap > (uint32_t)d) return (uint32_t)d + 1u;
  return edit_distance(peq_i + i * PEQ_STRIDE, ma, keys_j[j], na) +
         edit_distance(sc.peq_i + i * PEQ_STRIDE, mb, sc.keys_j[j], nb);
}

template <int THREADS>
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* s_w, uint32_t& excl) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL_MASK, inc, o);
    if (lane >= (uint32_t)o) inc += t;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  uint32_t off = 0, total = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) {
    if (w < (int)warp) off += s_w[w];
    total += s_w[w];
  }
  excl = off + inc - v;
  __syncthreads();
  return total;
}

constexpr uint32_t VER_STASH = 256;  // survivor words a warp collects before a flush

__global__ void __launch_bounds__(256)
    k_verify_candidates(const uint64_t* __restrict__ cand, uint64_t n_cap,
                        const uint64_t* __restrict__ n_dev, uint32_t j_bits,
                        const uint32_t* __restrict__ peq_i, const uint8_t* __restrict__ lens_i,
                        uint64_t n_i, const Key128* __restrict__ keys_j,
                        const uint8_t* __restrict__ lens_j, uint64_t n_j,
                        const uint32_t* __restrict__ seq_rep, int self_mode, int d, int metric,
                        uint64_t* __restrict__ surv, uint64_t surv_cap,
                        unsigned long long* __restrict__ n_surv, uint32_t* __restrict__ hist,
                        int hist_hi, uint32_t* __restrict__ err, SecondChain sc) {
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  // survivors collect per warp and go out VER_STASH - 31 or more at a time:
  // one reservation on the shared counter per flush, not per 32 candidates
  __shared__ uint64_t s_stash[256 / 32][VER_STASH];
  const int passes = (hist_hi + 7) / 8;
  for (int k = threadIdx.x; k < passes * RADIX; k += blockDim.x) s_hist[k] = 0;
  __syncthreads();
  const uint64_t n = n_dev ? min(*n_dev, n_cap) : n_cap;
  const uint32_t lane = lane_id();
  uint64_t* stash = s_stash[threadIdx.x >> 5];
  uint32_t held = 0;  // words in this warp's stash
  auto flush = [&]() {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(n_surv, (unsigned long long)held);
    base = __shfl_sync(FULL_MASK, base, 0);
    for (uint32_t k = lane; k < held; k += 32) {
      if (base + k < surv_cap) surv[base + k] = stash[k];
      else atomicOr(err, DERR_RANGE);
    }
    __syncwarp();  // the stash is refilled next
    held = 0;
  };
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t jmask = (1ull << j_bits) - 1ull;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < n;
       t0 += stride) {
    const uint64_t t = t0 + lane;
    bool ok = false;
    uint64_t w = 0;
    if (t < n) {
      w = cand[t];
      const uint64_t i = w >> j_bits, j = w & jmask;
      ok = i < n_i && j < n_j;
      if (!ok) atomicOr(err, DERR_RANGE);
      if (self_mode) ok = ok && i != j;
      if (ok && seq_rep) ok = (seq_rep[i] == seq_rep[j]) == (self_mode != 2);
      if (ok) {
        const uint32_t dist = cand_distance(metric, d, peq_i, lens_i, keys_j, lens_j, sc, i, j);
        ok = dist <= (uint32_t)d;
        // the distance rides above the pair bits, for the dedup to write it
        if (ok && hist_hi + 8 <= 64) w |= (uint64_t)dist << hist_hi;
      }
    }
    const uint32_t bal = __ballot_sync(FULL_MASK, ok);
    if (ok) {
      stash[held + __popc(bal & lt_mask)] = w;
      for (int p = 0; p < passes; ++p) {
        const int sh = 8 * p;
        const int bits = min(8, hist_hi - sh);
        atomicAdd(&s_hist[p * RADIX + (uint32_t)((w >> sh) & ((1u << bits) - 1u))], 1u);
      }
    }
    held += (uint32_t)__popc(bal);
    __syncwarp();
    if (held > VER_STASH - 32) flush();  // warp-uniform
  }
  if (held) flush();
  __syncthreads();
  for (int k = threadIdx.x; k < passes * RADIX; k += blockDim.x)
    if (s_hist[k]) atomicAdd(&hist[k], s_hist[k]);
}

void launch_verify_candidates(const uint64_t* cand, uint64_t n, const uint64_t* n_dev,
                              uint32_t j_bits,
                              const uint32_t* peq_i, const uint8_t* lens_i, uint64_t n_i,
                              const Key128* keys_j, const uint8_t* lens_j, uint64_t n_j,
                              const uint32_t* seq_rep, int self_mode, int d, int metric,
                              uint64_t* surv, uint64_t surv_cap, uint64_t* n_surv, uint32_t* hist,
                              int hist_hi, int sms, uint32_t* err, cudaStream_t s,
                              const SecondChain& sc) {
  if (n == 0) return;
  const int blocks = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 8);
  prof_begin(s, "k_verify_candidates", (double)n * (8.0 + 2 * 17.0 + 4.0 * 4));
  k_verify_candidates<<<blocks, 256, 0, s>>>(
      cand, n, n_dev, j_bits, peq_i, lens_i, n_i, keys_j, lens_j, n_j, seq_rep, self_mode, d, metric, surv,
      surv_cap, reinterpret_cast<unsigned long long*>(n_surv), hist, hist_hi, err, sc);
  prof_end(s);
}

__global__ void __launch_bounds__(VER_THREADS)
    k_unique_finalize(const uint64_t* __restrict__ pairs, int64_t n_cap,
                      const uint64_t* __restrict__ n_dev, uint32_t j_bits,
                      const uint32_t* __restrict__ peq_i, const uint8_t* __restrict__ lens_i,
                      uint64_t n_i, const Key128* __restrict__ keys_j,
                      const uint8_t* __restrict__ lens_j, uint64_t n_j,
                      int metric, xtn_triple* __restrict__ out, int64_t cap,
                      uint64_t* __restrict__ status, uint32_t* __restrict__ ctr,
                      uint32_t* __restrict__ err, uint64_t* __restrict__ total_out,
                      SecondChain sc, int dist_shift) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_w[VER_THREADS / 32];
  __shared__ uint64_t s_prefix;
  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t jmask = (1ull << j_bits) - 1ull;
  // persistent: every block takes tiles in start order until the input runs out
  for (;;) {
  const uint32_t tile = tile_id(ctr, &s_tile);
  const int64_t tbase = (int64_t)tile * VER_TILE;
  if (tbase >= n) break;
  // warp w covers positions [wbase, wbase + 32 * ITEMS), lane l position
  // wbase + it * 32 + l of round it: reads coalesce and the rounds follow
  // position order, so ballots compact each round in order
  const int64_t wbase = tbase + (int64_t)warp * 32 * VER_ITEMS;
  uint32_t keep = 0, wtotal = 0;
  uint32_t rank[VER_ITEMS], dist[VER_ITEMS];
  uint64_t word[VER_ITEMS];
#pragma unroll
  for (int it = 0; it < VER_ITEMS; ++it) {
    const int64_t p = wbase + it * 32 + lane;
    bool ok = false;
    dist[it] = 0;
    word[it] = 0;
    if (p < n) {
      const uint64_t w = pairs[p];
      const uint64_t prev = p > 0 ? pairs[p - 1] : ~w;
      // with dist_shift the verified distance sits above the pair bits (the
      // same pair always carries the same distance, so equal pairs are equal
      // words); else it is computed again
      const uint64_t pw = dist_shift ? (w & ((1ull << dist_shift) - 1ull)) : w;
      const uint64_t i = pw >> j_bits, j = pw & jmask;
      ok = w != prev;
      if (i >= n_i || j >= n_j) {
        atomicOr(err, DERR_RANGE);
        ok = false;
      }
      if (ok)
        dist[it] = dist_shift ? (uint32_t)((w >> dist_shift) & 0xffu)
                              : cand_distance(metric, 2 * XTN_MAX_LEN, peq_i, lens_i, keys_j,
                                              lens_j, sc, i, j);
      word[it] = pw;
    }
    const uint32_t bal = __ballot_sync(FULL_MASK, ok);
    rank[it] = wtotal + __popc(bal & lt_mask);
    wtotal += __popc(bal);
    keep |= (uint32_t)ok << it;
  }
  if (lane == 0) s_w[warp] = wtotal;
  __syncthreads();
  uint32_t woff = 0, total = 0;
#pragma unroll
  for (int w = 0; w < VER_THREADS / 32; ++w) {
    if (w < (int)warp) woff += s_w[w];
    total += s_w[w];
  }
  if (warp == 0) {
    const uint64_t pre = warp_lookback(status, tile, total, err);
    if (lane == 0) {
      s_prefix = pre;
      if (tbase + VER_TILE >= n) *total_out = pre + total;
    }
  }
  __syncthreads();
  const int64_t o0 = (int64_t)(s_prefix + woff);
#pragma unroll
  for (int it = 0; it < VER_ITEMS; ++it) {
    if (keep >> it & 1u) {
      const int64_t o = o0 + rank[it];
      if (o < cap) {
        xtn_triple t;
        t.i = (uint32_t)(word[it] >> j_bits);
        t.j = (uint32_t)(word[it] & jmask);
        t.dist = dist[it];
        out[o] = t;
      }
    }
  }
  __syncthreads();  // s_prefix, s_w and s_tile are reused by the next tile
  }
}

size_t verify_status_bytes(int64_t n) { return verify_status_bytes_for(n); }

void launch_unique_finalize(const uint64_t* pairs, int64_t n, const uint64_t* n_dev,
                            uint32_t j_bits,
                            const uint32_t* peq_i, const uint8_t* lens_i, uint64_t n_i,
                            const Key128* keys_j, const uint8_t* lens_j, uint64_t n_j,
                            int metric, xtn_triple* out, int64_t cap, uint64_t* status,
                            uint32_t* err, uint64_t* total, cudaStream_t s,
                            const SecondChain& sc, int dist_shift) {
  if (n <= 0) return;
  const size_t st = verify_status_bytes(n);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(status) + st - 16);
  cudaMemsetAsync(status, 0, st, s);
  prof_begin(s, "k_unique_finalize", (double)n * 8.0);
  k_unique_finalize<<<std::min<uint32_t>(div_up_u32(n, VER_TILE), 152 * 8), VER_THREADS, 0, s>>>(
      pairs, n, n_dev, j_bits, peq_i, lens_i, n_i, keys_j, lens_j, n_j, metric, out, cap, status,
      ctr, err, total, sc, dist_shift);
  prof_end(s);
}

// ------------------------------------------------------------- TCRdist ---
// BLOSUM62 (Henikoff & Henikoff 1992), rows and columns in residue-code order
// A C D E F G H I K L M N P Q R S T V W Y.
__constant__ int8_t c_blosum62[20][20] = {
    /*A*/ {4, 0, -2, -1, -2, 0, -2, -1, -1, -1, -1, -2, -1, -1, -1, 1, 0, 0, -3, -2},
    /*C*/ {0, 9, -3, -4, -2, -3, -3, -1, -3, -1, -1, -3, -3, -3, -3, -1, -1, -1, -2, -2},
    /*D*/ {-2, -3, 6, 2, -3, -1, -1, -3, -1, -4, -3, 1, -1, 0, -2, 0, -1, -3, -4, -3},
    /*E*/ {-1, -4, 2, 5, -3, -2, 0, -3, 1, -3, -2, 0, -1, 2, 0, 0, -1, -2, -3, -2},
    /*F*/ {-2, -2, -3, -3, 6, -3, -1, 0, -3, 0, 0, -3, -4, -3, -3, -2, -2, -1, 1, 3},
    /*G*/ {0, -3, -1, -2, -3, 6, -2, -4, -2, -4, -3, 0, -2, -2, -2, 0, -2, -3, -2, -3},
    /*H*/ {-2, -3, -1, 0, -1, -2, 8, -3, -1, -3, -2, 1, -2, 0, 0, -1, -2, -3, -2, 2},
    /*I*/ {-1, -1, -3, -3, 0, -4, -3, 4, -3, 2, 1, -3, -3, -3, -3, -2, -1, 3, -3, -1},
    /*K*/ {-1, -3, -1, 1, -3, -2, -1, -3, 5, -2, -1, 0, -1, 1, 2, 0, -1, -2, -3, -2},
    /*L*/ {-1, -1, -4, -3, 0, -4, -3, 2, -2, 4, 2, -3, -3, -2, -2, -2, -1, 1, -2, -1},
    /*M*/ {-1, -1, -3, -2, 0, -3, -2, 1, -1, 2, 5, -2, -2, 0, -1, -1, -1, 1, -1, -1},
    /*N*/ {-2, -3, 1, 0, -3, 0, 1, -3, 0, -3, -2, 6, -2, 0, 0, 1, 0, -3, -4, -2},
    /*P*/ {-1, -3, -1, -1, -4, -2, -2, -3, -1, -3, -2, -2, 7, -1, -2, -1, -1, -2, -4, -3},
    /*Q*/ {-1, -3, 0, 2, -3, -2, 0, -3, 1, -2, 0, 0, -1, 5, 1, 0, -1, -2, -2, -1},
    /*R*/ {-1, -3, -2, 0, -3, -2, 0, -3, 2, -2, -1, 0, -2, 1, 5, -1, -1, -3, -3, -2},
    /*S*/ {1, -1, 0, 0, -2, 0, -1, -2, 0, -2, -1, 1, -1, 0, -1, 4, 1, -2, -3, -2},
    /*T*/ {0, -1, -1, -1, -2, -2, -2, -1, -1, -1, -1, 0, -1, -1, -1, 1, 5, 0, -2, -2},
    /*V*/ {0, -1, -3, -2, -1, -3, -3, 3, -2, 1, 1, -3, -2, -2, -3, -2, 0, 4, -3, -1},
    /*W*/ {-3, -2, -4, -3, 1, -2, -2, -3, -3, -2, -1, -4, -4, -2, -3, -3, -2, -3, 11, 2},
    /*Y*/ {-2, -2, -3, -2, 3, -3, 2, -1, -2, -1, -1, -2, -3, -1, -2, -2, -2, -1, 2, 7},
};

// TCRdist-style CDR3 score: gaps after the first floor(m/2) residues of the
// shorter sequence, mismatch cost min(4, 4 - BLOSUM62), gap cost 4, weight 3.
__device__ __forceinline__ int tcrdist_score(const Key128& a, int la, const Key128& b, int lb) {
  const bool a_short = la <= lb;
  const Key128& sk = a_short ? a : b;
  const Key128& lk = a_short ? b : a;
  const int m = a_short ? la : lb;
  const int g = (a_short ? lb : la) - m;
  const int p = m / 2;
  int sum = 0;
  for (int k = 0; k < m; ++k) {
    const uint32_t x = code_at(sk, k);
    const uint32_t y = code_at(lk, k < p ? k : k + g);
    if (x != y) sum += min(4, 4 - (int)c_blosum62[x - 1][y - 1]);
  }
  return 3 * (sum + 4 * g);
}

__global__ void __launch_bounds__(VER_THREADS)
    k_tcrdist_filter(const xtn_triple* __restrict__ in, int64_t n, const Key128* __restrict__ keys,
                     const uint8_t* __restrict__ lens, int64_t n_seq, int max_score,
                     xtn_triple* __restrict__ out, uint64_t* __restrict__ status,
                     uint32_t* __restrict__ ctr, uint32_t* __restrict__ err,
                     uint64_t* __restrict__ total_out) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_w[VER_THREADS / 32];
  __shared__ uint64_t s_prefix;
  const uint32_t tile = tile_id(ctr, &s_tile);
  const int64_t tbase = (int64_t)tile * VER_TILE;
  const int64_t base = tbase + (int64_t)threadIdx.x * VER_ITEMS;
  uint32_t keep = 0, cnt = 0;
#pragma unroll
  for (int it = 0; it < VER_ITEMS; ++it) {
    const int64_t p = base + it;
    if (p < n) {
      const xtn_triple t = in[p];
      bool ok = false;
      if (t.i < n_seq && t.j < n_seq) {
        ok = tcrdist_score(keys[t.i], lens[t.i], keys[t.j], lens[t.j]) <= max_score;
      } else {
        atomicOr(err, DERR_RANGE);
      }
      keep |= (uint32_t)ok << it;
      cnt += ok;
    }
  }
  uint32_t excl;
  const uint32_t total = block_excl_scan_u32<VER_THREADS>(cnt, s_w, excl);
  if (threadIdx.x < 32) {
    const uint64_t pre = warp_lookback(status, tile, total, err);
    if (threadIdx.x == 0) {
      s_prefix = pre;
      if (tbase + VER_TILE >= n) *total_out = pre + total;
    }
  }
  __syncthreads();
  int64_t o = (int64_t)(s_prefix + excl);
#pragma unroll
  for (int it = 0; it < VER_ITEMS; ++it)
    if (keep >> it & 1u) {
      if (o < n) out[o] = in[base + it];
      ++o;
    }
}

void launch_tcrdist_filter(const xtn_triple* in, int64_t n, const Key128* keys,
                           const uint8_t* lens, int64_t n_seq, int max_score, xtn_triple* out,
                           uint64_t* status, uint32_t* err, uint64_t* total, cudaStream_t s) {
  if (n <= 0) return;
  const size_t st = verify_status_bytes(n);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(status) + st - 16);
  cudaMemsetAsync(status, 0, st, s);
  prof_begin(s, "k_tcrdist_filter", (double)n * (12.0 * 2 + 2 * 17.0));
  k_tcrdist_filter<<<div_up_u32(n, VER_TILE), VER_THREADS, 0, s>>>(
      in, n, keys, lens, n_seq, max_score, out, status, ctr, err, total);
  prof_end(s);
}

}  // namespace xtn
