// Duplicate removal and exact verification (Appendix A, XTNeighbor steps 6-7:
// `unique` after the pair sort, then `map` + `if` with the edit distance),
// and the TCRdist post-filter (Results, "SymDel lookup can be combined with
// more advanced similarity metrics").
//
// k_unique_verify reads the sorted pair words, drops a word equal to its
// predecessor (the duplicates of Fig. 1C), drops i == j (one sequence sharing
// a variant with itself through repeated residues) and pairs from different
// repertoires, and computes the Levenshtein distance with a band of 2d+1
// diagonals: only cells with |x - y| <= d can lie on a path of cost <= d, and
// values are capped at d+1, so the band decides "<= d" exactly and returns
// the exact distance when it is <= d.  Survivors are compacted in input
// order (single-pass prefix sum with decoupled look-back), so the output
// stays sorted by (i, j).
#include <algorithm>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

constexpr int VER_THREADS = 256;
constexpr int VER_ITEMS = 8;
constexpr int VER_TILE = VER_THREADS * VER_ITEMS;

// Exact edit distance of a (length la) and b (length lb) if it is <= d,
// otherwise d + 1.  Band index k holds cell (x, y = x + k - d).
__device__ __forceinline__ uint32_t lev_banded(const Key128& a, int la, const Key128& b, int lb,
                                               int d) {
  const int INF = d + 1;
  if (la - lb > d || lb - la > d) return (uint32_t)INF;
  constexpr int W = 2 * XTN_MAX_D + 1;
  int band[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const int y = k - d;
    band[k] = (k <= 2 * d && y >= 0 && y <= lb) ? y : INF;
  }
  for (int x = 1; x <= la; ++x) {
    const uint32_t ca = code_at(a, x - 1);
    int left = INF, rowmin = INF;
    int nb[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      int v = INF;
      const int y = x + k - d;
      if (k <= 2 * d) {
        if (y == 0) {
          v = min(x, INF);
        } else if (y >= 1 && y <= lb) {
          const int diag = band[k] + (ca != code_at(b, y - 1) ? 1 : 0);
          const int up = (k + 1 <= 2 * d) ? band[k + 1] + 1 : INF;
          v = min(min(diag, up), min(left + 1, INF));
        }
      }
      nb[k] = v;
      left = v;
      rowmin = min(rowmin, v);
    }
#pragma unroll
    for (int k = 0; k < W; ++k) band[k] = nb[k];
    if (rowmin > d) return (uint32_t)INF;
  }
  return (uint32_t)min(band[lb - la + d], INF);
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

__global__ void __launch_bounds__(VER_THREADS)
    k_unique_verify(const uint64_t* __restrict__ pairs, int64_t n, uint32_t j_bits,
                    const Key128* __restrict__ keys_i, const uint8_t* __restrict__ lens_i,
                    const Key128* __restrict__ keys_j, const uint8_t* __restrict__ lens_j,
                    uint64_t n_i, uint64_t n_j, const uint32_t* __restrict__ seq_rep,
                    int self_mode, int d,
                    xtn_triple* __restrict__ out, int64_t cap, uint64_t* __restrict__ status,
                    uint32_t* __restrict__ ctr, uint32_t* __restrict__ err,
                    uint64_t* __restrict__ total_out) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_w[VER_THREADS / 32];
  __shared__ uint64_t s_prefix;
  const uint32_t tile = tile_id(ctr, &s_tile);
  const int64_t tbase = (int64_t)tile * VER_TILE;
  const int64_t base = tbase + (int64_t)threadIdx.x * VER_ITEMS;
  const uint64_t jmask = (1ull << j_bits) - 1ull;
  uint64_t prev = (base > 0 && base - 1 < n) ? pairs[base - 1] : ~0ull;
  uint32_t keep = 0;
  uint32_t dist[VER_ITEMS];
  uint32_t cnt = 0;
#pragma unroll
  for (int it = 0; it < VER_ITEMS; ++it) {
    dist[it] = 0;
    const int64_t p = base + it;
    if (p < n) {
      const uint64_t w = pairs[p];
      const uint32_t i = (uint32_t)(w >> j_bits), j = (uint32_t)(w & jmask);
      bool ok = w != prev;
      if (i >= n_i || j >= n_j) {
        atomicOr(err, DERR_RANGE);
        ok = false;
      }
      if (self_mode) ok = ok && i != j;
      if (ok && seq_rep) ok = seq_rep[i] == seq_rep[j];
      if (ok) {
        const uint32_t dd = lev_banded(keys_i[i], lens_i[i], keys_j[j], lens_j[j], d);
        ok = dd <= (uint32_t)d;
        dist[it] = dd;
      }
      keep |= (uint32_t)ok << it;
      cnt += ok;
      prev = w;
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
  for (int it = 0; it < VER_ITEMS; ++it) {
    if (keep >> it & 1u) {
      if (o < cap) {
        const uint64_t w = pairs[base + it];
        xtn_triple t;
        t.i = (uint32_t)(w >> j_bits);
        t.j = (uint32_t)(w & jmask);
        t.dist = dist[it];
        out[o] = t;
      }
      ++o;
    }
  }
}

size_t verify_status_bytes(int64_t n) { return (size_t)((n + VER_TILE - 1) / VER_TILE) * 8 + 16; }

void launch_unique_verify(const uint64_t* pairs, int64_t n, uint32_t j_bits, const Key128* keys_i,
                          const uint8_t* lens_i, const Key128* keys_j, const uint8_t* lens_j,
                          uint64_t n_i, uint64_t n_j, const uint32_t* seq_rep, int self_mode,
                          int d, xtn_triple* out,
                          int64_t cap, uint64_t* status, uint32_t* err, uint64_t* total,
                          cudaStream_t s) {
  if (n <= 0) return;
  const size_t st = verify_status_bytes(n);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(status) + st - 16);
  cudaMemsetAsync(status, 0, st, s);
  prof_begin(s, "k_unique_verify", (double)n * (8.0 + 2 * 17.0));
  k_unique_verify<<<div_up_u32(n, VER_TILE), VER_THREADS, 0, s>>>(
      pairs, n, j_bits, keys_i, lens_i, keys_j, lens_j, n_i, n_j, seq_rep, self_mode, d, out, cap,
      status, ctr, err, total);
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
