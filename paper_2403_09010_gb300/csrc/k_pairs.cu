// Grouping and candidate-pair generation (Appendix A, XTNeighbor steps 4-5).
//
//   k_scan_counts  : exclusive prefix sum (single pass, decoupled look-back)
//                    of per-sequence variant counts -> record offsets, and of
//                    per-group pair counts -> pair offsets (the paper's
//                    `cumulativeSum`).
//   k_group_bounds : on the sorted records, a group is a run of equal
//                    fingerprints (the paper's `uniqueCount`).  Only groups of
//                    two or more records can yield pairs; their first and
//                    last positions are compacted into S[] and E[] in one read
//                    of the records.  The k-th group start and the k-th group
//                    end describe the same group, so no thread ever walks a
//                    group, however large.
//   k_emit_pairs   : the `expand` of step 5.  Group k owns C(E-S+1, 2) output
//                    slots; output slot t finds its group by binary search over
//                    the pair offsets (staged in shared memory per tile), turns
//                    its rank inside the group into positions a < b and writes
//                    (id_a << b) | id_b.  Work per thread is constant whatever
//                    the group sizes, so one huge bucket is spread over every
//                    block instead of serialising one of them.
#include <algorithm>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct CountsU32 {
  const uint32_t* v;
  __device__ uint64_t operator()(int64_t k) const { return v[k]; }
};
struct PairsOfGroup {
  const uint32_t* S;
  const uint32_t* E;
  __device__ uint64_t operator()(int64_t k) const {
    const uint64_t m = (uint64_t)E[k] - S[k] + 1;
    return m * (m - 1) / 2;
  }
};

// Block-wide exclusive scan of one u64 per thread; returns the block total.
template <int THREADS>
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* s_w, uint64_t& excl) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint64_t inc = warp_incl_scan_u64(v);
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  uint64_t off = 0, total = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) {
    if (w < (int)warp) off += s_w[w];
    total += s_w[w];
  }
  excl = off + inc - v;
  __syncthreads();
  return total;
}

// out[k] = sum_{k' < k} f(k') for k <= n (out[n] = total).
template <class F>
__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_counts(F f, int64_t n, uint64_t* __restrict__ out, uint64_t* __restrict__ status,
                  uint32_t* __restrict__ ctr, uint32_t* __restrict__ err) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_w[SCAN_THREADS / 32];
  __shared__ uint64_t s_prefix;
  const uint32_t tile = tile_id(ctr, &s_tile);
  const int64_t base = (int64_t)tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint64_t v[SCAN_ITEMS];
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = (base + i < n) ? f(base + i) : 0ull;
    sum += v[i];
  }
  uint64_t excl;
  const uint64_t total = block_excl_scan<SCAN_THREADS>(sum, s_w, excl);
  if (threadIdx.x < 32) {
    const uint64_t p = warp_lookback(status, tile, total, err);
    if (threadIdx.x == 0) s_prefix = p;
  }
  __syncthreads();
  uint64_t run = s_prefix + excl;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
    if (base + i == n - 1) out[n] = run;
  }
}

size_t scan_status_bytes(int64_t n) {
  return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) * 8 + 16;
}

template <class F>
static void scan_launch(F f, int64_t n, uint64_t* out, uint64_t* status, uint32_t* err,
                        const char* tag, double bytes, cudaStream_t s) {
  const size_t st = scan_status_bytes(n);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(status) + st - 16);
  cudaMemsetAsync(status, 0, st, s);
  prof_begin(s, tag, bytes);
  k_scan_counts<<<div_up_u32(n, SCAN_TILE), SCAN_THREADS, 0, s>>>(f, n, out, status, ctr, err);
  prof_end(s);
}

void launch_scan_counts(const uint32_t* counts, int64_t n, uint64_t* out, uint64_t* status,
                        uint32_t* err, cudaStream_t s) {
  if (n <= 0) return;
  scan_launch(CountsU32{counts}, n, out, status, err, "k_scan_counts", (double)n * 12.0, s);
}

void launch_scan_group_pairs(const uint32_t* S, const uint32_t* E, int64_t n_groups,
                             uint64_t* out, uint64_t* status, uint32_t* err, cudaStream_t s) {
  if (n_groups <= 0) return;
  scan_launch(PairsOfGroup{S, E}, n_groups, out, status, err, "k_scan_group_pairs",
              (double)n_groups * 16.0, s);
}

// ----------------------------------------------------------- group bounds ---
constexpr int GB_THREADS = 256;
constexpr int GB_ITEMS = 16;
constexpr int GB_TILE = GB_THREADS * GB_ITEMS;

__global__ void __launch_bounds__(GB_THREADS)
    k_group_bounds(const uint64_t* __restrict__ keys, int64_t n, int gshift,
                   uint32_t* __restrict__ S, uint32_t* __restrict__ E, uint64_t cap,
                   uint64_t* __restrict__ status, uint32_t* __restrict__ ctr,
                   uint32_t* __restrict__ err, uint64_t* __restrict__ n_groups) {
  __shared__ uint64_t s_g[GB_TILE + 2];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_w[GB_THREADS / 32];
  __shared__ uint64_t s_prefix;
  const uint32_t tile = tile_id(ctr, &s_tile);
  const int64_t tbase = (int64_t)tile * GB_TILE;
  // s_g[j] = group key of position tbase - 1 + j; out-of-range positions get
  // sentinels that differ from every real key (keys are >> gshift < 2^(64-gshift)).
  const uint64_t sentinel = ~0ull;
  for (int j = threadIdx.x; j < GB_TILE + 2; j += GB_THREADS) {
    const int64_t p = tbase - 1 + j;
    s_g[j] = (p >= 0 && p < n) ? (__ldcs(keys + p) >> gshift) : sentinel - (p < 0 ? 1 : 0);
  }
  __syncthreads();
  // a multi-record group starts at p when g(p) != g(p-1) and g(p) == g(p+1);
  // it ends at p when g(p) != g(p+1) and g(p) == g(p-1).
  const int j0 = threadIdx.x * GB_ITEMS;
  uint32_t heads = 0, tails = 0;
  uint32_t hmask = 0, tmask = 0;
#pragma unroll
  for (int i = 0; i < GB_ITEMS; ++i) {
    const int64_t p = tbase + j0 + i;
    if (p < n) {
      const uint64_t prev = s_g[j0 + i], cur = s_g[j0 + i + 1], next = s_g[j0 + i + 2];
      const bool h = cur != prev && cur == next;
      const bool t = cur != next && cur == prev;
      hmask |= (uint32_t)h << i;
      tmask |= (uint32_t)t << i;
      heads += h;
      tails += t;
    }
  }
  const uint64_t packed = ((uint64_t)heads << 31) | tails;
  uint64_t excl;
  const uint64_t total = block_excl_scan<GB_THREADS>(packed, s_w, excl);
  if (threadIdx.x < 32) {
    const uint64_t pre = warp_lookback(status, tile, total, err);
    if (threadIdx.x == 0) {
      s_prefix = pre;
      if (tbase + GB_TILE >= n) *n_groups = (pre + total) >> 31;  // last tile
    }
  }
  __syncthreads();
  const uint64_t start = s_prefix + excl;
  uint64_t hk = start >> 31, tk = start & 0x7fffffffull;
#pragma unroll
  for (int i = 0; i < GB_ITEMS; ++i) {
    const uint32_t p = (uint32_t)(tbase + j0 + i);
    if (hmask >> i & 1u) {
      if (hk < cap) S[hk] = p; else atomicOr(err, DERR_RANGE);
      ++hk;
    }
    if (tmask >> i & 1u) {
      if (tk < cap) E[tk] = p; else atomicOr(err, DERR_RANGE);
      ++tk;
    }
  }
}

void launch_group_bounds(const uint64_t* keys, int64_t n, int gshift, uint32_t* S, uint32_t* E,
                         uint64_t cap, uint64_t* status, uint32_t* err, uint64_t* n_groups, cudaStream_t s) {
  if (n <= 0) return;
  const size_t st = (size_t)((n + GB_TILE - 1) / GB_TILE) * 8 + 16;
  uint32_t* ctr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(status) + st - 16);
  cudaMemsetAsync(status, 0, st, s);
  prof_begin(s, "k_group_bounds", (double)n * 8.0);
  k_group_bounds<<<div_up_u32(n, GB_TILE), GB_THREADS, 0, s>>>(keys, n, gshift, S, E, cap, status,
                                                              ctr, err, n_groups);
  prof_end(s);
}

size_t group_status_bytes(int64_t n) { return (size_t)((n + GB_TILE - 1) / GB_TILE) * 8 + 16; }

// ------------------------------------------------------------ pair emit ---
constexpr int EMIT_THREADS = 256;
constexpr int EMIT_ITEMS = 8;
constexpr int EMIT_TILE = EMIT_THREADS * EMIT_ITEMS;

// Largest k in [lo, hi) with off[k] <= t (off non-decreasing, off[lo] <= t).
__device__ __forceinline__ int64_t upper_index(const uint64_t* off, int64_t lo, int64_t hi,
                                               uint64_t t) {
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (off[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// rank l of the pair {a < b} with colex rank b(b-1)/2 + a
__device__ __forceinline__ void unrank_pair(uint64_t l, uint64_t& a, uint64_t& b) {
  b = (uint64_t)((1.0 + sqrt(1.0 + 8.0 * (double)l)) * 0.5);
  while (b * (b - 1) / 2 > l) --b;
  while ((b + 1) * b / 2 <= l) ++b;
  a = l - b * (b - 1) / 2;
}

__global__ void __launch_bounds__(EMIT_THREADS)
    k_emit_pairs(const uint64_t* __restrict__ keys, uint64_t n_keys, const uint32_t* __restrict__ S,
                 const uint64_t* __restrict__ pair_off, int64_t n_groups, uint64_t n_pairs,
                 uint32_t id_bits, uint64_t* __restrict__ out, uint32_t* __restrict__ hist,
                 int hist_hi, uint32_t* __restrict__ err) {
  __shared__ uint64_t s_off[EMIT_TILE + 1];
  __shared__ int64_t s_k0, s_k1;
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  const int passes = (hist_hi + 7) / 8;
  for (int k = threadIdx.x; k < passes * RADIX; k += EMIT_THREADS) s_hist[k] = 0;
  const uint64_t idmask = (1ull << id_bits) - 1ull;
  for (uint64_t t0 = (uint64_t)blockIdx.x * EMIT_TILE; t0 < n_pairs;
       t0 += (uint64_t)gridDim.x * EMIT_TILE) {
    const uint64_t t_last = (t0 + EMIT_TILE < n_pairs ? t0 + EMIT_TILE : n_pairs) - 1;
    if (threadIdx.x == 0) {
      s_k0 = upper_index(pair_off, 0, n_groups, t0);
      s_k1 = upper_index(pair_off, s_k0, n_groups, t_last);
    }
    __syncthreads();
    const int64_t k0 = s_k0;
    int64_t nk = s_k1 - s_k0 + 1;  // <= EMIT_TILE: every group owns >= 1 pair
    if (nk > EMIT_TILE) {
      if (threadIdx.x == 0) atomicOr(err, DERR_RANGE);
      nk = 0;
    }
    for (int j = threadIdx.x; j <= nk; j += EMIT_THREADS) s_off[j] = pair_off[k0 + j];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < EMIT_ITEMS; ++i) {
      const uint64_t t = t0 + (uint64_t)i * EMIT_THREADS + threadIdx.x;
      if (t < n_pairs && nk > 0) {
        int64_t lo = 0, hi = nk;
        while (hi - lo > 1) {
          const int64_t mid = (lo + hi) >> 1;
          if (s_off[mid] <= t) lo = mid; else hi = mid;
        }
        uint64_t a, b;
        unrank_pair(t - s_off[lo], a, b);
        const uint64_t s0 = S[k0 + lo];
        uint64_t w = 0;
        if (s0 + b < n_keys) {
          w = ((keys[s0 + a] & idmask) << id_bits) | (keys[s0 + b] & idmask);
        } else {
          atomicOr(err, DERR_RANGE);
        }
        out[t] = w;
        for (int p = 0; p < passes; ++p) {
          const int sh = 8 * p;
          const int bits = min(8, hist_hi - sh);
          atomicAdd(&s_hist[p * RADIX + (uint32_t)((w >> sh) & ((1u << bits) - 1u))], 1u);
        }
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < passes * RADIX; k += EMIT_THREADS)
    if (s_hist[k]) atomicAdd(&hist[k], s_hist[k]);
}

void launch_emit_pairs(const uint64_t* keys, uint64_t n_keys, const uint32_t* S,
                       const uint64_t* pair_off, int64_t n_groups, uint64_t n_pairs,
                       uint32_t id_bits, uint64_t* out, uint32_t* hist, int sms, uint32_t* err,
                       cudaStream_t s) {
  if (n_pairs == 0) return;
  const uint64_t tiles = (n_pairs + EMIT_TILE - 1) / EMIT_TILE;
  const int blocks = (int)std::min<uint64_t>(tiles, (uint64_t)sms * 8);
  prof_begin(s, "k_emit_pairs", (double)n_pairs * (8.0 + 16.0));
  k_emit_pairs<<<blocks, EMIT_THREADS, 0, s>>>(keys, n_keys, S, pair_off, n_groups, n_pairs,
                                               id_bits, out, hist, (int)(2 * id_bits), err);
  prof_end(s);
}

}  // namespace xtn
