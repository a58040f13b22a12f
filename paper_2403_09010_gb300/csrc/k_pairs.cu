// Grouping and candidate-pair generation (Appendix A, XTNeighbor steps 4-5).
//
//   k_scan_counts  : exclusive prefix sum (single pass, decoupled look-back)
//                    of per-sequence variant counts -> record offsets, and of
//                    per-group pair counts -> pair offsets (the paper's
//                    `cumulativeSum`).
//   group bounds   : on the sorted records, a group is a run of equal
//                    fingerprints (the paper's `uniqueCount`).  Only groups of
//                    two or more records can yield pairs; their first and
//                    last positions are compacted into S[] and E[] with one
//                    read of the records (k_group_flags, k_group_write below).
//                    The k-th group start and the k-th group end describe the
//                    same group, so no thread ever walks a group, however
//                    large.
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
    k_scan_counts(F f, int64_t n_cap, const uint64_t* __restrict__ n_dev,
                  uint64_t* __restrict__ out, uint64_t* __restrict__ status,
                  uint32_t* __restrict__ ctr, uint32_t* __restrict__ err) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_w[SCAN_THREADS / 32];
  __shared__ uint64_t s_prefix;
  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  if (n == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
    return;
  }
  // persistent: every block takes tiles in start order until the input runs out
  for (;;) {
  const uint32_t tile = tile_id(ctr, &s_tile);
  if ((int64_t)tile * SCAN_TILE >= n) break;
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
  __syncthreads();  // s_prefix and s_tile are reused by the next tile
  }
}

size_t scan_status_bytes(int64_t n) {
  return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) * 8 + 16;
}

template <class F>
static void scan_launch(F f, int64_t n, const uint64_t* n_dev, uint64_t* out, uint64_t* status,
                        uint32_t* err, const char* tag, double bytes, cudaStream_t s) {
  const size_t st = scan_status_bytes(n);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(status) + st - 16);
  cudaMemsetAsync(status, 0, st, s);
  prof_begin(s, tag, bytes);
  k_scan_counts<<<std::min<uint32_t>(div_up_u32(n, SCAN_TILE), 152 * 16), SCAN_THREADS, 0, s>>>(
      f, n, n_dev, out, status, ctr, err);
  prof_end(s);
}

void launch_scan_counts(const uint32_t* counts, int64_t n, uint64_t* out, uint64_t* status,
                        uint32_t* err, cudaStream_t s) {
  if (n <= 0) return;
  scan_launch(CountsU32{counts}, n, nullptr, out, status, err, "k_scan_counts", (double)n * 12.0,
              s);
}

void launch_scan_group_pairs(const uint32_t* S, const uint32_t* E, int64_t n_groups,
                             const uint64_t* n_groups_dev, uint64_t* out, uint64_t* status,
                             uint32_t* err, cudaStream_t s) {
  if (n_groups <= 0) return;
  scan_launch(PairsOfGroup{S, E}, n_groups, n_groups_dev, out, status, err, "k_scan_group_pairs",
              (double)n_groups * 16.0, s);
}

// ----------------------------------------------------------- group bounds ---
// Two kernels instead of one single-pass compaction: the per-position work is
// too light for a decoupled look-back (the chain of tile prefixes, not the
// memory, would set the pace), so
//   k_group_flags : reads the records once; per 32 positions writes one word
//                   (head ballot | tail ballot << 32) and per tile the number
//                   of heads and tails (no inter-tile waiting);
//   k_scan_counts : prefix over the tile counts (small);
//   k_group_write : reads only the flag words and writes the k-th head to S[k]
//                   and the k-th tail to E[k].
// A multi-record group starts at p when g(p) != g(p-1) and g(p) == g(p+1) and
// ends at p when g(p) != g(p+1) and g(p) == g(p-1), g = key >> gshift (no
// g(-1), no g(n)).
constexpr int GB_THREADS = 512;
constexpr int GB_WARPS = GB_THREADS / 32;
constexpr int GB_ITEMS = 16;   // positions per lane per chunk
constexpr int GB_CHUNKS = 4;
constexpr int GB_WARP_SPAN = 32 * GB_ITEMS * GB_CHUNKS;
constexpr int GB_TILE = GB_THREADS * GB_ITEMS * GB_CHUNKS;  // 32768 positions
static_assert(GB_TILE == GROUP_FLAG_TILE, "flag tiles shared with k_bucket_sort");

// K = uint32_t when the group key (key >> gshift) fits in 32 bits.
template <typename K>
__global__ void __launch_bounds__(GB_THREADS)
    k_group_flags(const uint64_t* __restrict__ keys, int64_t n_cap,
                  const uint64_t* __restrict__ n_dev, int gshift, uint64_t* __restrict__ flags,
                  uint64_t* __restrict__ tile_counts) {
  __shared__ uint64_t s_wtot[GB_WARPS];
  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  const int64_t tbase = (int64_t)blockIdx.x * GB_TILE;
  if (tbase >= n) {
    if (threadIdx.x == 0) tile_counts[blockIdx.x] = 0;
    return;
  }
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const int64_t wbase = tbase + (int64_t)warp * GB_WARP_SPAN;
  // the value before position wbase (made different from it at position 0)
  K carry = (wbase >= 1 && wbase - 1 < n) ? (K)(keys[wbase - 1] >> gshift) : (K)0;
  uint32_t heads = 0, tails = 0;
#pragma unroll 1
  for (int c = 0; c < GB_CHUNKS; ++c) {
    const int64_t cbase = wbase + (int64_t)c * 32 * GB_ITEMS;
    K cur[GB_ITEMS];
#pragma unroll
    for (int i = 0; i < GB_ITEMS; ++i) {
      const int64_t p = cbase + i * 32 + lane;
      cur[i] = p < n ? (K)(__ldcs(keys + p) >> gshift) : (K)0;
    }
    const int64_t pe = cbase + 32 * GB_ITEMS;
    const K after = (pe < n) ? (K)(keys[pe] >> gshift) : (K)0;
    uint64_t mine = 0;  // lane i keeps the flag word of item i
#pragma unroll
    for (int i = 0; i < GB_ITEMS; ++i) {
      const int64_t p = cbase + i * 32 + lane;
      K prev = __shfl_up_sync(FULL_MASK, cur[i], 1);
      if (lane == 0) prev = carry;
      K next = __shfl_down_sync(FULL_MASK, cur[i], 1);
      const K first_next =
          (i + 1 < GB_ITEMS) ? __shfl_sync(FULL_MASK, cur[i + 1 < GB_ITEMS ? i + 1 : i], 0) : after;
      if (lane == 31) next = first_next;
      carry = __shfl_sync(FULL_MASK, cur[i], 31);
      if (p == 0) prev = cur[i] ^ (K)1;      // nothing before the first position
      if (p == n - 1) next = cur[i] ^ (K)1;  // nothing after the last one
      const bool valid = p < n;
      const uint32_t hb = __ballot_sync(FULL_MASK, valid && cur[i] != prev && cur[i] == next);
      const uint32_t tb = __ballot_sync(FULL_MASK, valid && cur[i] != next && cur[i] == prev);
      if (lane == (uint32_t)i) mine = ((uint64_t)tb << 32) | hb;
      heads += __popc(hb);
      tails += __popc(tb);
    }
    const int64_t word = cbase / 32 + lane;  // 16 consecutive words per chunk
    if (lane < GB_ITEMS && word * 32 < n) flags[word] = mine;
  }
  if (lane == 0) s_wtot[warp] = ((uint64_t)heads << 31) | tails;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t total = 0;
#pragma unroll
    for (int w = 0; w < GB_WARPS; ++w) total += s_wtot[w];
    tile_counts[blockIdx.x] = total;
  }
}

__global__ void __launch_bounds__(GB_THREADS)
    k_group_write(const uint64_t* __restrict__ flags, int64_t n_cap,
                  const uint64_t* __restrict__ n_dev, const uint64_t* __restrict__ tile_prefix,
                  uint32_t* __restrict__ S, uint32_t* __restrict__ E, uint64_t cap,
                  uint32_t* __restrict__ err) {
  __shared__ uint64_t s_w[GB_WARPS];
  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  const int64_t tbase = (int64_t)blockIdx.x * GB_TILE;
  if (tbase >= n) return;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  // each warp owns GB_WARP_SPAN / 32 flag words; lane l holds words l, l+32, ...
  constexpr int WPW = GB_WARP_SPAN / 32;  // words per warp (64)
  const int64_t w0 = tbase / 32 + (int64_t)warp * WPW;
  const int64_t n_words = (n + 31) / 32;
  uint64_t fw[WPW / 32];
  uint32_t h = 0, t = 0;
#pragma unroll
  for (int k = 0; k < WPW / 32; ++k) {
    const int64_t wi = w0 + k * 32 + lane;
    fw[k] = wi < n_words ? flags[wi] : 0ull;
    h += __popc((uint32_t)fw[k]);
    t += __popc((uint32_t)(fw[k] >> 32));
  }
  // exclusive prefix of (h, t) over lanes in word order, then over warps
  uint64_t mine = ((uint64_t)h << 31) | t;
  const uint64_t inc = warp_incl_scan_u64(mine);
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  uint64_t off = tile_prefix[blockIdx.x];
#pragma unroll
  for (int w = 0; w < GB_WARPS; ++w)
    if (w < (int)warp) off += s_w[w];
  uint64_t hk = off >> 31, tk = off & 0x7fffffffull;
#pragma unroll
  for (int k = 0; k < WPW / 32; ++k) {
    // lane l holds word w0 + 32k + l; prefix over lanes of this round
    const uint32_t hc = __popc((uint32_t)fw[k]), tc = __popc((uint32_t)(fw[k] >> 32));
    uint32_t hx = hc, tx = tc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t a = __shfl_up_sync(FULL_MASK, hx, o);
      const uint32_t b = __shfl_up_sync(FULL_MASK, tx, o);
      if (lane >= (uint32_t)o) {
        hx += a;
        tx += b;
      }
    }
    const uint32_t htot = __shfl_sync(FULL_MASK, hx, 31), ttot = __shfl_sync(FULL_MASK, tx, 31);
    uint64_t hq = hk + hx - hc, tq = tk + tx - tc;
    const uint32_t pbase = (uint32_t)((w0 + k * 32 + lane) * 32);
    uint32_t hb = (uint32_t)fw[k], tb = (uint32_t)(fw[k] >> 32);
    while (hb) {
      const int b = __ffs(hb) - 1;
      hb &= hb - 1;
      if (hq < cap) S[hq] = pbase + b; else atomicOr(err, DERR_RANGE);
      ++hq;
    }
    while (tb) {
      const int b = __ffs(tb) - 1;
      tb &= tb - 1;
      if (tq < cap) E[tq] = pbase + b; else atomicOr(err, DERR_RANGE);
      ++tq;
    }
    hk += htot;
    tk += ttot;
  }
}

__global__ void k_groups_total(const uint64_t* __restrict__ total, uint64_t* __restrict__ n_groups) {
  *n_groups = *total >> 31;
}

struct CountsU64 {
  const uint64_t* v;
  __device__ uint64_t operator()(int64_t k) const { return v[k]; }
};

size_t group_status_bytes(int64_t n) {
  const int64_t tiles = (n + GB_TILE - 1) / GB_TILE;
  return scan_status_bytes(tiles) + (size_t)tiles * 16 + 64;
}

size_t group_flag_words(int64_t n) { return (size_t)((n + 31) / 32); }

// Scratch layout in `status`: [scan status][tile counts][tile prefix (tiles+1)].
uint64_t* group_tile_counts(uint64_t* status, int64_t n) {
  const int64_t tiles = (n + GB_TILE - 1) / GB_TILE;
  return reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(status) + scan_status_bytes(tiles));
}

void launch_group_flags(const uint64_t* keys, int64_t n, const uint64_t* n_dev, int gshift,
                        uint64_t* flags, uint64_t* status, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t tiles = (n + GB_TILE - 1) / GB_TILE;
  uint64_t* tile_counts = group_tile_counts(status, n);
  prof_begin(s, "k_group_flags", (double)n * 8.0 + (double)(n / 32) * 8.0);
  if (gshift >= 32)
    k_group_flags<uint32_t><<<(unsigned)tiles, GB_THREADS, 0, s>>>(keys, n, n_dev, gshift, flags,
                                                                   tile_counts);
  else
    k_group_flags<uint64_t><<<(unsigned)tiles, GB_THREADS, 0, s>>>(keys, n, n_dev, gshift, flags,
                                                                   tile_counts);
  prof_end(s);
}

void launch_group_finish(const uint64_t* flags, int64_t n, const uint64_t* n_dev, uint32_t* S,
                         uint32_t* E, uint64_t cap, uint64_t* status, uint32_t* err,
                         uint64_t* n_groups, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t tiles = (n + GB_TILE - 1) / GB_TILE;
  const size_t st = scan_status_bytes(tiles);
  uint64_t* tile_counts = group_tile_counts(status, n);
  uint64_t* tile_prefix = tile_counts + tiles;
  uint32_t* ctr = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(status) + st - 16);
  cudaMemsetAsync(status, 0, st, s);
  prof_begin(s, "k_scan_tiles", (double)tiles * 16.0);
  k_scan_counts<<<std::min<uint32_t>(div_up_u32(tiles, SCAN_TILE), 152 * 16), SCAN_THREADS, 0,
                  s>>>(CountsU64{tile_counts}, tiles, nullptr, tile_prefix, status, ctr, err);
  prof_end(s);
  prof_begin(s, "k_group_write", (double)(n / 32) * 8.0);
  k_group_write<<<(unsigned)tiles, GB_THREADS, 0, s>>>(flags, n, n_dev, tile_prefix, S, E, cap,
                                                       err);
  prof_end(s);
  // number of groups = heads in the total (high field of tile_prefix[tiles])
  k_groups_total<<<1, 1, 0, s>>>(tile_prefix + tiles, n_groups);
}

void launch_group_bounds(const uint64_t* keys, int64_t n, const uint64_t* n_dev, int gshift,
                         uint32_t* S, uint32_t* E, uint64_t cap, uint64_t* flags,
                         uint64_t* status, uint32_t* err, uint64_t* n_groups, cudaStream_t s) {
  launch_group_flags(keys, n, n_dev, gshift, flags, status, s);
  launch_group_finish(flags, n, n_dev, S, E, cap, status, err, n_groups, s);
}


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
                 const uint64_t* __restrict__ pair_off, int64_t n_groups_cap,
                 const uint64_t* __restrict__ n_groups_dev, uint64_t pair_cap, uint32_t id_bits,
                 uint64_t* __restrict__ out, const uint64_t* __restrict__ out_base,
                 uint64_t* __restrict__ n_pairs_out, uint32_t* __restrict__ err) {
  __shared__ uint64_t s_off[EMIT_TILE + 1];
  __shared__ int64_t s_k0, s_k1;
  // group count and pair count may only be known on the device
  const int64_t n_groups = n_groups_dev ? min((int64_t)*n_groups_dev, n_groups_cap) : n_groups_cap;
  const uint64_t n_all = pair_off[n_groups];
  // words already in `out` (written by the bucket pass): ours follow them
  const uint64_t base = out_base ? *out_base : 0ull;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n_pairs_out) *n_pairs_out = base + n_all;
    if (base + n_all > pair_cap) atomicOr(err, DERR_CAPACITY);
  }
  const uint64_t room = base < pair_cap ? pair_cap - base : 0ull;
  const uint64_t n_pairs = n_all < room ? n_all : room;
  out += base;
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
          // members of a group need not be in id order: the word is (min, max)
          const uint64_t ia = keys[s0 + a] & idmask, ib = keys[s0 + b] & idmask;
          w = ((ia < ib ? ia : ib) << id_bits) | (ia < ib ? ib : ia);
        } else {
          atomicOr(err, DERR_RANGE);
        }
        out[t] = w;
      }
    }
    __syncthreads();
  }
}

void launch_emit_pairs(const uint64_t* keys, uint64_t n_keys, const uint32_t* S,
                       const uint64_t* pair_off, int64_t n_groups, const uint64_t* n_groups_dev,
                       uint64_t pair_cap, uint32_t id_bits, uint64_t* out,
                       const uint64_t* out_base, uint64_t* n_pairs_out, int sms, uint32_t* err,
                       cudaStream_t s) {
  if (pair_cap == 0 || n_groups <= 0) return;
  const uint64_t tiles = (pair_cap + EMIT_TILE - 1) / EMIT_TILE;
  const int blocks = (int)std::min<uint64_t>(tiles, (uint64_t)sms * 8);
  prof_begin(s, "k_emit_pairs", (double)pair_cap * (8.0 + 16.0));
  k_emit_pairs<<<blocks, EMIT_THREADS, 0, s>>>(keys, n_keys, S, pair_off, n_groups, n_groups_dev,
                                               pair_cap, id_bits, out, out_base, n_pairs_out,
                                               err);
  prof_end(s);
}

}  // namespace xtn
