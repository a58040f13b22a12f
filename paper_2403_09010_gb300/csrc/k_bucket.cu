// Shared-memory finish of the grouping step, with the group flags (Appendix
// A, XTNeighbor step 4: `sort` + `uniqueCount`).
//
// The global radix passes order the variant records by the top G bits of
// their group key only; the records of one such value (a "bucket") are then
// contiguous, and the last pass leaves the first position of every bucket
// (radix_sort_passes, bucket_start).  Each block of k_bucket takes K
// consecutive buckets -- one to two thousand records for the 1M workload --
// and, in shared memory, brings the records of every group (equal group key)
// together:
//   HASH  (self-search): a hash table keyed by the composite key
//         (bucket - first bucket of the block) << L | low L group-key bits
//         numbers the groups; a counting scatter by table slot makes them
//         contiguous.  Order inside a group and between groups is arbitrary:
//         the pair emitter orders each pair itself.
//   !HASH (reference index): stable LSD passes of 9-bit digits over the same
//         composite key, i.e. exactly the array further global passes give.
// Either way one read and one write of the records replace the remaining
// global passes.  From the grouped block the kernel also writes the
// head/tail flag words and per-tile head/tail counts that k_group_write
// consumes, which replaces a separate flag pass over the records.
//
// A bucket with more records than a block holds (many copies of one
// sequence) is sorted by the one block that owns it, in global memory: per
// digit pass a histogram over the bucket, then stable ranking chunk by chunk,
// alternating between the input buffer (scratch within the bucket's own
// range) and the output.
#include <algorithm>
#include <mutex>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

namespace {

constexpr int BK_THREADS = 256;
constexpr int BK_WARPS = BK_THREADS / 32;
constexpr int SORT_ITEMS = 16;  // !HASH: 4096 records per segment, 2 blocks/SM
constexpr int HASH_ITEMS = 8;   // HASH: 2048 records per segment, 5 blocks/SM

// Radix digits of the shared-memory passes: 9 bits for the sorting variant
// (two passes cover 17 bits); 8 for the hashing one, whose ranking only runs
// on oversized buckets and whose smaller tables leave room for a fifth block.
template <bool HASH>
struct Bk {
  static constexpr int ITEMS = HASH ? HASH_ITEMS : SORT_ITEMS;
  static constexpr int CAP = BK_THREADS * ITEMS;
  static constexpr int MIN_BLOCKS = HASH ? 5 : 2;
  static constexpr int BITS = HASH ? 8 : 9;
  static constexpr int BINS = 1 << BITS;
  static constexpr int HB = HASH ? 12 : 0;  // log2 of the hash slots (2 per record)
  static constexpr int H = 1 << HB;
  static constexpr size_t keys = (size_t)CAP * 8;
  static constexpr size_t rank_tables = (size_t)2 * BK_WARPS * BINS * 4;  // wh + mb
  static constexpr size_t hash_tables = HASH ? (size_t)H * 4 + (size_t)H * 2 : 0;
  static constexpr size_t region = rank_tables > hash_tables ? rank_tables : hash_tables;
  static constexpr size_t base = (size_t)BINS * 4;
  static constexpr size_t bytes = keys + region + base;
};
static_assert(Bk<true>::H >= 2 * Bk<true>::CAP, "hash load factor <= 1/2");

constexpr unsigned long long NO_START = ~0ull;
constexpr uint32_t EMPTY_SLOT = 0xffffffffu;
constexpr uint64_t NO_GROUP = ~0ull;  // above every group key (at most 40 bits)

// First recorded bucket start at index >= b (bucket starts increase with the
// bucket index), or n when no later bucket holds records.  Whole warp.
__device__ int64_t first_start(const unsigned long long* __restrict__ bs, int64_t b, int64_t nb,
                               int64_t n, uint32_t lane) {
  for (int64_t base = b; base < nb; base += 32) {
    const int64_t idx = base + lane;
    const unsigned long long v = idx < nb ? bs[idx] : NO_START;
    const uint32_t m = __ballot_sync(FULL_MASK, v != NO_START);
    if (m) {
      const unsigned long long f = __shfl_sync(FULL_MASK, v, __ffs(m) - 1);
      return (int64_t)f < n ? (int64_t)f : n;
    }
  }
  return n;
}

// Block-wide exclusive scan of one u32 per thread.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_wsum) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL_MASK, inc, o);
    if (lane >= (uint32_t)o) inc += t;
  }
  if (lane == 31) s_wsum[warp] = inc;
  __syncthreads();
  uint32_t off = 0;
#pragma unroll
  for (int w = 0; w < BK_WARPS; ++w)
    if (w < (int)warp) off += s_wsum[w];
  __syncthreads();  // s_wsum is reused by the next scan
  return off + inc - v;
}

// One stable ranking pass over the block's items (item i of lane l of warp w
// is position w*32*ITEMS + i*32 + l; positions >= m are absent).  On return
// s_wh[w*BINS + d] holds the position at which warp w's first record of
// digit d goes: the digit's start within the block (scan of the block's
// digit counts) or, when `running` is set, s_base[d] -- which then advances
// by the block's count of d.  The peer bins s_mb must be zero on entry
// (clear_mb) and are zero again on return.
template <int ITEMS, int BINS, class DigitF>
__device__ __forceinline__ void rank_pass(const uint64_t (&key)[ITEMS], uint16_t (&rank)[ITEMS],
                                          int m, DigitF digit, uint32_t* s_wh, uint32_t* s_mb,
                                          uint32_t* s_base, bool running, bool clear_mb,
                                          uint32_t* s_wsum) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int k = threadIdx.x; k < BK_WARPS * BINS; k += BK_THREADS) {
    s_wh[k] = 0;
    if (clear_mb) s_mb[k] = 0;
  }
  __syncthreads();
  uint32_t* wh = s_wh + warp * BINS;
  uint32_t* mb = s_mb + warp * BINS;
  const int wbase = (int)warp * 32 * ITEMS;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const bool valid = wbase + i * 32 + (int)lane < m;
    const uint32_t dig = valid ? digit(key[i]) : 0u;
    if (valid) atomicOr(&mb[dig], 1u << lane);
    __syncwarp();
    const uint32_t peers = valid ? mb[dig] : 0u;
    __syncwarp();
    const uint32_t before = peers & lt_mask;
    uint32_t old = 0;
    if (valid && before == 0) {
      old = wh[dig];
      wh[dig] = old + __popc(peers);
      mb[dig] = 0u;
    }
    old = __shfl_sync(FULL_MASK, old, valid ? __ffs(peers) - 1 : (int)lane);
    rank[i] = (uint16_t)(old + __popc(before));
    __syncwarp();
  }
  __syncthreads();
  // thread t owns digits DPT*t .. DPT*t + DPT - 1: per-warp exclusive
  // offsets, then the digits' starts
  constexpr int DPT = BINS / BK_THREADS;
  static_assert(DPT >= 1 && BINS % BK_THREADS == 0, "whole digits per thread");
  const int d0 = DPT * threadIdx.x;
  uint32_t r[DPT];
#pragma unroll
  for (int k = 0; k < DPT; ++k) r[k] = 0;
#pragma unroll
  for (int w = 0; w < BK_WARPS; ++w) {
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      const uint32_t c = s_wh[w * BINS + d0 + k];
      s_wh[w * BINS + d0 + k] = r[k];
      r[k] += c;
    }
  }
  uint32_t st[DPT];
  if (running) {
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      st[k] = s_base[d0 + k];
      s_base[d0 + k] = st[k] + r[k];
    }
  } else {
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < DPT; ++k) tot += r[k];
    uint32_t x = block_excl_scan(tot, s_wsum);
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      st[k] = x;
      x += r[k];
    }
  }
#pragma unroll
  for (int w = 0; w < BK_WARPS; ++w)
#pragma unroll
    for (int k = 0; k < DPT; ++k) s_wh[w * BINS + d0 + k] += st[k];
  __syncthreads();
}

// Packed head/tail counts, the layout k_group_write expects.
__device__ __forceinline__ uint64_t pack_ht(uint32_t h, uint32_t t) {
  return ((uint64_t)h << 31) | t;
}

// Flag words (head ballot | tail ballot << 32) of the grouped records
// [p, p + m), whose group keys `gkey(j)` (j relative to p) differ from
// everything outside the range.  Words wholly inside the range are stored,
// the edge words (shared with the neighbouring ranges) are OR-ed into the
// zeroed array.  Head/tail counts of flag tiles t0 and t0 + 1 accumulate in
// acc0 / acc1 (packed, lane 0 of each warp), other tiles' go straight to
// tile_counts.
template <class GKey>
__device__ __forceinline__ void write_flags(int64_t p, int64_t m, GKey gkey, uint64_t* flags,
                                            uint64_t* tile_counts, int64_t t0, uint64_t& acc0,
                                            uint64_t& acc1) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const int64_t gw0 = p >> 5, gw1 = (p + m - 1) >> 5;
  for (int64_t gw = gw0 + warp; gw <= gw1; gw += BK_WARPS) {
    const int64_t j = gw * 32 + lane - p;
    const bool valid = j >= 0 && j < m;
    const uint64_t g = valid ? gkey(j) : NO_GROUP;
    uint64_t gp = __shfl_up_sync(FULL_MASK, g, 1);
    uint64_t gn = __shfl_down_sync(FULL_MASK, g, 1);
    if (lane == 0) gp = (j - 1 >= 0 && j - 1 < m) ? gkey(j - 1) : NO_GROUP;
    if (lane == 31) gn = (j + 1 >= 0 && j + 1 < m) ? gkey(j + 1) : NO_GROUP;
    const uint32_t hb = __ballot_sync(FULL_MASK, valid && g != gp && g == gn);
    const uint32_t tb = __ballot_sync(FULL_MASK, valid && g == gp && g != gn);
    if (lane == 0) {
      const uint64_t word = ((uint64_t)tb << 32) | hb;
      const bool whole = gw * 32 >= p && gw * 32 + 32 <= p + m;
      if (whole) flags[gw] = word;
      else if (word) atomicOr(reinterpret_cast<unsigned long long*>(&flags[gw]),
                              (unsigned long long)word);
      if (word) {
        const uint64_t c = pack_ht(__popc(hb), __popc(tb));
        const int64_t t = gw * 32 / GROUP_FLAG_TILE;
        if (t == t0) acc0 += c;
        else if (t == t0 + 1) acc1 += c;
        else atomicAdd(reinterpret_cast<unsigned long long*>(&tile_counts[t]), (unsigned long long)c);
      }
    }
  }
}

// One block of buckets (number blk) of k_bucket.
template <bool HASH>
__device__ __forceinline__ void bucket_block(
    uint64_t blk, uint64_t* __restrict__ A, uint64_t* __restrict__ Y, int64_t n_cap,
    const uint64_t* __restrict__ n_dev, const unsigned long long* __restrict__ bucket_start, int G,
    int kbits, int lo, int L, int cap, uint64_t* __restrict__ flags,
    uint64_t* __restrict__ tile_counts, uint64_t* __restrict__ cand, uint64_t cand_cap,
    unsigned long long* __restrict__ cand_count, int id_bits, uint32_t* __restrict__ err) {
  using C = Bk<HASH>;
  constexpr int ITEMS = C::ITEMS;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_k = reinterpret_cast<uint64_t*>(smem);
  uint32_t* s_wh = reinterpret_cast<uint32_t*>(smem + C::keys);  // rank tables or hash tables
  uint32_t* s_mb = s_wh + BK_WARPS * C::BINS;
  uint32_t* s_base = reinterpret_cast<uint32_t*>(smem + C::keys + C::region);
  __shared__ uint32_t s_wsum[BK_WARPS];
  __shared__ int64_t s_range[2];
  __shared__ unsigned long long s_acc[2];

  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  const int64_t nb = 1ll << G;
  const int64_t K = 1ll << kbits;
  const int64_t b0 = (int64_t)blk * K;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const int wbase = (int)warp * 32 * ITEMS;

  // [s, e) of buckets [bf, bl)
  auto bucket_range = [&](int64_t bf, int64_t bl) {
    if (warp == 0) {
      int64_t s = 0, e = n;
      if (G > 0) {
        s = first_start(bucket_start, bf, nb, n, lane);
        e = bl >= nb ? n : first_start(bucket_start, bl, nb, n, lane);
      }
      if (lane == 0) {
        s_range[0] = s;
        s_range[1] = e < s ? s : e;
      }
    }
    __syncthreads();
  };
  // empty hash table (composite keys all ones, counts zero), 16 bytes a store
  auto clear_hash = [&]() {
    uint4* t4 = reinterpret_cast<uint4*>(s_wh);
    constexpr int KEY4 = C::H / 4, ALL4 = (C::H + C::H / 2) / 4;
    for (int k = threadIdx.x; k < ALL4; k += BK_THREADS)
      t4[k] = k < KEY4 ? make_uint4(EMPTY_SLOT, EMPTY_SLOT, EMPTY_SLOT, EMPTY_SLOT)
                       : make_uint4(0u, 0u, 0u, 0u);
  };
  if (threadIdx.x == 0) s_acc[0] = s_acc[1] = 0;
  if constexpr (HASH) {
    // warp 0 finds the block's first record, warp 1 its end, the rest clear
    if (warp < 2) {
      int64_t v = warp == 0 ? 0 : n;
      if (G > 0) {
        const int64_t bf = warp == 0 ? b0 : b0 + K;
        v = bf >= nb ? n : first_start(bucket_start, bf, nb, n, lane);
      }
      if (lane == 0) s_range[warp] = v;
    } else {
      for (int k = threadIdx.x - 64; k < (C::H + C::H / 2) / 4; k += BK_THREADS - 64)
        reinterpret_cast<uint4*>(s_wh)[k] =
            k < C::H / 4 ? make_uint4(EMPTY_SLOT, EMPTY_SLOT, EMPTY_SLOT, EMPTY_SLOT)
                         : make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
  } else {
    bucket_range(b0, b0 + K);
  }
  const int64_t s = s_range[0], e = s_range[1] < s_range[0] ? s_range[0] : s_range[1];
  __syncthreads();
  if (s >= n || s >= e) return;
  uint64_t acc0 = 0, acc1 = 0;  // head/tail counts of this block's first two flag tiles
  const int64_t tile_first = s / GROUP_FLAG_TILE;
  auto gkey_of = [lo](uint64_t k) { return k >> lo; };

  auto finish = [&](int64_t p, int m) {
    for (int j = threadIdx.x; j < m; j += BK_THREADS) Y[p + j] = s_k[j];
    if (flags)
      write_flags(p, m, [&](int64_t j) { return gkey_of(s_k[j]); }, flags, tile_counts, tile_first,
                  acc0, acc1);
    __syncthreads();  // s_k and the tables are reused by the next segment
  };

  // ---- candidate pairs of a grouped segment, straight from shared memory ----
  // The ids of every group of two or more records lie contiguously in s_k
  // (as u32), the group of slot h from start(h) (packed u16 in tc) with
  // size tk[h].  Every pair of such a group becomes a candidate word
  // (min id << id_bits | max id), appended to `cand` from `off` on (room
  // reserved per warp during the slot scan).  gmask marks this thread's slots
  // with such groups (bit k = slot threadIdx.x * H / THREADS + k); the warp
  // takes the marked slots one at a time and spreads each group's pairs over
  // its lanes.  No block-wide step.
  auto emit_segment = [&](const uint32_t* tc, const uint32_t* tk, uint32_t gmask, uint64_t off) {
    constexpr uint32_t PER = C::H / BK_THREADS;
    const uint32_t* s_ids = reinterpret_cast<const uint32_t*>(s_k);
    while (__any_sync(FULL_MASK, gmask != 0)) {
      uint32_t st = 0, c = 0;
      if (gmask) {
        const uint32_t h = threadIdx.x * PER + (uint32_t)(__ffs(gmask) - 1);
        gmask &= gmask - 1;
        st = (tc[h >> 1] >> ((h & 1) * 16)) & 0xffffu;
        c = tk[h];
      }
      uint32_t groups = __ballot_sync(FULL_MASK, c >= 2);
      while (groups) {
        const int src = __ffs(groups) - 1;
        groups &= groups - 1;
        const uint32_t gst = __shfl_sync(FULL_MASK, st, src);
        const uint32_t gc = __shfl_sync(FULL_MASK, c, src);
        const uint32_t pairs = gc * (gc - 1) / 2;
        for (uint32_t l = lane; l < pairs; l += 32) {
          // colex unranking: l = b (b - 1) / 2 + a, a < b
          uint32_t b = (uint32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)l)) * 0.5f);
          while (b * (b - 1) / 2 > l) --b;
          while ((b + 1) * b / 2 <= l) ++b;
          const uint32_t a = l - b * (b - 1) / 2;
          const uint64_t ia = s_ids[gst + a], ib = s_ids[gst + b];
          if (off + l < cand_cap)
            cand[off + l] = ((ia < ib ? ia : ib) << id_bits) | (ia < ib ? ib : ia);
        }
        off += pairs;
      }
    }
    __syncthreads();  // s_k and the tables are reused by the next segment
  };

  // ---- one segment [p, q) of at most `cap` records, buckets from bA ----
  // composite key: (key >> lo) - (bA << L) = (bucket - bA) << L | low L bits
  auto segment = [&](int64_t p, int64_t q, uint64_t bA, int kb, bool cleared) {
    const int m = (int)(q - p);
    const uint64_t cbase = bA << L;
    auto comp = [&](uint64_t k) { return (uint32_t)((k >> lo) - cbase); };
    uint64_t key[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int pos = wbase + i * 32 + (int)lane;
      key[i] = pos < m ? __ldcs(A + p + pos) : 0ull;
    }
    if constexpr (HASH) {
      uint32_t* tk = s_wh;                                   // H composite keys
      uint32_t* tc = tk + C::H;                              // H u16 counts, two per word
      if (!cleared) {
        clear_hash();
        __syncthreads();
      }
      uint32_t sr[ITEMS];  // slot << 16 | rank within the slot's group
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        sr[i] = 0;
        if (wbase + i * 32 + (int)lane < m) {
          const uint32_t c = comp(key[i]);
          uint32_t h = (c * 0x9E3779B1u) >> (32 - C::HB);
          bool found = false;
          for (int probe = 0; probe < C::H; ++probe) {  // at most m <= H/2 keys: always ends
            const uint32_t old = atomicCAS(&tk[h], EMPTY_SLOT, c);
            if (old == EMPTY_SLOT || old == c) {
              found = true;
              break;
            }
            h = (h + 1) & (C::H - 1);
          }
          if (found) {
            const uint32_t sh = (h & 1) * 16;
            const uint32_t r = (atomicAdd(&tc[h >> 1], 1u << sh) >> sh) & 0xffffu;
            sr[i] = (h << 16) | r;
          } else {
            atomicOr(err, DERR_RANGE);
            sr[i] = 0xffffffffu;
          }
        }
      }
      __syncthreads();
      // slot starts: exclusive scan of the counts in slot order (thread t owns
      // H / THREADS consecutive slots), written back over the counts
      constexpr int PER = C::H / BK_THREADS;
      static_assert(PER % 2 == 0, "whole count words per thread");
      // With `cand` only the groups of two or more records are placed (as
      // 4-byte ids): single records pair with nothing, so they get start
      // NO_PLACE and leave no trace; such a slot's size goes to the key table
      // (free now) for the emitter.
      constexpr uint32_t NO_PLACE = 0xffffu;
      uint32_t w[PER / 2];
      uint32_t tot = 0;
#pragma unroll
      for (int k = 0; k < PER / 2; ++k) {
        w[k] = tc[threadIdx.x * (PER / 2) + k];
        const uint32_t a = w[k] & 0xffffu, b = w[k] >> 16;
        tot += cand ? (a >= 2 ? a : 0u) + (b >= 2 ? b : 0u) : a + b;
      }
      uint32_t run = block_excl_scan(tot, s_wsum);
      // with `cand`: slots of this thread holding groups of two or more (bit
      // k = slot threadIdx.x * PER + k) and their pairs
      uint32_t gmask = 0, np = 0;
#pragma unroll
      for (int k = 0; k < PER / 2; ++k) {
        const uint32_t a = w[k] & 0xffffu, b = w[k] >> 16;
        if (cand) {
          const uint32_t h = threadIdx.x * PER + 2 * k;
          const uint32_t sa = a >= 2 ? run : NO_PLACE;
          run += a >= 2 ? a : 0u;
          const uint32_t sb = b >= 2 ? run : NO_PLACE;
          run += b >= 2 ? b : 0u;
          tc[threadIdx.x * (PER / 2) + k] = sa | (sb << 16);
          if (a >= 2) tk[h] = a;
          if (b >= 2) tk[h + 1] = b;
        } else {
          tc[threadIdx.x * (PER / 2) + k] = run | ((run + a) << 16);
          run += a + b;
        }
        if (a >= 2) {
          gmask |= 1u << (2 * k);
          np += a * (a - 1) / 2;
        }
        if (b >= 2) {
          gmask |= 2u << (2 * k);
          np += b * (b - 1) / 2;
        }
      }
      uint64_t cbase = 0;  // where this thread's warp writes its candidates
      if (cand) {
        uint32_t wp = np;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wp += __shfl_xor_sync(FULL_MASK, wp, o);
        unsigned long long b = 0;
        if (lane == 0 && wp) {
          b = atomicAdd(cand_count, (unsigned long long)wp);
          if (b + wp > cand_cap) atomicOr(err, DERR_CAPACITY);
        }
        cbase = __shfl_sync(FULL_MASK, b, 0);
      }
      __syncthreads();
      if (cand) {
        uint32_t* s_ids = reinterpret_cast<uint32_t*>(s_k);
        const uint64_t idmask = (1ull << id_bits) - 1ull;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          if (wbase + i * 32 + (int)lane < m && sr[i] != 0xffffffffu) {
            const uint32_t h = sr[i] >> 16;
            const uint32_t start = (tc[h >> 1] >> ((h & 1) * 16)) & 0xffffu;
            if (start != NO_PLACE) {
              const uint32_t pos = start + (sr[i] & 0xffffu);
              if (pos < (uint32_t)m) s_ids[pos] = (uint32_t)(key[i] & idmask);
              else atomicOr(err, DERR_RANGE);
            }
          }
        }
        __syncthreads();
        emit_segment(tc, tk, gmask, cbase);
        return;
      }
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        if (wbase + i * 32 + (int)lane < m && sr[i] != 0xffffffffu) {
          const uint32_t h = sr[i] >> 16;
          const uint32_t start = (tc[h >> 1] >> ((h & 1) * 16)) & 0xffffu;
          const uint32_t pos = start + (sr[i] & 0xffffu);
          if (pos < (uint32_t)m) s_k[pos] = key[i];
          else atomicOr(err, DERR_RANGE);
        }
      }
      __syncthreads();
    } else {
      const int passes = (L + kb + C::BITS - 1) / C::BITS;
      uint16_t rank[ITEMS];
      for (int pass = 0; pass < passes; ++pass) {
        const int sh = C::BITS * pass;
        auto digit = [&](uint64_t k) { return (comp(k) >> sh) & (C::BINS - 1); };
        rank_pass<ITEMS, C::BINS>(key, rank, m, digit, s_wh, s_mb, s_base, false, pass == 0,
                                  s_wsum);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          if (wbase + i * 32 + (int)lane < m) {
            const uint32_t pos = s_wh[warp * C::BINS + digit(key[i])] + rank[i];
            if (pos < (uint32_t)m) s_k[pos] = key[i];
            else atomicOr(err, DERR_RANGE);
          }
        }
        __syncthreads();
        if (pass + 1 < passes) {
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
            const int pos = wbase + i * 32 + (int)lane;
            key[i] = pos < m ? s_k[pos] : 0ull;
          }
          __syncthreads();  // every read done before the next pass scatters
        }
      }
    }
    finish(p, m);
  };

  // ---- one bucket [p, q) larger than `cap`, sorted in global memory ----
  auto large = [&](int64_t p, int64_t q) {
    if (cand && threadIdx.x == 0) atomicAdd(cand_count + 1, (unsigned long long)(q - p));
    const uint64_t lmask = (1ull << L) - 1ull;  // one bucket: the low L bits decide
    const int passes = (L + C::BITS - 1) / C::BITS;
    uint64_t* src = A;
    uint64_t* dst = Y;
    uint64_t key[ITEMS];
    uint16_t rank[ITEMS];
    for (int pass = 0; pass < passes; ++pass) {
      const int sh = C::BITS * pass;
      auto digit = [&](uint64_t k) {
        return (uint32_t)((((k >> lo) & lmask) >> sh) & (C::BINS - 1));
      };
      for (int k = threadIdx.x; k < C::BINS; k += BK_THREADS) s_base[k] = 0;
      __syncthreads();
      for (int64_t c = p; c < q; c += cap) {
        const int cm = (int)min((int64_t)cap, q - c);
        for (int j = threadIdx.x; j < cm; j += BK_THREADS) atomicAdd(&s_base[digit(src[c + j])], 1u);
      }
      __syncthreads();
      {
        constexpr int DPT = C::BINS / BK_THREADS;
        uint32_t c[DPT], tot = 0;
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
          c[k] = s_base[DPT * threadIdx.x + k];
          tot += c[k];
        }
        uint32_t x = block_excl_scan(tot, s_wsum);
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
          s_base[DPT * threadIdx.x + k] = x;
          x += c[k];
        }
        __syncthreads();
      }
      bool first = true;
      for (int64_t c = p; c < q; c += cap) {
        const int cm = (int)min((int64_t)cap, q - c);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          const int pos = wbase + i * 32 + (int)lane;
          key[i] = pos < cm ? src[c + pos] : 0ull;
        }
        rank_pass<ITEMS, C::BINS>(key, rank, cm, digit, s_wh, s_mb, s_base, true, first, s_wsum);
        first = false;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          if (wbase + i * 32 + (int)lane < cm) {
            const uint64_t pos = (uint64_t)s_wh[warp * C::BINS + digit(key[i])] + rank[i];
            if (pos < (uint64_t)(q - p)) dst[p + pos] = key[i];
            else atomicOr(err, DERR_RANGE);
          }
        }
        __syncthreads();
      }
      uint64_t* t = src;
      src = dst;
      dst = t;
    }
    if (src != Y) {
      for (int64_t j = p + threadIdx.x; j < q; j += BK_THREADS) Y[j] = src[j];
      __syncthreads();
    }
    if (flags)
      write_flags(p, q - p, [&](int64_t j) { return gkey_of(Y[p + j]); }, flags, tile_counts,
                  tile_first, acc0, acc1);
    __syncthreads();
  };

  if (e - s <= cap) {
    segment(s, e, (uint64_t)b0, kbits, HASH);
  } else {
    // too many records for one segment: bucket by bucket
    for (int64_t b = b0; b < b0 + K && b < nb; ++b) {
      bucket_range(b, b + 1);
      const int64_t p = s_range[0], q = s_range[1];
      __syncthreads();
      if (p >= q) continue;
      if (q - p <= cap) segment(p, q, (uint64_t)b, 0, false);
      else large(p, q);
    }
  }

  // head/tail counts of the first two flag tiles this block touched
  if (flags && lane == 0 && (acc0 | acc1)) {
    if (acc0) atomicAdd(&s_acc[0], (unsigned long long)acc0);
    if (acc1) atomicAdd(&s_acc[1], (unsigned long long)acc1);
  }
  __syncthreads();
  if (flags && threadIdx.x == 0) {
    if (s_acc[0])
      atomicAdd(reinterpret_cast<unsigned long long*>(&tile_counts[tile_first]), s_acc[0]);
    if (s_acc[1])
      atomicAdd(reinterpret_cast<unsigned long long*>(&tile_counts[tile_first + 1]), s_acc[1]);
  }
}

// Every block of buckets, or with seg_list only the *seg_count blocks listed
// there (the ones the singleton filter left), in a grid-stride loop.
template <bool HASH>
__global__ void __launch_bounds__(BK_THREADS, Bk<HASH>::MIN_BLOCKS)
    k_bucket(uint64_t* __restrict__ A, uint64_t* __restrict__ Y, int64_t n_cap,
             const uint64_t* __restrict__ n_dev,
             const unsigned long long* __restrict__ bucket_start, int G, int kbits, int lo, int L,
             int cap, uint64_t* __restrict__ flags, uint64_t* __restrict__ tile_counts,
             uint64_t* __restrict__ cand, uint64_t cand_cap,
             unsigned long long* __restrict__ cand_count, int id_bits,
             const uint32_t* __restrict__ seg_list, const uint32_t* __restrict__ seg_count,
             uint32_t* __restrict__ err) {
  if (!seg_list) {
    bucket_block<HASH>(blockIdx.x, A, Y, n_cap, n_dev, bucket_start, G, kbits, lo, L, cap, flags,
                       tile_counts, cand, cand_cap, cand_count, id_bits, err);
    return;
  }
  const uint32_t count = *seg_count;
  const uint64_t n_blocks = ((uint64_t)1 << G) >> kbits;
  for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const uint32_t blk = seg_list[i];
    if (blk < n_blocks)
      bucket_block<HASH>(blk, A, Y, n_cap, n_dev, bucket_start, G, kbits, lo, L, cap, flags,
                         tile_counts, cand, cand_cap, cand_count, id_bits, err);
    else if (threadIdx.x == 0)
      atomicOr(err, DERR_RANGE);
    __syncthreads();  // shared memory is reused by the next listed block
  }
}

}  // namespace

int bucket_capacity(bool hash) { return hash ? Bk<true>::CAP : Bk<false>::CAP; }

GroupingShape choose_grouping(uint64_t n_rec, int hs, bool hash) {
  GroupingShape g;
  // global bits: until the average bucket holds at most ~2k records, with at
  // least 8 and at most 24 bits left to the shared-memory step
  int G = 0;
  while (G + 8 <= hs - 8 && (n_rec >> G) > 2048) G += 8;
  while (hs - G > 24) G += 8;
  g.G = G;
  g.L = hs - G;
  // buckets per block: a power of two, on average at most ~80% of a segment;
  // the composite key keeps to 31 bits
  const uint64_t avg = std::max<uint64_t>(1, n_rec >> G);
  const uint64_t fill = (uint64_t)bucket_capacity(hash) * 4 / 5;
  int kb = 0;
  while (kb < G && g.L + kb + 1 <= 31 && (avg << (kb + 1)) <= fill) ++kb;
  g.kbits = kb;
  return g;
}

void launch_bucket(bool hash, uint64_t* A, uint64_t* Y, int64_t n, const uint64_t* n_dev,
                   const uint64_t* bucket_start, const GroupingShape& g, int lo, int cap,
                   uint64_t* flags, uint64_t* tile_counts, uint64_t* cand, uint64_t cand_cap,
                   uint64_t* cand_count, int id_bits, uint32_t* err, cudaStream_t s,
                   const uint32_t* seg_list, const uint32_t* seg_count, int sms) {
  if (n <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_bucket<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Bk<true>::bytes);
    cudaFuncSetAttribute(k_bucket<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_bucket<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Bk<false>::bytes);
    cudaFuncSetAttribute(k_bucket<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
  const int full = bucket_capacity(hash);
  if (cap <= 0 || cap > full) cap = full;
  // a listed subset runs in a grid-stride loop over the list
  const uint64_t blocks = seg_list ? (uint64_t)std::max(1, sms) * Bk<true>::MIN_BLOCKS
                                   : ((uint64_t)1 << g.G) >> g.kbits;
  // algorithmic bytes: every record read once; written back unless the
  // candidates leave straight from shared memory (their words are not counted:
  // their number is unknown at launch and small next to the records)
  const double bytes = (hash && cand) ? (double)n * 8.0
                                      : (double)n * 16.0 + (flags ? (double)n / 4.0 : 0.0);
  const unsigned long long* bs = reinterpret_cast<const unsigned long long*>(bucket_start);
  if (hash) {
    prof_begin(s, seg_list ? "k_bucket_group_listed" : "k_bucket_group", seg_list ? 0.0 : bytes);
    k_bucket<true><<<(unsigned)blocks, BK_THREADS, Bk<true>::bytes, s>>>(
        A, Y, n, n_dev, bs, g.G, g.kbits, lo, g.L, cap, flags, tile_counts, cand, cand_cap,
        reinterpret_cast<unsigned long long*>(cand_count), id_bits, seg_list, seg_count, err);
  } else {
    prof_begin(s, "k_bucket_sort", bytes);
    k_bucket<false><<<(unsigned)blocks, BK_THREADS, Bk<false>::bytes, s>>>(
        A, Y, n, n_dev, bs, g.G, g.kbits, lo, g.L, cap, flags, tile_counts, nullptr, 0, nullptr,
        0, nullptr, nullptr, err);
  }
  prof_end(s);
}

}  // namespace xtn
