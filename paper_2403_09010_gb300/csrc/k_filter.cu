// Grouping of variant records by their full group key, with the candidate
// pairs written at once (Appendix A, XTNeighbor steps 4-5), for the buckets
// left by the global radix passes on the top G key bits.
//
// Nearly every variant record shares its group key with no other record
// (about 91% of the 1M workload's records are alone), so the exact grouping
// only needs the few that do.  Each block of k_bucket_filter takes a segment
// of 2^kf consecutive buckets (contiguous in the sorted records) and
//   1. marks, in two bitmaps, the keys seen (indexed by the composite key:
//      bucket offset in the segment above the low L key bits, hashed when
//      wider than the bitmap's index) and the keys seen again (a 16-bit
//      hash of it);
//   2. keeps the records whose key was seen again -- all members of groups
//      of two or more, plus the rare lone record whose bit another key also
//      hit -- in a short list;
//   3. groups the list exactly in a hash table sized to it (at least twice
//      the kept records), places each group's ids contiguously, and writes
//      every pair of a group of two or more as a candidate word (min id <<
//      id_bits | max id), reserving output space once per block.
// Every phase spreads its work over all the block's threads, and the fixed
// work per block (table clearing and scanning) scales with the kept records,
// not with the segment.  A segment whose list overflows appends the k_bucket
// blocks it covers to a list instead; k_bucket then groups the listed blocks
// as before.
#include <algorithm>
#include <mutex>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

namespace {

constexpr int BF_THREADS = 256;
constexpr int BF_WARPS = BF_THREADS / 32;

constexpr int BF_BITS = 16;                        // log2 of the bits of each filter bitmap
constexpr int BF_WORDS = (1 << BF_BITS) / 32;
constexpr uint32_t BF_EMPTY = 0xffffffffu;
constexpr uint32_t BF_NO_PLACE = 0xffffu;
constexpr uint32_t BF_SMALL = 8;                   // groups up to this size: one lane each

constexpr unsigned long long BF_NO_START = ~0ull;

// First recorded bucket start at index >= b, or n (whole warp).
__device__ __forceinline__ int64_t bf_first_start(const unsigned long long* __restrict__ bs,
                                                  int64_t b, int64_t nb, int64_t n,
                                                  uint32_t lane) {
  for (int64_t base = b; base < nb; base += 32) {
    const int64_t idx = base + lane;
    const unsigned long long v = idx < nb ? bs[idx] : BF_NO_START;
    const uint32_t m = __ballot_sync(FULL_MASK, v != BF_NO_START);
    if (m) {
      const unsigned long long f = __shfl_sync(FULL_MASK, v, __ffs(m) - 1);
      return (int64_t)f < n ? (int64_t)f : n;
    }
  }
  return n;
}

// Shared memory of a filter block keeping up to LIST records, with a
// 2^SEEN-bit "seen" bitmap (the "seen again" one has 2^BF_BITS bits).
template <int LIST, int SEEN>
struct BfSmem {
  uint32_t seen[(1 << SEEN) / 32];
  uint32_t again[BF_WORDS];
  uint64_t list[LIST];
  uint32_t tk[2 * LIST];
  uint32_t tc[LIST];
  uint32_t ids[LIST];
};

// BF_LIST: records a block may keep (512 for two-bucket segments, whose
// direct 17-bit "seen" bitmap keeps about 8% of ~3,200 records; 1,024 for
// one bucket and 2,048 for larger segments with 16-bit bitmaps).
// BF_ITEMS: records per thread of one chunk in registers (a segment of up to
// BF_THREADS * BF_ITEMS records is read once).
// HIW (lo >= 32): the group key lies in the record's high word, so the
// composite key comes from a 32-bit shift.
// SEEN: log2 of the bits of the "seen" bitmap.  With SEEN = 17 a two-bucket
// segment's composite keys (17 bits) index it directly, so only keys that
// really occur twice (or share their 32-bit group key) set "seen again"; its
// own 16-bit index is hashed, and a rare collision there only keeps a
// record that the exact grouping then finds alone.
template <int BF_LIST, int BF_ITEMS, bool HIW, int SEEN>
__global__ void __launch_bounds__(BF_THREADS, BF_LIST <= 1024 ? 5 : 3)
    k_bucket_filter(const uint64_t* __restrict__ A, int64_t n_cap,
                    const uint64_t* __restrict__ n_dev,
                    const unsigned long long* __restrict__ bucket_start, int G, int kf, int fx,
                    int lo, int L, uint64_t* __restrict__ cand, uint64_t cand_cap,
                    unsigned long long* __restrict__ cand_count, int id_bits,
                    uint32_t* __restrict__ seg_list, uint32_t* __restrict__ seg_count,
                    uint32_t* __restrict__ err) {
  constexpr int BF_CHUNK = BF_THREADS * BF_ITEMS;  // records per chunk
  constexpr int BF_HMAX = 2 * BF_LIST;          // slots of the exact grouping, at most
  constexpr int BF_PT = BF_LIST / BF_THREADS;   // kept records per thread, at most
  extern __shared__ __align__(16) unsigned char bf_smem[];
  BfSmem<BF_LIST, SEEN>& S = *reinterpret_cast<BfSmem<BF_LIST, SEEN>*>(bf_smem);
  constexpr int SEEN_WORDS = (1 << SEEN) / 32;
  uint32_t* s_seen = S.seen;
  uint32_t* s_again = S.again;
  uint64_t* s_list = S.list;
  uint32_t* s_tk = S.tk;  // composite keys, then group sizes
  uint32_t* s_tc = S.tc;  // u16 counts, then u16 starts
  uint32_t* s_ids = S.ids;
  __shared__ int64_t s_range[2];
  __shared__ uint32_t s_nlist;
  __shared__ uint32_t s_wsum[BF_WARPS];
  __shared__ uint32_t s_wp[BF_WARPS];  // candidate words of each warp
  __shared__ unsigned long long s_obase;

  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  const int64_t nb = 1ll << G;
  const int64_t K = 1ll << kf;
  const int64_t b0 = (int64_t)blockIdx.x * K;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const bool direct = L + kf <= SEEN;
  const uint64_t idmask = (1ull << id_bits) - 1ull;
  // warps 0 and 1 find the segment's first and end record, the rest clear
  if (warp < 2) {
    int64_t v = warp == 0 ? 0 : n;
    if (G > 0) {
      const int64_t bf = warp == 0 ? b0 : b0 + K;
      v = bf >= nb ? n : bf_first_start(bucket_start, bf, nb, n, lane);
    }
    if (lane == 0) s_range[warp] = v;
  } else {
    for (int k = threadIdx.x - 64; k < (SEEN_WORDS + BF_WORDS) / 4; k += BF_THREADS - 64) {
      uint4* z = k < SEEN_WORDS / 4 ? reinterpret_cast<uint4*>(s_seen) + k
                                    : reinterpret_cast<uint4*>(s_again) + (k - SEEN_WORDS / 4);
      *z = make_uint4(0u, 0u, 0u, 0u);
    }
    // the exact grouping's tables, whole (they are first used after several
    // barriers; clearing them here saves that phase its own barrier)
    for (int k = threadIdx.x - 64; k < 2 * BF_LIST / 4; k += BF_THREADS - 64)
      reinterpret_cast<uint4*>(s_tk)[k] = make_uint4(BF_EMPTY, BF_EMPTY, BF_EMPTY, BF_EMPTY);
    for (int k = threadIdx.x - 64; k < BF_LIST / 4; k += BF_THREADS - 64)
      reinterpret_cast<uint4*>(s_tc)[k] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (threadIdx.x == 0) s_nlist = 0;
  __syncthreads();
  const int64_t s = s_range[0], e = s_range[1] > s_range[0] ? s_range[1] : s_range[0];
  const int64_t m = e - s;
  if (m < 2) return;  // block-uniform
  const uint64_t cbase = (uint64_t)b0 << L;
  auto comp = [&](uint64_t key) {
    return HIW ? ((uint32_t)(key >> 32) >> (lo - 32)) - (uint32_t)cbase
               : (uint32_t)((key >> lo) - cbase);
  };
  auto bit_of = [&](uint32_t c) {  // index in "seen"
    return (direct ? c : (c * 0x9E3779B1u) >> (32 - SEEN)) & ((1u << SEEN) - 1u);
  };
  auto again_of = [&](uint32_t c) {  // index in "seen again"
    return SEEN == BF_BITS ? bit_of(c) : (c * 0x9E3779B1u) >> (32 - BF_BITS);
  };
  const int wbase = (int)warp * 32 * BF_ITEMS;
  // 1. mark keys seen and seen again (chunk by chunk; the last chunk stays in
  // registers)
  uint64_t key[BF_ITEMS];
  for (int64_t c0 = 0; c0 < m; c0 += BF_CHUNK) {
    const int cm = (int)min((int64_t)BF_CHUNK, m - c0);
#pragma unroll
    for (int i = 0; i < BF_ITEMS; ++i) {
      const int pos = wbase + i * 32 + (int)lane;
      key[i] = pos < cm ? A[s + c0 + pos] : 0ull;
    }
#pragma unroll
    for (int i = 0; i < BF_ITEMS; ++i) {
      if (wbase + i * 32 + (int)lane < cm) {
        const uint32_t c = comp(key[i]);
        const uint32_t h = bit_of(c), bit = 1u << (h & 31u);
        if (atomicOr(&s_seen[h >> 5], bit) & bit) {
          const uint32_t a = again_of(c);
          atomicOr(&s_again[a >> 5], 1u << (a & 31u));
        }
      }
    }
  }
  __syncthreads();
  // 2. keep the records whose key was seen again
  for (int64_t c0 = 0; c0 < m; c0 += BF_CHUNK) {
    const int cm = (int)min((int64_t)BF_CHUNK, m - c0);
    if (m > BF_CHUNK) {
#pragma unroll
      for (int i = 0; i < BF_ITEMS; ++i) {
        const int pos = wbase + i * 32 + (int)lane;
        key[i] = pos < cm ? A[s + c0 + pos] : 0ull;
      }
    }
    // the warp's kept records of the chunk, one reservation for all items
    uint32_t bal[BF_ITEMS];
    uint32_t wkept = 0;
#pragma unroll
    for (int i = 0; i < BF_ITEMS; ++i) {
      bool keep = false;
      if (wbase + i * 32 + (int)lane < cm) {
        const uint32_t a = again_of(comp(key[i]));
        keep = (s_again[a >> 5] >> (a & 31u)) & 1u;
      }
      bal[i] = __ballot_sync(FULL_MASK, keep);
      wkept += (uint32_t)__popc(bal[i]);
    }
    uint32_t at = 0;
    if (lane == 0 && wkept) at = atomicAdd(&s_nlist, wkept);
    at = __shfl_sync(FULL_MASK, at, 0);
#pragma unroll
    for (int i = 0; i < BF_ITEMS; ++i) {
      if ((bal[i] >> lane) & 1u) {
        const uint32_t a = at + (uint32_t)__popc(bal[i] & lt_mask);
        if (a < (uint32_t)BF_LIST) s_list[a] = key[i];
      }
      at += (uint32_t)__popc(bal[i]);
    }
  }
  __syncthreads();
  const uint32_t kept = s_nlist;
  if (kept > (uint32_t)BF_LIST) {  // too many: k_bucket groups this segment's blocks
    __shared__ uint32_t s_at;
    if (threadIdx.x == 0) s_at = atomicAdd(seg_count, 1u << fx);
    __syncthreads();
    const uint32_t f0 = (uint32_t)blockIdx.x << fx;
    for (uint32_t f = threadIdx.x; f < (1u << fx); f += BF_THREADS) seg_list[s_at + f] = f0 + f;
    return;
  }
  if (kept < 2) return;
  // 3. exact grouping of the kept records: H = 2^hb >= 2 kept slots, at least
  // two per thread; thread t owns slots [t PER, t PER + PER)
  int hb = 9;
  while ((1u << hb) < 2 * kept) ++hb;
  const uint32_t H = 1u << hb;  // 512 .. BF_HMAX; tables cleared in phase 0
  const uint32_t PER = H / BF_THREADS;
  uint32_t sr[BF_PT];  // slot << 16 | rank in the slot's group
#pragma unroll
  for (int i = 0; i < BF_PT; ++i) {
    const uint32_t j = threadIdx.x + (uint32_t)i * BF_THREADS;
    sr[i] = 0xffffffffu;
    if (j < kept) {
      const uint32_t c = comp(s_list[j]);
      uint32_t h = (c * 0x9E3779B1u) >> (32 - hb);
      bool found = false;
      for (uint32_t probe = 0; probe < H; ++probe) {  // at most kept <= H/2 keys: ends
        const uint32_t old = atomicCAS(&s_tk[h], BF_EMPTY, c);
        if (old == BF_EMPTY || old == c) {
          found = true;
          break;
        }
        h = (h + 1) & (H - 1);
      }
      if (found) {
        const uint32_t sh = (h & 1u) * 16;
        sr[i] = (h << 16) | ((atomicAdd(&s_tc[h >> 1], 1u << sh) >> sh) & 0xffffu);
      } else {
        atomicOr(err, DERR_RANGE);
      }
    }
  }
  __syncthreads();
  // slot scan: only groups of two or more are placed; their sizes go to the
  // key table, their starts over the counts
  uint32_t tot = 0;
  for (uint32_t q = 0; q < PER / 2; ++q) {
    const uint32_t w = s_tc[threadIdx.x * (PER / 2) + q];
    const uint32_t a = w & 0xffffu, b = w >> 16;
    tot += (a >= 2 ? a : 0u) + (b >= 2 ? b : 0u);
  }
  uint32_t inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL_MASK, inc, o);
    if (lane >= (uint32_t)o) inc += t;
  }
  if (lane == 31) s_wsum[warp] = inc;
  __syncthreads();
  uint32_t run = inc - tot;
  for (uint32_t w = 0; w < warp; ++w) run += s_wsum[w];
  uint32_t gmask = 0, np = 0;  // bit k: slot threadIdx.x * PER + k holds a group
  for (uint32_t q = 0; q < PER / 2; ++q) {
    const uint32_t idx = threadIdx.x * (PER / 2) + q;
    const uint32_t w = s_tc[idx];
    const uint32_t a = w & 0xffffu, b = w >> 16;
    const uint32_t h = 2 * idx;
    const uint32_t sa = a >= 2 ? run : BF_NO_PLACE;
    run += a >= 2 ? a : 0u;
    const uint32_t sb = b >= 2 ? run : BF_NO_PLACE;
    run += b >= 2 ? b : 0u;
    s_tc[idx] = sa | (sb << 16);
    if (a >= 2) {
      s_tk[h] = a;
      gmask |= 1u << (2 * q);
      np += a * (a - 1) / 2;
    }
    if (b >= 2) {
      s_tk[h + 1] = b;
      gmask |= 2u << (2 * q);
      np += b * (b - 1) / 2;
    }
  }
  // output room: the pairs of a lane's small groups (at most BF_SMALL ids)
  // at the lane's offset in its warp's room, those of large groups after all
  // small ones; the block reserves the room of all its warps at once (one
  // atomic on the shared counter per block, not per warp, which kept the
  // counter's address busy)
  uint32_t np_small = 0;
  for (uint32_t g = gmask; g; g &= g - 1) {
    const uint32_t c = s_tk[threadIdx.x * PER + (uint32_t)(__ffs(g) - 1)];
    if (c <= BF_SMALL) np_small += c * (c - 1) / 2;
  }
  uint32_t small_incl = np_small;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL_MASK, small_incl, o);
    if (lane >= (uint32_t)o) small_incl += t;
  }
  const uint32_t small_total = __shfl_sync(FULL_MASK, small_incl, 31);
  uint32_t wp = np;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wp += __shfl_xor_sync(FULL_MASK, wp, o);
  if (lane == 0) s_wp[warp] = wp;
  __syncthreads();
  unsigned long long bres = 0;  // thread 0: the block's room (its wait overlaps step 4)
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < BF_WARPS; ++w) tot += s_wp[w];
    if (tot) {
      bres = atomicAdd(cand_count, (unsigned long long)tot);
      if (bres + tot > cand_cap) atomicOr(err, DERR_CAPACITY);
    }
  }
  // 4. each group's ids, contiguous
#pragma unroll
  for (int i = 0; i < BF_PT; ++i) {
    if (sr[i] != 0xffffffffu) {
      const uint32_t h = sr[i] >> 16;
      const uint32_t start = (s_tc[h >> 1] >> ((h & 1u) * 16)) & 0xffffu;
      if (start != BF_NO_PLACE) {
        const uint32_t pos = start + (sr[i] & 0xffffu);
        const uint32_t j = threadIdx.x + (uint32_t)i * BF_THREADS;
        if (pos < kept) s_ids[pos] = (uint32_t)(s_list[j] & idmask);
        else atomicOr(err, DERR_RANGE);
      }
    }
  }
  if (threadIdx.x == 0) s_obase = bres;
  __syncthreads();
  unsigned long long obase = s_obase;
  for (uint32_t w = 0; w < warp; ++w) obase += s_wp[w];
  auto word = [&](uint64_t ia, uint64_t ib) {
    return ((ia < ib ? ia : ib) << id_bits) | (ia < ib ? ib : ia);
  };
  // 5a. small groups: the owning lane writes all their pairs
  {
    unsigned long long o = obase + (small_incl - np_small);
    uint32_t large = 0;  // this lane's large groups (bit k: slot threadIdx.x * PER + k)
    for (uint32_t g = gmask; g; g &= g - 1) {
      const uint32_t k = (uint32_t)(__ffs(g) - 1);
      const uint32_t h = threadIdx.x * PER + k;
      const uint32_t c = s_tk[h];
      if (c > BF_SMALL) {
        large |= 1u << k;
        continue;
      }
      const uint32_t gst = (s_tc[h >> 1] >> ((h & 1u) * 16)) & 0xffffu;
      if (gst + c > (uint32_t)BF_LIST) continue;
      for (uint32_t x = 0; x + 1 < c; ++x) {
        const uint64_t ia = s_ids[gst + x];
        for (uint32_t y = x + 1; y < c; ++y, ++o)
          if (o < cand_cap) cand[o] = word(ia, s_ids[gst + y]);
      }
    }
    gmask = large;
  }
  // 5b. large groups: the warp spreads each one's pairs over its lanes
  // (colex rank l = b (b - 1) / 2 + a, a < b)
  obase += small_total;
  while (__any_sync(FULL_MASK, gmask != 0)) {
    uint32_t st = 0, c = 0;
    if (gmask) {
      const uint32_t h = threadIdx.x * PER + (uint32_t)(__ffs(gmask) - 1);
      gmask &= gmask - 1;
      st = (s_tc[h >> 1] >> ((h & 1u) * 16)) & 0xffffu;
      c = s_tk[h];
    }
    uint32_t groups = __ballot_sync(FULL_MASK, c >= 2);
    while (groups) {
      const int src = __ffs(groups) - 1;
      groups &= groups - 1;
      const uint32_t gst = __shfl_sync(FULL_MASK, st, src);
      const uint32_t gc = __shfl_sync(FULL_MASK, c, src);
      const uint32_t pairs = gc * (gc - 1) / 2;
      for (uint32_t l = lane; l < pairs; l += 32) {
        uint32_t bb = (uint32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)l)) * 0.5f);
        while (bb * (bb - 1) / 2 > l) --bb;
        while ((bb + 1) * bb / 2 <= l) ++bb;
        const uint32_t aa = l - bb * (bb - 1) / 2;
        if (gst + bb < (uint32_t)BF_LIST && obase + l < cand_cap)
          cand[obase + l] = word(s_ids[gst + aa], s_ids[gst + bb]);
      }
      obase += pairs;
    }
  }
}

}  // namespace

template <int LIST, int ITEMS, int SEEN>
void bucket_filter_launch(uint64_t blocks, bool hiw, const uint64_t* A, int64_t n,
                          const uint64_t* n_dev, const unsigned long long* bs,
                          const GroupingShape& g, int kf, int fx, int lo, uint64_t* cand,
                          uint64_t cand_cap, unsigned long long* cc, int id_bits,
                          uint32_t* seg_list, uint32_t* seg_count, uint32_t* err,
                          cudaStream_t s) {
  static std::once_flag once;
  std::call_once(once, [] {
    for (auto f : {k_bucket_filter<LIST, ITEMS, false, SEEN>, k_bucket_filter<LIST, ITEMS, true, SEEN>}) {
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(BfSmem<LIST, SEEN>));
      cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
  });
  auto f = hiw ? k_bucket_filter<LIST, ITEMS, true, SEEN> : k_bucket_filter<LIST, ITEMS, false, SEEN>;
  f<<<(uint32_t)blocks, BF_THREADS, sizeof(BfSmem<LIST, SEEN>), s>>>(A, n, n_dev, bs, g.G, kf, fx, lo,
                                                               g.L, cand, cand_cap, cc, id_bits,
                                                               seg_list, seg_count, err);
}

void launch_bucket_filter(const uint64_t* A, int64_t n, const uint64_t* n_dev,
                          const uint64_t* bucket_start, const GroupingShape& g, int fx, int lo,
                          uint64_t* cand, uint64_t cand_cap, uint64_t* cand_count, int id_bits,
                          uint32_t* seg_list, uint32_t* seg_count, uint32_t* err, cudaStream_t s) {
  if (n <= 0) return;
  // the filter's segments: 2^fx of k_bucket's blocks of buckets each
  while (fx > 0 && (g.kbits + fx > g.G || g.L + g.kbits + fx > 31)) --fx;
  const int kf = g.kbits + fx;
  const uint64_t blocks = ((uint64_t)1 << g.G) >> kf;
  const auto bs = reinterpret_cast<const unsigned long long*>(bucket_start);
  const auto cc = reinterpret_cast<unsigned long long*>(cand_count);
  const bool hiw = lo >= 32;
  prof_begin(s, "k_bucket_filter", (double)n * 8.0);
  // the chunk in registers covers the expected segment: ~1,600 records a
  // bucket at the sizes G is chosen for
  if (fx >= 2)
    bucket_filter_launch<2048, 8, BF_BITS>(blocks, hiw, A, n, n_dev, bs, g, kf, fx, lo, cand,
                                           cand_cap, cc, id_bits, seg_list, seg_count, err, s);
  else if (fx == 1)
    bucket_filter_launch<512, 13, 17>(blocks, hiw, A, n, n_dev, bs, g, kf, fx, lo, cand, cand_cap,
                                      cc, id_bits, seg_list, seg_count, err, s);
  else
    bucket_filter_launch<1024, 8, BF_BITS>(blocks, hiw, A, n, n_dev, bs, g, kf, fx, lo, cand,
                                           cand_cap, cc, id_bits, seg_list, seg_count, err, s);
  prof_end(s);
}

}  // namespace xtn
