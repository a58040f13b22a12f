// Least-significant-digit radix sort of 64-bit keys on a bit range [lo, hi),
// 8-bit digits, one read and one write of the keys per digit ("onesweep":
// the digit offsets of a tile come from a decoupled look-back over the
// preceding tiles instead of a separate upsweep pass; Adinets & Merrill 2022).
// This is the grouping step of Appendix A, XTNeighbor step 4 (the paper's
// `sortKeyValues`) and the pair sort of step 6 (`sort`).  The output is
// sorted on [lo, hi); keys equal on those bits come in no particular order
// (every first pass ranks unstably), which no caller needs.
//
// k_onesweep, one tile = THREADS x ITEMS keys:
//   1. load: warp w reads its contiguous 32*ITEMS keys, item-major, so each
//      load instruction is a 256-byte coalesced run;
//   2. rank: per item, the lanes holding the same digit are found with one
//      ballot per digit bit; the lowest of them bumps the warp's private
//      256-bin counter in shared memory (stable warp-level multi-split);
//   3. the per-warp counts become per-digit warp offsets and tile counts;
//      the tile count of each digit is published for the look-back;
//   4. keys are scattered into shared memory in digit order;
//   5. thread t looks back along digit t's chain to get the number of keys
//      with digit t in all earlier tiles;
//   6. keys leave shared memory in digit order: runs of one digit land on
//      consecutive addresses.
// k_onesweep_runs (further down) keeps the same steps but counts and places
// keys with shared-memory atomics instead of keeping ranks in registers.
#include <algorithm>
#include <mutex>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

// Global digit histograms of every pass in one read of the keys.
__global__ void k_histogram(const uint64_t* __restrict__ keys, int64_t n, int lo, int hi,
                            uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  const int passes = (hi - lo + 7) / 8;
  for (int k = threadIdx.x; k < passes * RADIX; k += blockDim.x) s_hist[k] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    for (int p = 0; p < passes; ++p) {
      const int sh = lo + 8 * p;
      const int bits = min(8, hi - sh);
      atomicAdd(&s_hist[p * RADIX + (uint32_t)((k >> sh) & ((1u << bits) - 1u))], 1u);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < passes * RADIX; k += blockDim.x)
    if (s_hist[k]) atomicAdd(&hist[k], s_hist[k]);
}

// digit_base[p][r] = number of keys whose pass-p digit is < r.
__global__ void k_digit_scan(const uint32_t* __restrict__ hist, uint64_t* __restrict__ digit_base) {
  __shared__ uint64_t s_w[RADIX / 32];
  const int p = blockIdx.x, t = threadIdx.x;
  const uint64_t v = hist[p * RADIX + t];
  const uint64_t inc = warp_incl_scan_u64(v);
  if ((t & 31) == 31) s_w[t >> 5] = inc;
  __syncthreads();
  uint64_t off = 0;
  for (int w = 0; w < (t >> 5); ++w) off += s_w[w];
  digit_base[p * RADIX + t] = off + inc - v;
}

template <int THREADS, int ITEMS, int MATCH = 0, int NCHAIN = 1>
struct OnesweepSmem {
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr size_t keys_bytes = (size_t)TILE * 8;
  static constexpr size_t whist_bytes = (size_t)NCHAIN * WARPS * RADIX * 4;
  static constexpr size_t match_bytes = MATCH == 2 ? (size_t)NCHAIN * WARPS * RADIX * 4 : 0;
  static constexpr size_t bytes = keys_bytes + whist_bytes + RADIX * 4 + RADIX * 8 + match_bytes;
};

// Lanes of the warp holding the same digit as this lane (lanes with !valid
// excluded).  MATCH = 0: one ballot per digit bit; MATCH = 1: match.any.
template <int MATCH>
__device__ __forceinline__ uint32_t digit_peers(uint32_t dig, uint32_t valid_mask) {
  if (MATCH == 1) return __match_any_sync(FULL_MASK, dig) & valid_mask;
  uint32_t peers = valid_mask;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const uint32_t bal = __ballot_sync(FULL_MASK, (dig >> b) & 1u);
    peers &= ((dig >> b) & 1u) ? bal : ~bal;
  }
  return peers;
}

// Stable rank of every item inside its warp (warp-private 256-bin counters).
// MATCH = 2: each lane ORs its bit into a per-warp bin of its digit and reads
// the bin back as its peer mask; the lowest peer bumps the counter, clears
// the bin and hands the old count to its peers with one shuffle.
template <int ITEMS, int MATCH, bool FULL>
__device__ __forceinline__ void rank_items(const uint64_t (&key)[ITEMS], uint16_t (&rank)[ITEMS],
                                           uint32_t* wh, uint32_t* mb, int64_t wbase, int64_t n,
                                           int shift, uint32_t dmask, uint32_t lane) {
  const uint32_t lt_mask = (1u << lane) - 1u;
  if (MATCH == 4) {
    // unstable: one shared-memory atomic per item.  Ranks within a warp
    // follow no order, so only a pass whose input order does not matter may
    // use it (the first pass of a sort).
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = FULL || (wbase + i * 32 + lane < n);
      if (valid) rank[i] = (uint16_t)atomicAdd(&wh[(uint32_t)(key[i] >> shift) & dmask], 1u);
    }
    return;
  }
  if (MATCH == 3) {
    // ballot match; the lowest peer adds the group's size to the warp counter
    // with one shared atomic and hands the old count to its peers
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = FULL || (wbase + i * 32 + lane < n);
      const uint32_t dig = (uint32_t)(key[i] >> shift) & dmask;
      const uint32_t vmask = FULL ? FULL_MASK : __ballot_sync(FULL_MASK, valid);
      const uint32_t peers = digit_peers<0>(dig, vmask);
      const uint32_t before = peers & lt_mask;
      uint32_t old = 0;
      if (valid && before == 0) old = atomicAdd(&wh[dig], (uint32_t)__popc(peers));
      old = __shfl_sync(FULL_MASK, old, valid ? __ffs(peers) - 1 : (int)lane);
      rank[i] = (uint16_t)(old + __popc(before));
      __syncwarp();  // this item's counter update is seen by the next item
    }
    return;
  }
  if (MATCH == 2) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = FULL || (wbase + i * 32 + lane < n);
      const uint32_t dig = (uint32_t)(key[i] >> shift) & dmask;
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
      const int leader = valid ? __ffs(peers) - 1 : (int)lane;
      old = __shfl_sync(FULL_MASK, old, leader);
      rank[i] = (uint16_t)(old + __popc(before));
      __syncwarp();
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const bool valid = FULL || (wbase + i * 32 + lane < n);
    const uint32_t dig = (uint32_t)(key[i] >> shift) & dmask;
    const uint32_t vmask = FULL ? FULL_MASK : __ballot_sync(FULL_MASK, valid);
    const uint32_t peers = digit_peers<MATCH>(dig, vmask);
    const uint32_t before = peers & lt_mask;
    uint32_t base = 0;
    if (valid) base = wh[dig];
    __syncwarp();
    if (valid && before == 0) wh[dig] = base + __popc(peers);
    __syncwarp();
    rank[i] = (uint16_t)(base + __popc(before));
  }
}

// Two ranking chains per warp: items [0, H) use counters whA / bins mbA and
// items [H, ITEMS) use whB / mbB, one item of each per step, so the shared-
// memory round trips of the two chains overlap.  The halves stay in item
// order; the scatter offsets second-half ranks by the first half's counts.
template <int ITEMS, int MATCH, bool FULL>
__device__ __forceinline__ void rank_items2(const uint64_t (&key)[ITEMS], uint16_t (&rank)[ITEMS],
                                            uint32_t* whA, uint32_t* whB, uint32_t* mbA,
                                            uint32_t* mbB, int64_t wbase, int64_t n, int shift,
                                            uint32_t dmask, uint32_t lane) {
  constexpr int H = ITEMS / 2;
  static_assert(ITEMS % 2 == 0, "two equal halves");
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const bool va = FULL || (wbase + k * 32 + lane < n);
    const bool vb = FULL || (wbase + (H + k) * 32 + lane < n);
    const uint32_t da = (uint32_t)(key[k] >> shift) & dmask;
    const uint32_t db = (uint32_t)(key[H + k] >> shift) & dmask;
    uint32_t pa, pb;
    if (MATCH == 2) {
      if (va) atomicOr(&mbA[da], 1u << lane);
      if (vb) atomicOr(&mbB[db], 1u << lane);
      __syncwarp();
      pa = va ? mbA[da] : 0u;
      pb = vb ? mbB[db] : 0u;
      __syncwarp();
    } else {
      const uint32_t vma = FULL ? FULL_MASK : __ballot_sync(FULL_MASK, va);
      const uint32_t vmb = FULL ? FULL_MASK : __ballot_sync(FULL_MASK, vb);
      pa = digit_peers<0>(da, vma);
      pb = digit_peers<0>(db, vmb);
    }
    const uint32_t ba = pa & lt_mask, bb = pb & lt_mask;
    uint32_t oa = 0, ob = 0;
    if (va && ba == 0) {
      oa = whA[da];
      whA[da] = oa + __popc(pa);
      if (MATCH == 2) mbA[da] = 0u;
    }
    if (vb && bb == 0) {
      ob = whB[db];
      whB[db] = ob + __popc(pb);
      if (MATCH == 2) mbB[db] = 0u;
    }
    oa = __shfl_sync(FULL_MASK, oa, va ? __ffs(pa) - 1 : (int)lane);
    ob = __shfl_sync(FULL_MASK, ob, vb ? __ffs(pb) - 1 : (int)lane);
    rank[k] = (uint16_t)(oa + __popc(ba));
    rank[H + k] = (uint16_t)(ob + __popc(bb));
    __syncwarp();
  }
}

template <int THREADS, int ITEMS, int MIN_BLOCKS, int MATCH, int NCHAIN = 1>
__global__ void __launch_bounds__(THREADS, MIN_BLOCKS)
    k_onesweep(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
               const uint64_t* __restrict__ n_dev, int64_t n_cap, int shift,
               int bits, const uint64_t* __restrict__ digit_base, uint64_t* __restrict__ status,
               uint32_t* __restrict__ ctr, uint32_t* __restrict__ err,
               uint32_t* __restrict__ next_hist, int next_bits,
               unsigned long long* __restrict__ bucket_start, int bucket_shift) {
  using SM = OnesweepSmem<THREADS, ITEMS, MATCH, NCHAIN>;
  constexpr int WARPS = SM::WARPS;
  constexpr int TILE = SM::TILE;
  static_assert(THREADS >= RADIX, "one thread per digit");
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);
  uint32_t* s_whist = reinterpret_cast<uint32_t*>(smem + SM::keys_bytes);
  uint32_t* s_tstart = s_whist + NCHAIN * WARPS * RADIX;
  int64_t* s_obase = reinterpret_cast<int64_t*>(s_tstart + RADIX);
  uint32_t* s_match = reinterpret_cast<uint32_t*>(s_obase + RADIX);
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wsum[THREADS / 32];
  __shared__ uint32_t s_next[RADIX];  // digit counts of the next pass (when next_hist)

  if (next_hist)
    for (int k = threadIdx.x; k < RADIX; k += THREADS) s_next[k] = 0;
  // key count: on the device when the caller did not know it at launch time
  // (grid sized for n_cap; blocks whose tile starts past the count leave at
  // once -- tiles are numbered in start order, so no live tile waits on them)
  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  const uint32_t tile = tile_id(ctr, &s_tile);
  const int64_t tile_base = (int64_t)tile * TILE;
  if (tile_base >= n) return;
  const bool full = tile_base + TILE <= n;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t dmask = (1u << bits) - 1u;

  for (int k = threadIdx.x; k < NCHAIN * WARPS * RADIX; k += THREADS) s_whist[k] = 0;
  if (MATCH == 2)
    for (int k = threadIdx.x; k < NCHAIN * WARPS * RADIX; k += THREADS) s_match[k] = 0;

  // 1. load: warp w reads its contiguous 32*ITEMS keys item-major
  uint64_t key[ITEMS];
  const int64_t wbase = tile_base + (int64_t)warp * 32 * ITEMS;
  if (full) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) key[i] = __ldcs(in + wbase + i * 32 + lane);
  } else {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int64_t pos = wbase + i * 32 + lane;
      key[i] = pos < n ? __ldcs(in + pos) : 0ull;
    }
  }
  __syncthreads();

  // 2. stable warp multi-split ranking
  // chain c of warp w keeps its counters at s_whist[(c * WARPS + w) * RADIX]
  uint32_t* wh = s_whist + warp * RADIX;
  uint32_t* whB = s_whist + (WARPS + warp) * RADIX;
  uint32_t* mb = s_match + warp * RADIX;
  uint32_t* mbB = s_match + (WARPS + warp) * RADIX;
  uint16_t rank[ITEMS];
  if (NCHAIN == 2) {
    if (full) rank_items2<ITEMS, MATCH, true>(key, rank, wh, whB, mb, mbB, wbase, n, shift, dmask, lane);
    else rank_items2<ITEMS, MATCH, false>(key, rank, wh, whB, mb, mbB, wbase, n, shift, dmask, lane);
  } else {
    if (full) rank_items<ITEMS, MATCH, true>(key, rank, wh, mb, wbase, n, shift, dmask, lane);
    else rank_items<ITEMS, MATCH, false>(key, rank, wh, mb, wbase, n, shift, dmask, lane);
  }
  __syncthreads();

  // 3. warp offsets per digit, tile counts, publish aggregates
  uint32_t tcount = 0;
  if (threadIdx.x < RADIX) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      const uint32_t c = s_whist[w * RADIX + threadIdx.x];
      s_whist[w * RADIX + threadIdx.x] = run;
      run += c;
      if (NCHAIN == 2) {
        const uint32_t c2 = s_whist[(WARPS + w) * RADIX + threadIdx.x];
        s_whist[(WARPS + w) * RADIX + threadIdx.x] = run;
        run += c2;
      }
    }
    tcount = run;
    st_status(&status[(uint64_t)tile * RADIX + threadIdx.x], (tile == 0 ? ST_INC : ST_AGG) | run);
  }
  // exclusive scan of tile counts over digits
  {
    const uint32_t v = tcount;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL_MASK, inc, o);
      if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (threadIdx.x < RADIX) {
      uint32_t off = 0;
      for (uint32_t w = 0; w < warp; ++w) off += s_wsum[w];
      const uint32_t ts = off + inc - v;
      s_tstart[threadIdx.x] = ts;
      // per-warp offsets become absolute positions in the tile's digit order
#pragma unroll
      for (int w = 0; w < NCHAIN * WARPS; ++w) s_whist[w * RADIX + threadIdx.x] += ts;
    }
    __syncthreads();
  }

  // 4. scatter into shared memory in digit order
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (full || wbase + i * 32 + lane < n) {
      const uint32_t dig = (uint32_t)(key[i] >> shift) & dmask;
      const uint32_t* whi = (NCHAIN == 2 && i >= ITEMS / 2) ? whB : wh;
      s_keys[whi[dig] + rank[i]] = key[i];
    }
  }

  // 5. look-back per digit
  if (threadIdx.x < RADIX) {
    uint64_t excl = 0;
    if (tile > 0) {
      excl = thread_lookback(status + threadIdx.x, tile, RADIX, err);
      st_status(&status[(uint64_t)tile * RADIX + threadIdx.x], ST_INC | (excl + tcount));
    }
    s_obase[threadIdx.x] = (int64_t)(digit_base[threadIdx.x] + excl) - (int64_t)s_tstart[threadIdx.x];
  }
  __syncthreads();

  // 6. write out in digit order (and count the next pass's digit: the keys
  // pass through registers here anyway, and the ranking above has none to spare)
  const int tile_n = full ? TILE : (int)(n - tile_base);
  for (int j = threadIdx.x; j < tile_n; j += THREADS) {
    const uint64_t k = s_keys[j];
    const uint32_t dig = (uint32_t)(k >> shift) & dmask;
    if (next_hist) atomicAdd(&s_next[(uint32_t)(k >> (shift + 8)) & ((1u << next_bits) - 1u)], 1u);
    const int64_t o = s_obase[dig] + j;
    if (o >= 0 && o < n) out[o] = k;
    else atomicOr(err, DERR_RANGE);
    // last pass: bucket = the bits this and the earlier passes sorted on
    // (from bucket_shift up).  A bucket starts at o when the record before it
    // in the output holds another bucket; for the first record of this tile's
    // digit run that record sits in another tile, so every such candidate
    // offers its position and the smallest one wins.
    if (bucket_start && o >= 0 && o < n) {
      const uint64_t b = k >> bucket_shift;
      if (j == (int)s_tstart[dig] || b != (s_keys[j - 1] >> bucket_shift))
        atomicMin(&bucket_start[b], (unsigned long long)o);
    }
  }
  if (next_hist) {  // uniform over the block
    __syncthreads();  // every count of the write loop is in
    if (threadIdx.x < RADIX && s_next[threadIdx.x])
      atomicAdd(&next_hist[threadIdx.x], s_next[threadIdx.x]);
  }
}

// ---------------------------------------------------------------------------
// k_onesweep_runs: a pass without per-key rank registers.
//
// The input of every pass after the first is sorted on the bits below the
// current digit, [lo, shift), so a tile of it holds a few runs of equal lower
// bits, in order.  When a tile spans at most OS_RUNS lower-bit values (its
// first and last keys tell), its keys are counted, and then placed, with
// shared-memory atomics on bins (run, digit): each digit leaves the tile with
// its keys ordered by run, and the tiles leave in order, so the output is
// sorted on [lo, shift + bits).  Keys equal on all those bits may change
// places, which no later pass and no caller needs (the first pass has no lower
// bits: one run).  A tile spanning more lower-bit values (an input with few
// keys per value) is ranked stably instead: per-warp counts first, then
// ballots in item order.  Without ranks in registers a block needs about 20
// fewer registers per thread, so more blocks fit on an SM.
// The last pass of a grouping sort (bucket_start given; the sort ends at bit
// 64) records where each bucket (key >> lo) starts: per run of a digit in the
// fast case, per key at a bucket change otherwise.
constexpr int OS_RUNS = 4;

template <int THREADS, int ITEMS>
struct RunsSmem {
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr int CNT = (OS_RUNS > WARPS ? OS_RUNS : WARPS) * RADIX;
  static constexpr size_t keys_bytes = (size_t)TILE * 8;
  static constexpr size_t bytes = keys_bytes + (size_t)CNT * 4 + RADIX * 4 + RADIX * 8;
};

template <int THREADS, int ITEMS, int MIN_BLOCKS, int LBW, int DB, int UW, bool HIW>
__global__ void __launch_bounds__(THREADS, MIN_BLOCKS)
    k_onesweep_runs(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                    const uint64_t* __restrict__ n_dev, int64_t n_cap, int shift, int bits, int lo,
                    const uint64_t* __restrict__ digit_base, uint64_t* __restrict__ status,
                    uint32_t* __restrict__ ctr, uint32_t* __restrict__ err,
                    uint32_t* __restrict__ next_hist, int next_bits,
                    unsigned long long* __restrict__ bucket_start,
                    uint64_t* __restrict__ status_next, uint32_t* __restrict__ ctr_next) {
  using SM = RunsSmem<THREADS, ITEMS>;
  constexpr int WARPS = SM::WARPS;
  constexpr int TILE = SM::TILE;
  static_assert(THREADS >= RADIX, "one thread per digit");
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + SM::keys_bytes);
  uint32_t* s_tstart = s_cnt + SM::CNT;
  int64_t* s_obase = reinterpret_cast<int64_t*>(s_tstart + RADIX);
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wsum[WARPS];
  __shared__ uint32_t s_next[RADIX];
  __shared__ uint64_t s_edge[2];  // first and last key of the tile
  __shared__ int s_shift;         // read back in step 4 (see there)

  if (next_hist)
    for (int k = threadIdx.x; k < RADIX; k += THREADS) s_next[k] = 0;
  if (threadIdx.x == 0) s_shift = shift;
  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  const uint32_t tile = tile_id(ctr, &s_tile);
  const int64_t tile_base = (int64_t)tile * TILE;
  if (tile_base >= n) return;
  const bool full = tile_base + TILE <= n;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t dmask = (1u << bits) - 1u;
  const int lbits = shift - lo;  // sorted bits below the digit
  const uint64_t lmask = lbits > 0 ? (~0ull >> (64 - lbits)) : 0ull;
  for (int k = threadIdx.x; k < SM::CNT; k += THREADS) s_cnt[k] = 0;

  // 1. load: warp w reads its contiguous 32*ITEMS keys item-major
  uint64_t key[ITEMS];
  const int64_t wbase = tile_base + (int64_t)warp * 32 * ITEMS;
  // keys of this warp that exist: items i*32 + lane below wn are valid
  const int wn = (int)max((int64_t)0, min((int64_t)32 * ITEMS, n - wbase));
  if (full) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) key[i] = __ldcs(in + wbase + i * 32 + lane);
    if (threadIdx.x == 0) s_edge[0] = key[0];
    if (threadIdx.x == THREADS - 1) s_edge[1] = key[ITEMS - 1];
  } else {
    const bool holds_last = wbase + wn == n;  // this warp's range ends the tile
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int p = i * 32 + (int)lane;
      key[i] = p < wn ? __ldcs(in + wbase + p) : 0ull;
      if (holds_last && p == wn - 1) s_edge[1] = key[i];
    }
    if (threadIdx.x == 0) s_edge[0] = key[0];
  }
  // DB: the digit's global start is read here, before the look-back, whose
  // ordered loads would otherwise hold it back until step 5 (one more
  // register through the pass; configurations short of registers read it in
  // step 5)
  const uint64_t dbase = DB && threadIdx.x < RADIX ? digit_base[threadIdx.x] : 0ull;
  __syncthreads();
  const uint64_t lf = (s_edge[0] >> lo) & lmask;
  const bool fast = ((s_edge[1] >> lo) & lmask) - lf < (uint64_t)OS_RUNS;  // block-uniform
  // HIW (lo >= 32): every sorted bit sits in the key's high word, so digits
  // and runs come from 32-bit shifts.  A run is the lower bits' difference
  // from the tile's first key, which modulo 2^32 is exact for the fast case's
  // differences below OS_RUNS.
  const uint32_t lmask32 = (uint32_t)lmask, lf32 = (uint32_t)lf;
  auto digit_of = [&](uint64_t k, int sh) -> uint32_t {
    if (HIW) return ((uint32_t)(k >> 32) >> (sh - 32)) & dmask;
    return (uint32_t)(k >> sh) & dmask;
  };
  // a run outside [0, OS_RUNS) means the input was not sorted on the lower
  // bits: clamped, and reported once per thread (`bad`) after the loop
  auto run_of = [&](uint64_t k, int at, uint32_t& bad) -> uint32_t {  // at: lo, or step 4's copy
    const uint32_t r = HIW ? (((uint32_t)(k >> 32) >> (at - 32)) & lmask32) - lf32
                           : (uint32_t)((k >> at) & lmask) - lf32;
    bad |= r >= (uint32_t)OS_RUNS;
    return min(r, (uint32_t)(OS_RUNS - 1));
  };

  // 2. counts: bins (run, digit) for the tile, or (warp, digit)
  if (fast) {
    uint32_t bad = 0;
    if (full) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        atomicAdd(&s_cnt[run_of(key[i], lo, bad) * RADIX + digit_of(key[i], shift)], 1u);
    } else {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        if (i * 32 + (int)lane < wn)
          atomicAdd(&s_cnt[run_of(key[i], lo, bad) * RADIX + digit_of(key[i], shift)], 1u);
    }
    if (bad) atomicOr(err, DERR_RANGE);
  } else {
    uint32_t* wc = s_cnt + warp * RADIX;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      if (full || i * 32 + (int)lane < wn) atomicAdd(&wc[digit_of(key[i], shift)], 1u);
  }
  __syncthreads();

  // 3. bin offsets within each digit, tile counts, aggregates for the look-back
  uint32_t tcount = 0;
  if (threadIdx.x < RADIX) {
    uint32_t acc = 0;
    if (fast) {
#pragma unroll
      for (int r = 0; r < OS_RUNS; ++r) {
        const uint32_t c = s_cnt[r * RADIX + threadIdx.x];
        s_cnt[r * RADIX + threadIdx.x] = acc;
        acc += c;
      }
    } else {
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_cnt[w * RADIX + threadIdx.x];
        s_cnt[w * RADIX + threadIdx.x] = acc;
        acc += c;
      }
    }
    tcount = acc;
    st_status(&status[(uint64_t)tile * RADIX + threadIdx.x], (tile == 0 ? ST_INC : ST_AGG) | acc);
  }
  {  // exclusive scan of the tile counts over digits
    const uint32_t v = tcount;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL_MASK, inc, o);
      if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (threadIdx.x < RADIX) {
      uint32_t off = 0;
      for (uint32_t w = 0; w < warp; ++w) off += s_wsum[w];
      const uint32_t ts = off + inc - v;
      s_tstart[threadIdx.x] = ts;
      const int slots = fast ? OS_RUNS : WARPS;
      for (int r = 0; r < slots; ++r) s_cnt[r * RADIX + threadIdx.x] += ts;
    }
    __syncthreads();
  }

  // 4. place the keys in shared memory in digit order.  The digit shift is
  // read back from shared memory so that the compiler recomputes every bin
  // here instead of keeping step 2's bins live across the barriers (ITEMS
  // more registers per thread).
  const int sh4 = s_shift;
  const int lo4 = sh4 - lbits;
  if (fast) {
    uint32_t bad = 0;
    auto place = [&](int i) {
      const uint32_t bin = run_of(key[i], lo4, bad) * RADIX + digit_of(key[i], sh4);
      const uint32_t pos = atomicAdd(&s_cnt[bin], 1u);
      bad |= pos >= (uint32_t)TILE;
      if (pos < (uint32_t)TILE) s_keys[pos] = key[i];
    };
    if (full) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) place(i);
    } else {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        if (i * 32 + (int)lane < wn) place(i);
    }
    if (bad) atomicOr(err, DERR_RANGE);
  } else {
    uint32_t* wc = s_cnt + warp * RADIX;
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = full || i * 32 + (int)lane < wn;
      const uint32_t dig = digit_of(key[i], sh4);
      const uint32_t vmask = full ? FULL_MASK : __ballot_sync(FULL_MASK, valid);
      const uint32_t peers = digit_peers<0>(dig, vmask);
      const uint32_t before = peers & lt_mask;
      const uint32_t base = valid ? wc[dig] : 0u;
      __syncwarp();
      if (valid && before == 0) wc[dig] = base + __popc(peers);
      __syncwarp();
      if (valid) {
        const uint32_t pos = base + __popc(before);
        if (pos < (uint32_t)TILE) s_keys[pos] = key[i];
        else atomicOr(err, DERR_RANGE);
      }
    }
  }

  // 5. look-back per digit
  if (threadIdx.x < RADIX) {
    uint64_t excl = 0;
    if (tile > 0) {
      excl = LBW > 1 ? thread_lookback_w<LBW>(status + threadIdx.x, tile, RADIX, err)
                     : thread_lookback(status + threadIdx.x, tile, RADIX, err);
      st_status(&status[(uint64_t)tile * RADIX + threadIdx.x], ST_INC | (excl + tcount));
    }
    s_obase[threadIdx.x] =
        (int64_t)((DB ? dbase : digit_base[threadIdx.x]) + excl) - (int64_t)s_tstart[threadIdx.x];
  }
  __syncthreads();

  // 6. write out in digit order (UW: a full tile's ITEMS keys per thread
  // unrolled); the per-key bucket marks of the slow case and the next pass's
  // digit counts in a loop of their own
  const bool mark_each = bucket_start && !fast;
  const int tile_n = full ? TILE : (int)(n - tile_base);
  uint32_t bad_out = 0;  // an output position out of range, reported once
  auto write_one = [&](int j, bool mark, bool count) {
    const uint64_t k = s_keys[j];
    const uint32_t dig = digit_of(k, shift);
    if (count) atomicAdd(&s_next[(uint32_t)(k >> (shift + 8)) & ((1u << next_bits) - 1u)], 1u);
    const int64_t o = s_obase[dig] + j;
    const bool in = o >= 0 && o < n;
    bad_out |= !in;
    if (in) out[o] = k;
    if (mark && in) {
      const uint64_t b = k >> lo;
      if (j == (int)s_tstart[dig] || b != (s_keys[j - 1] >> lo))
        atomicMin(&bucket_start[b], (unsigned long long)o);
    }
  };
  const bool count = next_hist != nullptr;
  if (mark_each || count) {
    for (int j = threadIdx.x; j < tile_n; j += THREADS) write_one(j, mark_each, count);
  } else if (UW && full) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) write_one((int)threadIdx.x + i * THREADS, false, false);
  } else {
    for (int j = threadIdx.x; j < tile_n; j += THREADS) write_one(j, false, false);
  }
  if (bad_out) atomicOr(err, DERR_RANGE);

  // 7. bucket starts of the fast case, after the write-out (which they do not
  // delay): digit t's runs sit at [start, end) of the tile, end being where
  // step 4 left the bin's counter
  if (bucket_start && fast && threadIdx.x < RADIX) {
    uint32_t start = s_tstart[threadIdx.x];
#pragma unroll
    for (int r = 0; r < OS_RUNS; ++r) {
      const uint32_t end = s_cnt[r * RADIX + threadIdx.x];
      if (end > start) {
        const int64_t o = s_obase[threadIdx.x] + start;
        const uint64_t b = ((uint64_t)threadIdx.x << lbits) | (lf + (uint64_t)r);
        if (o >= 0 && o < n && (b >> (lbits + bits)) == 0)
          atomicMin(&bucket_start[b], (unsigned long long)o);
      }
      start = end;
    }
  }

  if (next_hist) {  // uniform over the block
    __syncthreads();
    if (threadIdx.x < RADIX && s_next[threadIdx.x])
      atomicAdd(&next_hist[threadIdx.x], s_next[threadIdx.x]);
  }
  // clear this tile's status words (and tile counter) for the next pass,
  // which runs after this kernel with the same tiles: no memset between
  // passes.  Tiles past the key count leave early; the next pass's tiles
  // there leave early too and read no status.
  if (status_next && threadIdx.x < RADIX) {
    status_next[(uint64_t)tile * RADIX + threadIdx.x] = 0ull;
    if (tile == 0 && threadIdx.x == 0) *ctr_next = 0u;
  }
}

// Tile configurations (id, threads, items per thread, min blocks per SM,
// ranking: 0 ballots / 1 match.any / 2 atomic-OR bins / 3 ballots with one
// leader atomic per group / 4 unstable, one atomic per key, ranking chains).
// Both sorts use configuration 9 by default; the autotuner may pick others
// among 0-19.  Configuration 100 is unstable, only for the first pass of a
// sort, whose input order does not matter; its tile is that of the default 9
// (see onesweep_unstable_config).
#define XTN_ONESWEEP_CONFIGS(X) \
  X(0, 256, 16, 3, 0, 1)           \
  X(1, 256, 24, 2, 0, 1)           \
  X(2, 512, 12, 2, 0, 1)           \
  X(3, 256, 8, 4, 0, 1)            \
  X(4, 256, 16, 3, 1, 1)           \
  X(5, 256, 20, 3, 0, 1)           \
  X(6, 384, 16, 2, 0, 1)           \
  X(7, 256, 12, 4, 0, 1)           \
  X(8, 256, 16, 3, 2, 1)           \
  X(9, 256, 20, 3, 2, 1)           \
  X(10, 512, 16, 1, 2, 1)          \
  X(11, 256, 24, 2, 2, 1)          \
  X(12, 256, 20, 3, 2, 2)       \
  X(13, 256, 16, 3, 2, 2)       \
  X(14, 256, 20, 3, 0, 2)       \
  X(15, 256, 12, 4, 0, 2)       \
  X(16, 256, 20, 3, 3, 1)       \
  X(17, 256, 16, 3, 3, 1)       \
  X(18, 256, 24, 2, 3, 1)       \
  X(19, 512, 12, 2, 3, 1)       \
  X(100, 256, 20, 3, 4, 1)

// k_onesweep_runs configurations (id, threads, items per thread, min blocks
// per SM, look-back window, digit start read early, write-out unrolled); a
// sort with one of them uses it for every pass.
#define XTN_ONESWEEP_RUNS_CONFIGS(X) \
  X(20, 384, 16, 3, 8, 0, 1)         \
  X(21, 256, 20, 4, 8, 0, 0)         \
  X(22, 384, 18, 3, 8, 0, 1)         \
  X(23, 384, 18, 3, 8, 0, 0)         \
  X(24, 512, 12, 3, 8, 0, 0)         \
  X(25, 512, 16, 2, 8, 1, 0)         \
  X(26, 384, 16, 3, 8, 0, 0)         \
  X(27, 384, 16, 3, 16, 0, 1)        \
  X(28, 256, 20, 4, 8, 0, 1)         \
  X(29, 384, 16, 3, 4, 0, 1)

int onesweep_tile(int cfg) {
  switch (cfg) {
#define X(id, T, I, B, M, C) \
  case id: return T * I;
    XTN_ONESWEEP_CONFIGS(X)
#undef X
#define X(id, T, I, B, W, D, U) \
  case id: return T * I;
    XTN_ONESWEEP_RUNS_CONFIGS(X)
#undef X
  }
  return 0;
}

int onesweep_configs() { return 30; }  // the tunable ones, 0-29

// Configurations 0-19 rank stably in every pass, so their first pass (whose
// input order does not matter) takes the unstable configuration 100 with the
// same tile; a k_onesweep_runs configuration serves every pass itself.
int onesweep_unstable_config(int cfg) { return cfg >= 20 && cfg < 30 ? cfg : 100; }

static cudaError_t onesweep_launch(int cfg, const uint64_t* in, uint64_t* out, int64_t n,
                                   const uint64_t* n_dev, int shift, int bits, const uint64_t* digit_base,
                                   uint64_t* status, uint32_t* ctr, uint32_t* err,
                                   uint32_t* next_hist, int next_bits,
                                   unsigned long long* bucket_start, int bucket_shift,
                                   uint64_t* status_next, uint32_t* ctr_next, cudaStream_t s) {
  switch (cfg) {
#define X(id, T, I, B, M, C)                                                                  \
  case id: {                                                                                  \
    using SM = OnesweepSmem<T, I, M, C>;                                                      \
    static std::once_flag once;                                                               \
    std::call_once(once, [] {                                                                 \
      cudaFuncSetAttribute(k_onesweep<T, I, B, M, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           (int)SM::bytes);                                                   \
      cudaFuncSetAttribute(k_onesweep<T, I, B, M, C>,                                            \
                           cudaFuncAttributePreferredSharedMemoryCarveout, 100);              \
    });                                                                                       \
    /* one tile per block; with the count on the device, n is its capacity */                \
    const uint32_t tiles = div_up_u32(n, SM::TILE);                                           \
    k_onesweep<T, I, B, M, C><<<tiles, T, SM::bytes, s>>>(in, out, n_dev, n, shift, bits,        \
                                                          digit_base,                         \
                                                       status, ctr, err, next_hist,           \
                                                       next_bits, bucket_start,               \
                                                       bucket_shift);                         \
    return cudaGetLastError();                                                                \
  }
    XTN_ONESWEEP_CONFIGS(X)
#undef X
#define X(id, T, I, B, W, D, U)                                                               \
  case id: {                                                                                  \
    using SM = RunsSmem<T, I>;                                                                \
    static std::once_flag once;                                                               \
    std::call_once(once, [] {                                                                 \
      for (auto f : {k_onesweep_runs<T, I, B, W, D, U, false>,                                \
                     k_onesweep_runs<T, I, B, W, D, U, true>}) {                              \
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes); \
        cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);         \
      }                                                                                       \
    });                                                                                       \
    const uint32_t tiles = div_up_u32(n, SM::TILE);                                           \
    auto f = bucket_shift >= 32 ? k_onesweep_runs<T, I, B, W, D, U, true>                     \
                                : k_onesweep_runs<T, I, B, W, D, U, false>;                   \
    f<<<tiles, T, SM::bytes, s>>>(in, out, n_dev, n, shift, bits, bucket_shift, digit_base,  \
                                  status, ctr, err, next_hist, next_bits, bucket_start,      \
                                  status_next, ctr_next);                                    \
    return cudaGetLastError();                                                                \
  }
    XTN_ONESWEEP_RUNS_CONFIGS(X)
#undef X
  }
  return cudaErrorInvalidValue;
}

// One pass's status words and tile counter; a sort holds two, used by
// alternate passes.
static size_t status_region_bytes(int64_t n, int cfg) {
  const int64_t tiles = (n + onesweep_tile(cfg) - 1) / onesweep_tile(cfg);
  return (size_t)tiles * RADIX * 8 + 16;
}

size_t radix_status_bytes(int64_t n, int cfg) { return 2 * status_region_bytes(n, cfg); }

void launch_histogram(const uint64_t* keys, int64_t n, int lo, int hi, uint32_t* hist, int sms,
                      cudaStream_t s) {
  if (n <= 0) return;
  int blocks = (int)std::min<int64_t>((n + 1023) / 1024, (int64_t)sms * 4);
  prof_begin(s, "k_histogram", (double)n * 8.0);
  k_histogram<<<blocks, 512, 0, s>>>(keys, n, lo, hi, hist);
  prof_end(s);
}

cudaError_t radix_sort_passes(uint64_t* a, uint64_t* b, int64_t n, int lo, int hi, uint32_t* hist,
                              uint64_t* digit_base, uint64_t* status, int cfg, uint32_t* err,
                              uint64_t** sorted, const char* tag, cudaStream_t s,
                              bool hist_in_passes, const uint64_t* n_dev,
                              uint64_t* bucket_start, int first_cfg, bool status_zeroed) {
  const int passes = (hi - lo + 7) / 8;
  // buckets are key >> lo: the sorted bits must reach the top of the key
  if (bucket_start && hi != 64) return cudaErrorInvalidValue;
  // the status words are sized for cfg's tile
  if (first_cfg >= 0 && onesweep_tile(first_cfg) != onesweep_tile(cfg)) first_cfg = -1;
  *sorted = a;
  if (n <= 1 || passes == 0) return cudaSuccess;
  // hist_in_passes: `hist` holds pass 0's counts on entry, pass p counts the
  // digits of pass p+1 into hist[(p+1) * RADIX], and each pass's offsets are
  // scanned just before it runs.
  if (!hist_in_passes) {
    prof_begin(s, "k_digit_scan", (double)passes * RADIX * 12.0);
    k_digit_scan<<<passes, RADIX, 0, s>>>(hist, digit_base);
    prof_end(s);
  }
  // two status regions for alternate passes; k_onesweep_runs clears the next
  // pass's region as it goes, so only the first is cleared here
  const size_t region = status_region_bytes(n, cfg);
  uint64_t* st[2] = {status, reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(status) + region)};
  auto ctr_of = [&](uint64_t* r) {
    return reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(r) + region - 16);
  };
  const bool clears_next = onesweep_unstable_config(cfg) == cfg;  // a k_onesweep_runs config
  uint64_t* src = a;
  uint64_t* dst = b;
  for (int p = 0; p < passes; ++p) {
    const int sh = lo + 8 * p;
    const int bits = std::min(8, hi - sh);
    if (hist_in_passes) {
      prof_begin(s, "k_digit_scan", (double)RADIX * 12.0);
      k_digit_scan<<<1, RADIX, 0, s>>>(hist + p * RADIX, digit_base + p * RADIX);
      prof_end(s);
    }
    uint32_t* next = (hist_in_passes && p + 1 < passes) ? hist + (p + 1) * RADIX : nullptr;
    const int next_bits = next ? std::min(8, hi - (sh + 8)) : 0;
    // a region is fresh for the first two passes when the caller cleared both;
    // later passes reuse one, cleared by the pass before (or by a memset)
    uint64_t* cur = st[p & 1];
    const bool fresh_next = status_zeroed && p + 1 < 2;
    uint64_t* nxt = clears_next && p + 1 < passes && !fresh_next ? st[(p + 1) & 1] : nullptr;
    cudaError_t e = cudaSuccess;
    const bool fresh = status_zeroed && p < 2;
    if (!fresh && (!clears_next || p == 0)) e = cudaMemsetAsync(cur, 0, region, s);
    if (e != cudaSuccess) return e;
    prof_begin(s, tag, (double)n * 16.0);
    unsigned long long* bs =
        p + 1 == passes ? reinterpret_cast<unsigned long long*>(bucket_start) : nullptr;
    e = onesweep_launch(p == 0 && first_cfg >= 0 ? first_cfg : cfg, src, dst, n, n_dev, sh, bits,
                        digit_base + p * RADIX, cur, ctr_of(cur), err,
                        next, next_bits, bs, lo, nxt, nxt ? ctr_of(nxt) : nullptr, s);
    prof_end(s);
    if (e != cudaSuccess) return e;
    std::swap(src, dst);
  }
  *sorted = src;
  return cudaSuccess;
}

}  // namespace xtn
