// Grouping of variant records by their full group key, with the candidate
// pairs written at once (Appendix A, XTNeighbor steps 4-5), for the buckets
// left by the global radix passes on the top G key bits.
//
// Nearly every variant record shares its group key with no other record, so
// the exact grouping only needs the few that do.  k_bucket_filter is a
// persistent kernel: each block takes segments (2^kbits consecutive buckets,
// contiguous in the sorted records) in turn and, while it works on one, the
// next one's records arrive in shared memory by a bulk asynchronous copy.
// For a segment it
//   1. marks, in two bitmaps indexed by the composite key (bucket offset in
//      the segment above the low L key bits; hashed to 16 bits when wider),
//      the keys seen and the keys seen again;
//   2. keeps the records whose key was seen again -- all members of groups
//      of two or more, plus the rare lone record whose bit another key also
//      hit -- in a short list;
//   3. groups the list exactly in a small hash table keyed by the composite
//      key, places each group's ids contiguously, and writes every pair of a
//      group of two or more as a candidate word (min id << id_bits | max id),
//      reserving output space once per warp.
// A segment with more records than a buffer holds, or whose list overflows,
// is flagged instead; k_bucket then groups the flagged segments as before.
#include <algorithm>
#include <mutex>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

namespace {

constexpr int BF_THREADS = 256;
constexpr int BF_WARPS = BF_THREADS / 32;
constexpr int BF_CAP = 2048;   // records of one segment held at once
constexpr int BF_LIST = 1024;  // records the filter may keep
constexpr int BF_HB = 11;      // log2 of the exact grouping's hash slots
constexpr int BF_H = 1 << BF_HB;
constexpr int BF_BITS = 16;    // log2 of the bits of each filter bitmap
constexpr int BF_WORDS = (1 << BF_BITS) / 32;
constexpr uint32_t BF_EMPTY = 0xffffffffu;
constexpr uint16_t BF_NO_PLACE = 0xffffu;
static_assert(BF_H >= 2 * BF_LIST, "hash load factor <= 1/2");
static_assert(BF_THREADS * 8 == BF_H, "eight hash slots per thread in the slot scan");

struct BfSmem {
  uint64_t buf[2][BF_CAP + 2];  // segments; a bulk copy starts at an even record
  uint32_t seen[BF_WORDS];
  uint32_t again[BF_WORDS];
  uint64_t list[BF_LIST];
  uint32_t tk[BF_H];            // composite keys, then group sizes
  uint32_t tc[BF_H / 2];        // u16 counts, then u16 starts, two per word
  uint32_t ids[BF_LIST];
  uint64_t bar[2];
  int64_t rng[2][2];            // [s, e) of the segment in each buffer
  uint32_t seg[2];
  uint32_t mode[2];             // 0 nothing to load, 1 bulk copy, 2 thread loads
  uint32_t off[2];              // first record's index in the buffer
  uint32_t nlist;
  uint32_t wsum[BF_WARPS];
};

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


__global__ void __launch_bounds__(BF_THREADS, 3)
    k_bucket_filter(const uint64_t* __restrict__ A, int64_t n_cap,
                    const uint64_t* __restrict__ n_dev,
                    const unsigned long long* __restrict__ bucket_start, int G, int kbits, int lo,
                    int L, uint64_t* __restrict__ cand, uint64_t cand_cap,
                    unsigned long long* __restrict__ cand_count, int id_bits,
                    uint8_t* __restrict__ seg_flags, uint32_t* __restrict__ seg_ctr,
                    uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BfSmem& S = *reinterpret_cast<BfSmem*>(smem_raw);
  const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
  const int64_t nb = 1ll << G;
  const int64_t K = 1ll << kbits;
  const uint32_t n_seg = (uint32_t)(nb >> kbits);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t limit = spin_limit(err);
  const bool bulk_ok = (reinterpret_cast<uintptr_t>(A) & 15u) == 0;
  const bool direct = L + kbits <= BF_BITS;
  const uint64_t idmask = (1ull << id_bits) - 1ull;

  // warp 0: take the next segment, find its records [s, e) and start their
  // load into buffer b (a bulk copy from an even record when it may read up
  // to an even end inside the valid records, else thread loads later)
  auto take = [&](int b) {
    uint32_t seg = 0;
    if (lane == 0) seg = atomicAdd(seg_ctr, 1u);
    seg = __shfl_sync(FULL_MASK, seg, 0);
    int64_t s = n, e = n;
    if (seg < n_seg) {
      const int64_t b0 = (int64_t)seg * K;
      if (G > 0) {
        s = bf_first_start(bucket_start, b0, nb, n, lane);
        e = b0 + K >= nb ? n : bf_first_start(bucket_start, b0 + K, nb, n, lane);
        if (e < s) e = s;
      } else {
        s = 0;
        e = n;
      }
    }
    if (lane == 0) {
      uint32_t mode = 0, off = 0;
      const int64_t m = e - s;
      if (seg < n_seg && m > 0 && m <= BF_CAP) {
        const int64_t s0 = s & ~1ll, e0 = (e + 1) & ~1ll;
        if (bulk_ok && e0 <= n) {
          mode = 1;
          off = (uint32_t)(s - s0);
          const uint32_t bytes = (uint32_t)((e0 - s0) * 8);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(&S.bar[b], bytes);
          bulk_load(S.buf[b], A + s0, bytes, &S.bar[b]);
        } else {
          mode = 2;
        }
      }
      S.seg[b] = seg;
      S.rng[b][0] = s;
      S.rng[b][1] = e;
      S.mode[b] = mode;
      S.off[b] = off;
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < 2 * BF_WORDS / 4; k += BF_THREADS)
    reinterpret_cast<uint4*>(S.seen)[k] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  if (warp == 0) take(0);
  __syncthreads();
  uint32_t phase = 0;  // bit b: parity of buffer b's next bulk completion
  for (int it = 0;; ++it) {
    const int b = it & 1;
    const uint32_t seg = S.seg[b];
    if (seg >= n_seg) break;  // block-uniform
    const int64_t s = S.rng[b][0], e = S.rng[b][1];
    const int m = (int)(e - s);
    const uint32_t mode = S.mode[b];
    const uint64_t* buf = S.buf[b] + S.off[b];
    // the next segment's load runs while this one is worked on (its buffer
    // was last read before the barrier that ended the previous iteration)
    if (warp == 0) take(b ^ 1);
    if (mode == 0) {  // empty, or more records than a buffer: k_bucket's
      if (m > 0 && threadIdx.x == 0) seg_flags[seg] = 1;
      __syncthreads();
      continue;
    }
    if (mode == 1) {
      uint32_t spins = 0;
      while (!mbar_try_wait(&S.bar[b], (phase >> b) & 1u)) {
        if (++spins > limit) {  // give up: flag it, wait (bounded) for the copy
          if (threadIdx.x == 0) atomicOr(err, DERR_TIMEOUT);
          for (uint32_t w = 0; w < limit && !mbar_try_wait(&S.bar[b], (phase >> b) & 1u); ++w) {
          }
          break;
        }
      }
      phase ^= 1u << b;
    } else {
      for (int j = threadIdx.x; j < m; j += BF_THREADS) S.buf[b][j] = A[s + j];
      __syncthreads();
    }
    const uint64_t cbase = ((uint64_t)seg * (uint64_t)K) << L;
    auto comp = [&](uint64_t key) { return (uint32_t)((key >> lo) - cbase); };
    auto bit_of = [&](uint32_t c) {
      return (direct ? c : (c * 0x9E3779B1u) >> (32 - BF_BITS)) & ((1u << BF_BITS) - 1u);
    };
    // 1. mark keys seen and seen again
    for (int j = threadIdx.x; j < m; j += BF_THREADS) {
      const uint32_t h = bit_of(comp(buf[j])), bit = 1u << (h & 31u);
      if (atomicOr(&S.seen[h >> 5], bit) & bit) atomicOr(&S.again[h >> 5], bit);
    }
    if (threadIdx.x == 0) S.nlist = 0;
    __syncthreads();
    // 2. keep the records whose key was seen again
    for (int j0 = (int)warp * 32; j0 < m; j0 += BF_THREADS) {
      const int j = j0 + (int)lane;
      bool keep = false;
      uint64_t key = 0;
      if (j < m) {
        key = buf[j];
        const uint32_t h = bit_of(comp(key));
        keep = (S.again[h >> 5] >> (h & 31u)) & 1u;
      }
      const uint32_t bal = __ballot_sync(FULL_MASK, keep);
      uint32_t at = 0;
      if (lane == 0 && bal) at = atomicAdd(&S.nlist, (uint32_t)__popc(bal));
      at = __shfl_sync(FULL_MASK, at, 0) + (uint32_t)__popc(bal & lt_mask);
      if (keep && at < (uint32_t)BF_LIST) S.list[at] = key;
    }
    __syncthreads();
    const uint32_t kept = S.nlist;
    // bitmaps back to zero for the next segment
    for (int k = threadIdx.x; k < 2 * BF_WORDS / 4; k += BF_THREADS)
      reinterpret_cast<uint4*>(S.seen)[k] = make_uint4(0u, 0u, 0u, 0u);
    if (kept > (uint32_t)BF_LIST || kept < 2) {
      if (kept > (uint32_t)BF_LIST && threadIdx.x == 0) seg_flags[seg] = 1;
      __syncthreads();
      continue;
    }
    // 3. exact grouping of the kept records in a table of 2^hb >= 2 kept slots
    int hb = 6;
    while ((1u << hb) < 2 * kept) ++hb;
    const uint32_t H = 1u << hb;  // <= BF_H
    for (uint32_t k = threadIdx.x; k < H / 4; k += BF_THREADS)
      reinterpret_cast<uint4*>(S.tk)[k] = make_uint4(BF_EMPTY, BF_EMPTY, BF_EMPTY, BF_EMPTY);
    for (uint32_t k = threadIdx.x; k < H / 8; k += BF_THREADS)
      reinterpret_cast<uint4*>(S.tc)[k] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    constexpr int PT = BF_LIST / BF_THREADS;  // kept records per thread, at most
    uint32_t sr[PT];                          // slot << 16 | rank in the slot's group
#pragma unroll
    for (int i = 0; i < PT; ++i) {
      const uint32_t j = threadIdx.x + (uint32_t)i * BF_THREADS;
      sr[i] = 0xffffffffu;
      if (j < kept) {
        const uint32_t c = comp(S.list[j]);
        uint32_t h = (c * 0x9E3779B1u) >> (32 - hb);
        bool found = false;
        for (uint32_t probe = 0; probe < H; ++probe) {  // at most kept <= H/2 keys: ends
          const uint32_t old = atomicCAS(&S.tk[h], BF_EMPTY, c);
          if (old == BF_EMPTY || old == c) {
            found = true;
            break;
          }
          h = (h + 1) & (H - 1);
        }
        if (found) {
          const uint32_t sh = (h & 1u) * 16;
          sr[i] = (h << 16) | ((atomicAdd(&S.tc[h >> 1], 1u << sh) >> sh) & 0xffffu);
        } else {
          atomicOr(err, DERR_RANGE);
        }
      }
    }
    __syncthreads();
    // slot scan: thread t owns slots 8t .. 8t+7 (those below H); only groups
    // of two or more are placed, their sizes go to the key table
    uint32_t w4[4];
    uint32_t tot = 0;
    const bool owner = 8u * threadIdx.x < H;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      w4[q] = owner ? S.tc[4 * threadIdx.x + q] : 0u;
      const uint32_t a = w4[q] & 0xffffu, c2 = w4[q] >> 16;
      tot += (a >= 2 ? a : 0u) + (c2 >= 2 ? c2 : 0u);
    }
    // block-wide exclusive scan of tot
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL_MASK, inc, o);
      if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) S.wsum[warp] = inc;
    __syncthreads();
    uint32_t run = inc - tot;
    for (uint32_t w = 0; w < warp; ++w) run += S.wsum[w];
    uint32_t gmask = 0, np = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t a = w4[q] & 0xffffu, c2 = w4[q] >> 16;
      const uint32_t h = 8u * threadIdx.x + 2u * q;
      const uint32_t sa = a >= 2 ? run : BF_NO_PLACE;
      run += a >= 2 ? a : 0u;
      const uint32_t sb = c2 >= 2 ? run : BF_NO_PLACE;
      run += c2 >= 2 ? c2 : 0u;
      if (owner) {
        S.tc[4 * threadIdx.x + q] = sa | (sb << 16);
        if (a >= 2) S.tk[h] = a;
        if (c2 >= 2) S.tk[h + 1] = c2;
      }
      if (a >= 2) {
        gmask |= 1u << (2 * q);
        np += a * (a - 1) / 2;
      }
      if (c2 >= 2) {
        gmask |= 2u << (2 * q);
        np += c2 * (c2 - 1) / 2;
      }
    }
    // output room of this warp's groups, reserved once
    uint32_t wp = np;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wp += __shfl_xor_sync(FULL_MASK, wp, o);
    unsigned long long obase = 0;
    if (lane == 0 && wp) {
      obase = atomicAdd(cand_count, (unsigned long long)wp);
      if (obase + wp > cand_cap) atomicOr(err, DERR_CAPACITY);
    }
    obase = __shfl_sync(FULL_MASK, obase, 0);
    __syncthreads();
    // 4. each group's ids, contiguous
#pragma unroll
    for (int i = 0; i < PT; ++i) {
      if (sr[i] != 0xffffffffu) {
        const uint32_t h = sr[i] >> 16;
        const uint32_t start = (S.tc[h >> 1] >> ((h & 1u) * 16)) & 0xffffu;
        if (start != BF_NO_PLACE) {
          const uint32_t pos = start + (sr[i] & 0xffffu);
          const uint32_t j = threadIdx.x + (uint32_t)i * BF_THREADS;
          if (pos < kept) S.ids[pos] = (uint32_t)(S.list[j] & idmask);
          else atomicOr(err, DERR_RANGE);
        }
      }
    }
    __syncthreads();
    // 5. every pair of every group of two or more, the warp spreading each
    // group's pairs over its lanes (colex rank l = b (b - 1) / 2 + a, a < b)
    while (__any_sync(FULL_MASK, gmask != 0)) {
      uint32_t st = 0, c = 0;
      if (gmask) {
        const uint32_t h = 8u * threadIdx.x + (uint32_t)(__ffs(gmask) - 1);
        gmask &= gmask - 1;
        st = (S.tc[h >> 1] >> ((h & 1u) * 16)) & 0xffffu;
        c = S.tk[h];
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
          if (gst + bb < (uint32_t)BF_LIST) {
            const uint64_t ia = S.ids[gst + aa], ib = S.ids[gst + bb];
            if (obase + l < cand_cap)
              cand[obase + l] = ((ia < ib ? ia : ib) << id_bits) | (ia < ib ? ib : ia);
          }
        }
        obase += pairs;
      }
    }
    __syncthreads();  // the list, ids and tables are reused by the next segment
  }
}

}  // namespace

size_t bucket_filter_smem() { return sizeof(BfSmem); }

void launch_bucket_filter(const uint64_t* A, int64_t n, const uint64_t* n_dev,
                          const uint64_t* bucket_start, const GroupingShape& g, int lo,
                          uint64_t* cand, uint64_t cand_cap, uint64_t* cand_count, int id_bits,
                          uint8_t* seg_flags, uint32_t* seg_ctr, int sms, uint32_t* err,
                          cudaStream_t s) {
  if (n <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_bucket_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(BfSmem));
    cudaFuncSetAttribute(k_bucket_filter, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
  const uint64_t n_seg = ((uint64_t)1 << g.G) >> g.kbits;
  const uint32_t blocks = (uint32_t)std::min<uint64_t>(n_seg, (uint64_t)sms * 3);
  prof_begin(s, "k_bucket_filter", (double)n * 8.0);
  k_bucket_filter<<<blocks, BF_THREADS, sizeof(BfSmem), s>>>(
      A, n, n_dev, reinterpret_cast<const unsigned long long*>(bucket_start), g.G, g.kbits, lo,
      g.L, cand, cand_cap, reinterpret_cast<unsigned long long*>(cand_count), id_bits, seg_flags,
      seg_ctr, err);
  prof_end(s);
}

}  // namespace xtn
