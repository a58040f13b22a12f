// Shared helpers of the sm_103a kernels: device status words for single-pass
// (decoupled look-back) prefix sums with bounded waits, error flags, the
// packed 5-bit residue representation, and the host-side launch bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xtn.h"

namespace xtn {

constexpr uint32_t FULL_MASK = 0xffffffffu;

// ---------------------------------------------------------------- errors ---
// Device error word bits (or-ed by kernels, read once by the host).
enum : uint32_t {
  DERR_BAD_RESIDUE = 1u << 0,
  DERR_TOO_LONG = 1u << 1,
  DERR_TIMEOUT = 1u << 2,
  DERR_RANGE = 1u << 3,   // an index outside the caller's sequence range
  DERR_CAPACITY = 1u << 4,  // more candidate pairs than a planned capacity
};

// A spin on a predecessor's status word gives up after this many polls
// (each poll sleeps ~0.25-1 us), sets DERR_TIMEOUT and carries on, so a kernel
// never waits without bound.  The error word array (4 words, zeroed by the
// host before a call's first kernel) carries an override in its second word:
// a non-zero err[1] replaces this limit (xtn_set_wait_limit).
constexpr uint32_t SPIN_LIMIT = 1u << 20;

__device__ __forceinline__ uint32_t spin_limit(const uint32_t* err) {
  const uint32_t v = err[1];
  return v ? v : SPIN_LIMIT;
}

// ----------------------------------------------------------- status words ---
// Tile status for decoupled look-back: 2 flag bits + 62 value bits in one
// 64-bit word, written and read whole so flag and value are seen together.
constexpr uint64_t ST_AGG = 1ull << 62;  // value = this tile's aggregate
constexpr uint64_t ST_INC = 2ull << 62;  // value = inclusive prefix through this tile
constexpr uint64_t ST_VAL = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t ld_status(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_status(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(FULL_MASK, v, o);
    if (lane >= (uint32_t)o) v += t;
  }
  return v;
}

// Decoupled look-back over one counter per tile, run by all 32 lanes of one
// warp: publishes `agg` for `tile`, sums the predecessors' values (a window of
// 32 tiles per step, stopping at the nearest inclusive prefix), publishes the
// inclusive prefix and returns the exclusive one (same value in all lanes).
// Tiles must be numbered in the order their blocks started (see tile_id), so
// every predecessor is resident or done and the wait ends.
__device__ __forceinline__ uint64_t warp_lookback(uint64_t* status, uint32_t tile, uint64_t agg,
                                                  uint32_t* err) {
  const uint32_t lane = lane_id();
  if (lane == 0) st_status(&status[tile], (tile == 0 ? ST_INC : ST_AGG) | agg);
  if (tile == 0) return 0;
  uint64_t excl = 0;
  int64_t top = (int64_t)tile - 1;
  uint32_t spins = 0;
  const uint32_t limit = spin_limit(err);
  while (true) {
    const int64_t idx = top - (int64_t)lane;
    const uint64_t w = idx >= 0 ? ld_status(&status[idx]) : (ST_INC | 0);
    const uint32_t flag = (uint32_t)(w >> 62);
    const uint32_t inc = __ballot_sync(FULL_MASK, flag == 2);
    const uint32_t not_ready = __ballot_sync(FULL_MASK, flag == 0);
    const uint32_t first_inc = inc ? (uint32_t)(__ffs(inc) - 1) : 32u;
    const uint32_t needed = first_inc >= 31 ? FULL_MASK : ((2u << first_inc) - 1u);
    if (not_ready & needed) {
      if (++spins > limit) {
        if (lane == 0) atomicOr(err, DERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
      continue;
    }
    excl += warp_sum_u64(lane <= first_inc ? (w & ST_VAL) : 0);
    if (first_inc < 32) break;
    top -= 32;
  }
  if (lane == 0) st_status(&status[tile], ST_INC | (excl + agg));
  return excl;
}

// Serial look-back of one counter chain (one thread per chain, as used per
// radix digit): sums predecessors of `tile` in the chain with stride `stride`.
__device__ __forceinline__ uint64_t thread_lookback(const uint64_t* status, uint32_t tile,
                                                    uint32_t stride, uint32_t* err) {
  uint64_t excl = 0;
  int64_t j = (int64_t)tile - 1;
  uint32_t spins = 0;
  const uint32_t limit = spin_limit(err);
  while (j >= 0) {
    const uint64_t w = ld_status(&status[(uint64_t)j * stride]);
    const uint64_t flag = w >> 62;
    if (flag == 0) {
      if (++spins > limit) {
        atomicOr(err, DERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
      continue;
    }
    excl += w & ST_VAL;
    if (flag == 2) break;
    --j;
  }
  return excl;
}

// The same look-back reading W predecessors per step (their loads in flight
// together), so a walk back over many tiles that have only published their
// aggregates takes 1/W of the dependent loads.  Statuses past the first
// unpublished tile of a window are not used; that tile is polled again.
template <int W>
__device__ __forceinline__ uint64_t thread_lookback_w(const uint64_t* status, uint32_t tile,
                                                      uint32_t stride, uint32_t* err) {
  uint64_t excl = 0;
  int64_t j = (int64_t)tile - 1;
  uint32_t spins = 0;
  const uint32_t limit = spin_limit(err);
  while (j >= 0) {
    uint64_t w[W];
#pragma unroll
    for (int k = 0; k < W; ++k)
      w[k] = j - k >= 0 ? ld_status(&status[(uint64_t)(j - k) * stride]) : (ST_INC | 0);
    int used = 0;
    bool done = false;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      if (done || used < k) break;  // stopped earlier in this window
      const uint64_t flag = w[k] >> 62;
      if (flag == 0) break;  // not published yet
      excl += w[k] & ST_VAL;
      used = k + 1;
      if (flag == 2) done = true;
    }
    if (done) break;
    j -= used;
    if (used == 0) {
      if (++spins > limit) {
        atomicOr(err, DERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
  }
  return excl;
}

// Tile number in block start order: the counter at `ctr` starts at zero.
__device__ __forceinline__ uint32_t tile_id(uint32_t* ctr, uint32_t* s_slot) {
  if (threadIdx.x == 0) *s_slot = atomicAdd(ctr, 1u);
  __syncthreads();
  return *s_slot;
}

// ------------------------------------------------- bulk copies, mbarriers ---
// One-dimensional bulk asynchronous copies (global -> this block's shared
// memory) whose completion is counted on an mbarrier in shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global memory into this block's shared memory, counted on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ------------------------------------------------------ packed sequences ---
// A sequence of length L <= 25 is a 128-bit integer (lo, hi): residue p sits
// at bits [5p, 5p+5) with codes 1..20 (alphabetical one-letter order), zero
// padding above 5L.  Distinct sequences give distinct keys; the length is the
// number of non-zero fields.
struct Key128 {
  uint64_t lo, hi;
};

// Residue code at position p (0 <= p < 25).
__device__ __forceinline__ uint32_t code_at(const Key128& k, int p) {
  const int m = 5 * p;
  uint64_t v;
  if (m < 64) {
    v = k.lo >> m;
    if (m > 59) v |= k.hi << (64 - m);
  } else {
    v = k.hi >> (m - 64);
  }
  return (uint32_t)(v & 31u);
}

// ------------------------------------------------------- fingerprints ---
// A residue string s_0..s_{L-1} (codes 1..20) is fingerprinted through the
// polynomial H(s) = sum_k s_k B^k mod 2^64 (B odd, so B is invertible mod
// 2^64), finished by mix64, a bijection that spreads every input bit over the
// top bits used for grouping.
// With prefix sums P[x] = sum_{k<x} s_k B^k, deleting positions
// p1 < p2 < p3 gives
//   H = P[p1] + (P[p2] - P[p1+1]) B^-1 + (P[p3] - P[p2+1]) B^-2 + (P[L] - P[p3+1]) B^-3,
// (fewer deletions: the missing positions are L, L+1, L+2 and P[x] = P[L]
// for x >= L), so a variant costs four table reads and three multiplies.
// Equal strings give equal fingerprints whatever they were derived from, so
// grouping by fingerprint finds every shared variant; unequal strings that
// collide only add candidate pairs, which the exact distance check removes.
constexpr uint64_t HASH_B = 0x9E3779B97F4A7C15ull;

__host__ __device__ constexpr uint64_t inverse_mod_2_64(uint64_t b) {
  uint64_t x = b;  // Newton iteration x <- x (2 - b x) doubles the valid low bits
  for (int i = 0; i < 6; ++i) x *= 2ull - b * x;
  return x;
}
constexpr uint64_t HASH_BINV = inverse_mod_2_64(HASH_B);
constexpr uint64_t HASH_BINV2 = HASH_BINV * HASH_BINV;
constexpr uint64_t HASH_BINV3 = HASH_BINV2 * HASH_BINV;
static_assert(HASH_B * HASH_BINV == 1ull, "B must be invertible mod 2^64");

// Xorshift-multiply-xorshift finaliser (a bijection on 64 bits).  The raw
// polynomial's top bits are far from uniform on residue strings; after this
// step the top-32-bit collision rate of real variant strings matches the
// ideal rate.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t h) {
  h ^= h >> 32;
  h *= 0xD6E8FEB86659FD93ull;
  h ^= h >> 32;
  return h;
}

__host__ __device__ __forceinline__ uint64_t rep_salt(uint64_t rep) {
  return rep == 0 ? 0ull : (rep * 0xA24BAED4963EE407ull) | 1ull;
}

// C(n, k) for the small n (<= 25) and k (<= 3) used here.
__host__ __device__ __forceinline__ uint32_t binom_small(uint32_t n, uint32_t k) {
  if (k > n) return 0;
  switch (k) {
    case 0: return 1;
    case 1: return n;
    case 2: return n * (n - 1) / 2;
    case 3: return n * (n - 1) * (n - 2) / 6;
    default: return 0;
  }
}

// Number of deletion positions subsets with at most d elements.
__host__ __device__ __forceinline__ uint32_t variant_count(uint32_t L, uint32_t d) {
  uint32_t c = 0;
  for (uint32_t k = 0; k <= d && k <= L; ++k) c += binom_small(L, k);
  return c;
}

// Deletion subsets of the positions {0..L-1} with at most d elements, ranked
// v = 0 (empty set), then every single position, every pair, every triple;
// each size in colexicographic order ({p<q} has rank C(q,2)+p among pairs,
// {p<q<r} has rank C(r,3)+C(q,2)+p among triples).  sum_{k<=d} C(L,k)
// subsets in all (variant_count).
struct Subset {
  uint32_t k, p, q, r;  // size and positions (p < q < r, unused ones 0)
};

__device__ __forceinline__ Subset unrank_subset(uint32_t L, uint32_t v) {
  Subset s{0u, 0u, 0u, 0u};
  if (v == 0) return s;
  if (v <= L) {
    s.k = 1;
    s.p = v - 1;
    return s;
  }
  uint32_t t = v - 1 - L;
  const uint32_t c2 = L * (L - 1) / 2;
  if (t < c2) {
    uint32_t q = (uint32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
    while (q * (q - 1) / 2 > t) --q;
    while ((q + 1) * q / 2 <= t) ++q;
    s.k = 2;
    s.q = q;
    s.p = t - q * (q - 1) / 2;
    return s;
  }
  t -= c2;
  uint32_t r = 2;
  while (binom_small(r + 1, 3) <= t) ++r;
  t -= binom_small(r, 3);
  uint32_t q = 1;
  while (binom_small(q + 1, 2) <= t) ++q;
  t -= binom_small(q, 2);
  s.k = 3;
  s.r = r;
  s.q = q;
  s.p = t;
  return s;
}

__device__ __forceinline__ uint32_t subset_mask(const Subset& s) {
  uint32_t m = 0;
  if (s.k >= 1) m |= 1u << s.p;
  if (s.k >= 2) m |= 1u << s.q;
  if (s.k >= 3) m |= 1u << s.r;
  return m;
}

// Within a run of equal residues, deleting any c of its positions leaves the
// same string, so only the leftmost-c choice is kept: a subset is canonical
// when every deleted position p whose left neighbour holds the same residue
// (bit p of `eqprev`) has that neighbour deleted too.  Every deletion variant
// string still arises from exactly one canonical subset per run pattern.
__device__ __forceinline__ bool is_canonical(uint32_t mask, uint32_t eqprev) {
  return (eqprev & mask & ~(mask << 1)) == 0;
}

// Number of canonical subsets with at most d elements: a canonical subset
// deletes a prefix of c_i positions from each run i, so the count is the sum
// of the coefficients of x^0..x^d in prod_i (1 + x + ... + x^{len_i}).
__host__ __device__ __forceinline__ uint32_t canonical_count(uint32_t eqprev, uint32_t L,
                                                             uint32_t d) {
  uint32_t poly[4] = {1u, 0u, 0u, 0u};
  uint32_t p = 0;
  while (p < L) {
    uint32_t run = 1;
    while (p + run < L && ((eqprev >> (p + run)) & 1u)) ++run;
    uint32_t next[4] = {0u, 0u, 0u, 0u};
    for (uint32_t k = 0; k <= d; ++k)
      for (uint32_t c = 0; c <= k && c <= run; ++c) next[k] += poly[k - c];
    for (uint32_t k = 0; k <= d; ++k) poly[k] = next[k];
    p += run;
  }
  uint32_t total = 0;
  for (uint32_t k = 0; k <= d; ++k) total += poly[k];
  return total;
}

// ------------------------------------------------------------ host side ---
// Launch bookkeeping: optional CUDA-event timing per kernel (see
// xtn_profile_enable), tagged with algorithmic bytes.
void prof_begin(cudaStream_t s, const char* name, double bytes);
void prof_end(cudaStream_t s);

inline uint32_t div_up_u32(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

}  // namespace xtn
