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
};

// A spin on a predecessor's status word gives up after this many polls
// (each poll sleeps ~0.25-1 us), sets DERR_TIMEOUT and carries on, so a kernel
// never waits without bound.
constexpr uint32_t SPIN_LIMIT = 1u << 20;

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
  while (true) {
    const int64_t idx = top - (int64_t)lane;
    const uint64_t w = idx >= 0 ? ld_status(&status[idx]) : (ST_INC | 0);
    const uint32_t flag = (uint32_t)(w >> 62);
    const uint32_t inc = __ballot_sync(FULL_MASK, flag == 2);
    const uint32_t not_ready = __ballot_sync(FULL_MASK, flag == 0);
    const uint32_t first_inc = inc ? (uint32_t)(__ffs(inc) - 1) : 32u;
    const uint32_t needed = first_inc >= 31 ? FULL_MASK : ((2u << first_inc) - 1u);
    if (not_ready & needed) {
      if (++spins > SPIN_LIMIT) {
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
  while (j >= 0) {
    const uint64_t w = ld_status(&status[(uint64_t)j * stride]);
    const uint64_t flag = w >> 62;
    if (flag == 0) {
      if (++spins > SPIN_LIMIT) {
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

// Tile number in block start order: the counter at `ctr` starts at zero.
__device__ __forceinline__ uint32_t tile_id(uint32_t* ctr, uint32_t* s_slot) {
  if (threadIdx.x == 0) *s_slot = atomicAdd(ctr, 1u);
  __syncthreads();
  return *s_slot;
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

// Delete residue p: residues above p move down one field.
__device__ __forceinline__ Key128 delete_at(const Key128& k, int p) {
  const int m = 5 * p;
  const uint64_t sh_lo = (k.lo >> 5) | (k.hi << 59);
  const uint64_t sh_hi = k.hi >> 5;
  Key128 r;
  if (m < 64) {
    const uint64_t low = m == 0 ? 0ull : ((1ull << m) - 1ull);
    r.lo = (k.lo & low) | (sh_lo & ~low);
    r.hi = sh_hi;
  } else {
    const uint64_t low = m == 64 ? 0ull : ((1ull << (m - 64)) - 1ull);
    r.lo = k.lo;
    r.hi = (k.hi & low) | (sh_hi & ~low);
  }
  return r;
}

// 64-bit fingerprint of a packed variant.  Equal variants give equal
// fingerprints, so grouping by fingerprint finds every shared variant; the
// rare unequal variants that collide only add candidate pairs, which the
// exact distance check removes.  `salt` separates repertoires.
// Mixing: odd-constant multiplies of both halves, then the SplitMix64
// finaliser (Steele, Lea & Flood 2014), a bijection on 64 bits.
__device__ __forceinline__ uint64_t fingerprint(const Key128& k, uint64_t salt) {
  uint64_t h = (k.lo * 0x9E3779B97F4A7C15ull) ^ ((k.hi + salt) * 0xD6E8FEB86659FD93ull);
  h ^= h >> 30;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 27;
  h *= 0x94D049BB133111EBull;
  h ^= h >> 31;
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

// Deletion variant v of key k (length L): v = 0 is k itself, then every single
// deletion, every pair, every triple; subsets in colexicographic order.
// sum_{j<=d} C(L, j) variants in all (variant_count).
__device__ __forceinline__ Key128 variant_of(const Key128& k, uint32_t L, uint32_t v) {
  if (v == 0) return k;
  if (v <= L) return delete_at(k, (int)(v - 1));
  uint32_t t = v - 1 - L;
  const uint32_t c2 = L * (L - 1) / 2;
  if (t < c2) {
    // {p < q} has colex rank q(q-1)/2 + p
    uint32_t q = (uint32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
    while (q * (q - 1) / 2 > t) --q;
    while ((q + 1) * q / 2 <= t) ++q;
    const uint32_t p = t - q * (q - 1) / 2;
    return delete_at(delete_at(k, (int)q), (int)p);
  }
  t -= c2;
  // {p < q < r} has colex rank C(r,3) + C(q,2) + p
  uint32_t r = 2;
  while (binom_small(r + 1, 3) <= t) ++r;
  t -= binom_small(r, 3);
  uint32_t q = 1;
  while (binom_small(q + 1, 2) <= t) ++q;
  t -= binom_small(q, 2);
  return delete_at(delete_at(delete_at(k, (int)r), (int)q), (int)t);
}

// ------------------------------------------------------------ host side ---
// Launch bookkeeping: optional CUDA-event timing per kernel (see
// xtn_profile_enable), tagged with algorithmic bytes.
void prof_begin(cudaStream_t s, const char* name, double bytes);
void prof_end(cudaStream_t s);

inline uint32_t div_up_u32(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

}  // namespace xtn
