// Warp-cooperative enumeration of the canonical deletion variants of one
// sequence and their fingerprints (Appendix A, XTNeighbor step 2; `expand`).
// Used by the self-search expansion and by the query lookup so that both
// sides fingerprint every variant string identically.
//
// For one sequence a warp builds, in shared memory:
//   P[x]  prefix sums of the polynomial fingerprint (P[x] = P[L] for x >= L),
//   rs[i] the position where run i of equal residues starts,
//   ds[i] the i-th run start whose run has length >= 2.
// Canonical subsets with at most 2 deletions are then numbered directly:
//   v = 0                         : no deletion
//   v = 1 .. R                    : first residue of run v-1
//   v = R+1 .. R+C(R,2)           : first residues of runs i < j (colex rank)
//   v = R+C(R,2)+1 .. (+nD)       : first two residues of the v-th long run
// which is exactly the set counted by canonical_count(), so no lane of the
// warp computes a variant that is then thrown away.  d = 3 enumerates every
// subset and keeps the canonical ones.
#pragma once

#include "xtn_common.cuh"

namespace xtn {

constexpr int PAIR_TABLE = XTN_MAX_LEN * (XTN_MAX_LEN - 1) / 2;  // 300

struct VariantTables {
  uint64_t pow[XTN_MAX_LEN + 1];  // B^k
  uint16_t pair[PAIR_TABLE];      // colex rank t -> (i | j << 8), i < j
};

// P is kept as two 32-bit halves so that lanes reading different entries
// never share a shared-memory bank.
struct WarpVariants {
  uint32_t Plo[32];
  uint32_t Phi[32];
  uint8_t rs[32];
  uint8_t ds[32];
};

__device__ __forceinline__ uint64_t prefix_at(const WarpVariants* w, uint32_t x) {
  return ((uint64_t)w->Phi[x] << 32) | w->Plo[x];
}

// Called by every thread of the block, followed by __syncthreads().
__device__ __forceinline__ void init_variant_tables(VariantTables* t) {
  for (int k = threadIdx.x; k <= XTN_MAX_LEN; k += blockDim.x) {
    uint64_t p = 1;
    for (int e = 0; e < k; ++e) p *= HASH_B;
    t->pow[k] = p;
  }
  for (int r = threadIdx.x; r < PAIR_TABLE; r += blockDim.x) {
    uint32_t j = 1;
    while ((j + 1) * j / 2 <= (uint32_t)r) ++j;
    t->pair[r] = (uint16_t)((r - j * (j - 1) / 2) | (j << 8));
  }
}

struct SeqShape {
  uint32_t L, R, nD;
};

// All 32 lanes: fill w for (key, L, eqprev).  Ends with __syncwarp().
__device__ __forceinline__ SeqShape warp_prepare(WarpVariants* w, const VariantTables* t,
                                                 const Key128& key, uint32_t L, uint32_t eq,
                                                 uint32_t lane) {
  __syncwarp();  // the previous sequence's readers are done with w
  const uint64_t term = lane < L ? (uint64_t)code_at(key, (int)lane) * t->pow[lane] : 0ull;
  const uint64_t incl = warp_incl_scan_u64(term);
  const uint64_t PL = L ? __shfl_sync(FULL_MASK, incl, (int)L - 1) : 0ull;
  if (lane < L + 3) {
    const uint64_t v = lane < L ? incl : PL;
    w->Plo[lane + 1] = (uint32_t)v;
    w->Phi[lane + 1] = (uint32_t)(v >> 32);
  }
  if (lane == 0) {
    w->Plo[0] = 0u;
    w->Phi[0] = 0u;
  }
  const uint32_t all = L ? (0xffffffffu >> (32 - L)) : 0u;
  const uint32_t runs = ~eq & all;
  const uint32_t dbl = runs & (eq >> 1);
  const uint32_t lt = (1u << lane) - 1u;
  if ((runs >> lane) & 1u) w->rs[__popc(runs & lt)] = (uint8_t)lane;
  if ((dbl >> lane) & 1u) w->ds[__popc(dbl & lt)] = (uint8_t)lane;
  __syncwarp();
  return SeqShape{L, (uint32_t)__popc(runs), (uint32_t)__popc(dbl)};
}

// Number of canonical variants with at most d <= 2 deletions.
__device__ __forceinline__ uint32_t canonical_total_d2(const SeqShape& sh, int d) {
  if (d <= 0) return 1u;
  if (d == 1) return 1u + sh.R;
  return 1u + sh.R + sh.R * (sh.R - 1) / 2 + sh.nD;
}

// Fingerprint of canonical variant v (d <= 2 numbering above): positions
// chosen without branches, then the two-deletion form of the prefix formula
// in Horner order, H = P[p1] + B^-1 ((P[p2] - P[p1+1]) + B^-1 (P[L] - P[p2+1])),
// with p2 = L for one deletion and p1 = L, p2 = L+1 for none.
__device__ __forceinline__ uint64_t canonical_fingerprint_d2(const WarpVariants* w,
                                                             const VariantTables* t,
                                                             const SeqShape& sh, uint32_t v,
                                                             uint64_t salt) {
  const uint32_t L = sh.L, R = sh.R;
  const uint32_t u = v - 1 - R;                       // valid when v > R
  const uint32_t c2 = R * (R - 1) / 2;
  const bool single = v >= 1 && v <= R;
  const bool pair = v > R && u < c2;
  const bool dbl = v > R && u >= c2;
  const uint32_t pr = t->pair[pair ? u : 0u];
  const uint32_t a = w->rs[single ? v - 1 : (pr & 255u)];
  const uint32_t b = w->rs[pr >> 8];
  const uint32_t c = w->ds[dbl ? u - c2 : 0u];
  const uint32_t p1 = single || pair ? a : (dbl ? c : L);
  const uint32_t p2 = pair ? b : (dbl ? c + 1 : (single ? L : L + 1));
  const uint64_t h = prefix_at(w, p1) +
                     HASH_BINV * ((prefix_at(w, p2) - prefix_at(w, p1 + 1)) +
                                  HASH_BINV * (prefix_at(w, L) - prefix_at(w, p2 + 1)));
  return mix64(h ^ salt);
}

// Fingerprint of an arbitrary subset (positions from unrank_subset).
__device__ __forceinline__ uint64_t subset_fingerprint(const WarpVariants* w, uint32_t L,
                                                       const Subset& ss, uint64_t salt) {
  uint32_t p1 = L, p2 = L + 1, p3 = L + 2;
  if (ss.k == 1) {
    p1 = ss.p;
    p2 = L;
    p3 = L + 1;
  } else if (ss.k == 2) {
    p1 = ss.p;
    p2 = ss.q;
    p3 = L;
  } else if (ss.k == 3) {
    p1 = ss.p;
    p2 = ss.q;
    p3 = ss.r;
  }
  const uint64_t h = prefix_at(w, p1) + (prefix_at(w, p2) - prefix_at(w, p1 + 1)) * HASH_BINV +
                     (prefix_at(w, p3) - prefix_at(w, p2 + 1)) * HASH_BINV2 +
                     (prefix_at(w, L) - prefix_at(w, p3 + 1)) * HASH_BINV3;
  return mix64(h ^ salt);
}

}  // namespace xtn
