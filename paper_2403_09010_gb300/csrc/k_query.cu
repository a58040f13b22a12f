// Query-vs-reference lookup against a resident, sorted variant index: the
// SymDel step "reuse x to look up the hash map" (Appendix A, SymDel steps 2-3)
// with the hash map realised as the sorted record array of Sec. 2.2.
//
//   k_build_dir    : dir[t] = first index record whose top `dir_bits`
//                    fingerprint bits are >= t, so a lookup starts from a
//                    range of ~n_rec / 2^dir_bits records (a few, with the
//                    directory sized at about one entry per 4 records)
//                    instead of all.
//   k_query_lookup : one warp per query, one lane per deletion variant (same
//                    order as the self-search expansion): binary search of the
//                    variant's fingerprint group inside its directory range;
//                    writes the group's start and size.
//   k_query_emit   : candidate t finds its query variant by binary search over
//                    the candidate offsets, reads the reference id at the
//                    matching index position and writes (q << ref_bits) | r.
#include <algorithm>

#include "variants.cuh"
#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

// One thread per sorted position p in [0, n_rec]: the directory entries t
// in (top(rec[p-1]), top(rec[p])] all start at p (top(rec[-1]) = -1,
// top(rec[n_rec]) = 2^dir_bits), so every entry is written exactly once in
// one coalesced pass over the records.
// The same pass counts the groups (positions whose group key, the bits from
// gshift up, differs from the previous record's) into *n_groups.
__global__ void k_build_dir(const uint64_t* __restrict__ rec, uint64_t n_rec, int dir_bits,
                            int gshift, uint32_t* __restrict__ dir,
                            unsigned long long* __restrict__ n_groups) {
  const int64_t n_dir = 1ll << dir_bits;
  uint32_t heads = 0;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= n_rec;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t prev = p == 0 ? -1 : (int64_t)(rec[p - 1] >> (64 - dir_bits));
    const int64_t cur = p == n_rec ? n_dir : (int64_t)(rec[p] >> (64 - dir_bits));
    for (int64_t t = prev + 1; t <= cur && t <= n_dir; ++t) dir[t] = (uint32_t)p;
    if (p < n_rec && (p == 0 || (rec[p] >> gshift) != (rec[p - 1] >> gshift))) ++heads;
  }
  heads = (uint32_t)__reduce_add_sync(FULL_MASK, heads);
  if (lane_id() == 0 && heads) atomicAdd(n_groups, (unsigned long long)heads);
}

void launch_build_dir(const uint64_t* rec, uint64_t n_rec, int dir_bits, int gshift,
                      uint32_t* dir, uint64_t* n_groups, cudaStream_t s) {
  const uint64_t n_dir = (1ull << dir_bits) + 1;
  prof_begin(s, "k_build_dir", (double)n_rec * 8.0 + (double)n_dir * 4.0);
  const uint32_t blocks = (uint32_t)std::min<uint64_t>((n_rec + 256) / 256, 152ull * 32);
  k_build_dir<<<blocks, 256, 0, s>>>(rec, n_rec, dir_bits, gshift, dir,
                                     reinterpret_cast<unsigned long long*>(n_groups));
  prof_end(s);
}

// Group [lo, hi) of fingerprint fp in the sorted index (empty if absent).
__device__ __forceinline__ void index_range(const uint64_t* __restrict__ rec, uint64_t n_rec,
                                            const uint32_t* __restrict__ dir, int dir_bits,
                                            int gshift, uint64_t fp, uint32_t* err, uint64_t& a,
                                            uint64_t& c) {
  const uint64_t g = fp >> gshift;
  const uint64_t top = fp >> (64 - dir_bits);
  uint64_t lo = dir[top], hi = dir[top + 1];
  if (hi > n_rec || lo > hi) {
    atomicOr(err, DERR_RANGE);
    lo = hi = 0;
  }
  a = lo;
  uint64_t b = hi;  // lower bound of g
  while (a < b) {
    const uint64_t mid = (a + b) >> 1;
    if ((rec[mid] >> gshift) < g) a = mid + 1; else b = mid;
  }
  c = a;
  uint64_t e = hi;  // upper bound of g
  while (c < e) {
    const uint64_t mid = (c + e) >> 1;
    if ((rec[mid] >> gshift) <= g) c = mid + 1; else e = mid;
  }
}

__global__ void __launch_bounds__(256)
    k_query_lookup(const Key128* __restrict__ qkeys, const uint8_t* __restrict__ qlens,
                   const uint32_t* __restrict__ qeqprev, const uint64_t* __restrict__ q_rec_off,
                   int64_t n_q, uint64_t n_qv, int d, const uint64_t* __restrict__ rec,
                   uint64_t n_rec, const uint32_t* __restrict__ dir, int dir_bits, int gshift,
                   uint32_t* __restrict__ qv_start, uint32_t* __restrict__ qv_cnt,
                   uint32_t* __restrict__ qv_q, uint32_t* __restrict__ err) {
  __shared__ VariantTables s_tab;
  __shared__ WarpVariants s_warp[8];
  init_variant_tables(&s_tab);
  __syncthreads();
  WarpVariants* w = &s_warp[threadIdx.x >> 5];
  const uint32_t lane = lane_id();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp0; q < n_q; q += n_warps) {
    const uint32_t L = qlens[q];
    const uint32_t eq = qeqprev[q];
    const uint64_t base = q_rec_off[q];
    uint32_t cnt = (uint32_t)(q_rec_off[q + 1] - base);
    if (base + cnt > n_qv) {
      if (lane == 0) atomicOr(err, DERR_RANGE);
      cnt = 0;
    }
    const SeqShape sh = warp_prepare(w, &s_tab, qkeys[q], L, eq, lane);
    if (d <= 2) {
      uint32_t total = canonical_total_d2(sh, d);
      if (total != cnt) {
        if (lane == 0) atomicOr(err, DERR_RANGE);
        total = 0;
      }
      for (uint32_t v = lane; v < total; v += 32) {
        uint64_t a, c;
        index_range(rec, n_rec, dir, dir_bits, gshift,
                    canonical_fingerprint_d2(w, &s_tab, sh, v, 0ull), err, a, c);
        qv_start[base + v] = (uint32_t)a;
        qv_cnt[base + v] = (uint32_t)(c - a);
        qv_q[base + v] = (uint32_t)q;
      }
    } else {
      const uint32_t total = cnt ? variant_count(L, (uint32_t)d) : 0u;
      uint32_t written = 0;
      for (uint32_t v0 = 0; v0 < total; v0 += 32) {
        const uint32_t v = v0 + lane;
        bool keep = false;
        Subset ss{0u, 0u, 0u, 0u};
        if (v < total) {
          ss = unrank_subset(L, v);
          keep = is_canonical(subset_mask(ss), eq);
        }
        const uint32_t bal = __ballot_sync(FULL_MASK, keep);
        const uint32_t slot = written + __popc(bal & lt_mask);
        written += __popc(bal);
        if (keep && slot < cnt) {
          uint64_t a, c;
          index_range(rec, n_rec, dir, dir_bits, gshift, subset_fingerprint(w, L, ss, 0ull), err,
                      a, c);
          qv_start[base + slot] = (uint32_t)a;
          qv_cnt[base + slot] = (uint32_t)(c - a);
          qv_q[base + slot] = (uint32_t)q;
        }
      }
    }
  }
}

void launch_query_lookup(const Key128* qkeys, const uint8_t* qlens, const uint32_t* qeqprev,
                         const uint64_t* q_rec_off, int64_t n_q, uint64_t n_qv, int d,
                         const uint64_t* rec, uint64_t n_rec, const uint32_t* dir,
                         int dir_bits, int gshift, uint32_t* qv_start, uint32_t* qv_cnt,
                         uint32_t* qv_q, int sms, uint32_t* err, cudaStream_t s) {
  if (n_q <= 0) return;
  const int blocks = (int)std::min<int64_t>((n_q + 7) / 8, (int64_t)sms * 8);
  prof_begin(s, "k_query_lookup", (double)n_q * 30.0);
  k_query_lookup<<<blocks, 256, 0, s>>>(qkeys, qlens, qeqprev, q_rec_off, n_q, n_qv, d, rec, n_rec,
                                        dir, dir_bits, gshift, qv_start, qv_cnt, qv_q, err);
  prof_end(s);
}

__global__ void __launch_bounds__(256)
    k_query_emit(const uint64_t* __restrict__ rec, uint64_t n_rec, uint32_t ref_bits,
                 const uint32_t* __restrict__ qv_start, const uint32_t* __restrict__ qv_q,
                 const uint64_t* __restrict__ cand_off, uint64_t n_qv, uint64_t n_cand,
                 uint64_t* __restrict__ out, uint32_t* __restrict__ err) {
  const uint64_t idmask = (1ull << ref_bits) - 1ull;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_cand;
       t += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t lo = 0, hi = n_qv;  // largest v with cand_off[v] <= t
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) >> 1;
      if (cand_off[mid] <= t) lo = mid; else hi = mid;
    }
    const uint64_t pos = (uint64_t)qv_start[lo] + (t - cand_off[lo]);
    uint64_t w = 0;
    if (pos < n_rec) {
      w = ((uint64_t)qv_q[lo] << ref_bits) | (rec[pos] & idmask);
    } else {
      atomicOr(err, DERR_RANGE);
    }
    out[t] = w;
  }
}

void launch_query_emit(const uint64_t* rec, uint64_t n_rec, uint32_t ref_bits,
                       const uint32_t* qv_start, const uint32_t* qv_q, const uint64_t* cand_off,
                       uint64_t n_qv, uint64_t n_cand, uint64_t* out, int sms, uint32_t* err,
                       cudaStream_t s) {
  if (n_cand == 0) return;
  const int blocks = (int)std::min<uint64_t>((n_cand + 255) / 256, (uint64_t)sms * 8);
  prof_begin(s, "k_query_emit", (double)n_cand * 24.0);
  k_query_emit<<<blocks, 256, 0, s>>>(rec, n_rec, ref_bits, qv_start, qv_q, cand_off, n_qv, n_cand,
                                      out, err);
  prof_end(s);
}

}  // namespace xtn
