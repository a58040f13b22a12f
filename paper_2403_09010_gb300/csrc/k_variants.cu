// Encoding and deletion-variant expansion (Appendix A, XTNeighbor steps 1-3;
// the `expand` primitive of Sec. 2.2: each input chunk writes a disjoint
// output chunk whose size is known ahead of time).
//
//   k_encode : ASCII sequence -> 128-bit key of 5-bit residue codes
//              (Appendix "Compression of TCR sequences"), its length, the
//              mask of positions equal to their left neighbour, and its
//              number of canonical deletion subsets (see is_canonical).
//   k_expand : one warp per sequence (metadata of 32 sequences fetched at
//              once); lane v takes canonical variant v (see variants.cuh),
//              fingerprints it from the prefix sums and writes the 64-bit
//              record  fingerprint[63:b] | id[b-1:0]  at rec_off[s] + v, so
//              every warp store is one contiguous run.  The kernel also
//              accumulates the digit histograms of the radix passes that will
//              sort the records (all of them, or only the first when each
//              sort pass counts the next).
//   k_peq    : per sequence, for each residue code c, the bit mask of the
//              positions holding c (the match vectors of the bit-parallel
//              edit distance used in verification).
#include <algorithm>

#include "variants.cuh"
#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

// 'A'..'Z' -> residue code (alphabetical order of the 20 one-letter codes),
// 0 for letters outside the alphabet (B J O U X Z) and for anything else.
// Computed, not looked up: lanes of a warp read different letters, which a
// constant-memory table would serve one at a time.
constexpr uint32_t NOT_RESIDUE = (1u << 1) | (1u << 9) | (1u << 14) | (1u << 20) | (1u << 23) |
                                 (1u << 25);  // B J O U X Z
__device__ __forceinline__ uint32_t letter_code(uint32_t ch) {
  const uint32_t x = ch - (uint32_t)'A';
  if (x >= 26u || ((NOT_RESIDUE >> x) & 1u)) return 0u;
  return x + 1u - (uint32_t)__popc(NOT_RESIDUE & ((1u << x) - 1u));
}

constexpr int ENCODE_WARPS = 8;

// One warp per 32 consecutive sequences: their letters form one contiguous
// byte span, copied to shared memory with coalesced loads; each lane then
// encodes its own sequence.  Offsets are validated per lane first; a warp
// with an invalid offset reads each valid lane's letters directly instead.
__global__ void __launch_bounds__(ENCODE_WARPS * 32)
    k_encode(const uint8_t* __restrict__ seqs, const int64_t* __restrict__ off, int64_t n, int d,
             Key128* __restrict__ keys, uint8_t* __restrict__ lens,
             uint32_t* __restrict__ eqprev_out, uint32_t* __restrict__ vcount,
             uint32_t* __restrict__ err) {
  __shared__ uint8_t s_bytes[ENCODE_WARPS][32 * XTN_MAX_LEN];
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const int64_t s0 = ((int64_t)blockIdx.x * ENCODE_WARPS + warp) * 32;
  if (s0 >= n) return;  // whole warp
  const int64_t i = s0 + lane;
  const bool in = i < n;
  const int64_t total = off[n];
  const int64_t a = in ? off[i] : 0, b = in ? off[i + 1] : 0;
  bool ok = in && a >= 0 && b >= a && b <= total;
  if (in && !ok) atomicOr(err, DERR_RANGE);
  if (i == 0 && a != 0) atomicOr(err, DERR_RANGE);  // offsets start at 0
  if (ok && b - a > XTN_MAX_LEN) {
    atomicOr(err, DERR_TOO_LONG);
    ok = false;
  }
  const bool all_ok = __all_sync(FULL_MASK, ok || !in);
  const int last = (int)((n - s0 < 32) ? (n - s0 - 1) : 31);
  const int64_t A = __shfl_sync(FULL_MASK, a, 0), Bend = __shfl_sync(FULL_MASK, b, last);
  uint8_t* buf = s_bytes[warp];
  const bool shared_span = all_ok && Bend - A <= 32 * XTN_MAX_LEN;
  if (shared_span) {
    for (int64_t k = lane; k < Bend - A; k += 32) buf[k] = seqs[A + k];
  }
  __syncwarp();
  Key128 key{0ull, 0ull};
  uint32_t L = 0, eqprev = 0;
  if (ok) {
    L = (uint32_t)(b - a);
    uint32_t prev = 0;
    for (uint32_t p = 0; p < L; ++p) {
      const uint32_t ch = shared_span ? buf[a - A + p] : seqs[a + p];
      const uint32_t c = letter_code(ch);
      if (c == 0) atomicOr(err, DERR_BAD_RESIDUE);
      if (p > 0 && c == prev) eqprev |= 1u << p;
      prev = c;
      const uint32_t m = 5 * p;
      if (m < 64) {
        key.lo |= (uint64_t)c << m;
        if (m > 59) key.hi |= (uint64_t)c >> (64 - m);
      } else {
        key.hi |= (uint64_t)c << (m - 64);
      }
    }
  }
  if (in) {
    keys[i] = key;
    lens[i] = (uint8_t)L;
    eqprev_out[i] = eqprev;
    if (d <= 2) {  // closed form of canonical_count, the one k_expand checks against
      const uint32_t all = L ? (0xffffffffu >> (32 - L)) : 0u;
      const uint32_t runs = ~eqprev & all;
      vcount[i] = canonical_total_d2(
          SeqShape{L, (uint32_t)__popc(runs), (uint32_t)__popc(runs & (eqprev >> 1))}, d);
    } else {
      vcount[i] = canonical_count(eqprev, L, (uint32_t)d);
    }
  }
}

constexpr int EXPAND_THREADS = 256;

// One count per radix pass for record `rec` (8-bit digits from bit `lo`; the
// last digit keeps only `last_mask`).
// HIW: lo >= 32 and every counted digit lies in the high word (32-bit shifts)
template <bool HIW = false>
__device__ __forceinline__ void count_digits(uint32_t* s_hist, uint64_t rec, int lo, int passes,
                                             uint32_t last_mask) {
  if (HIW) {
    const uint32_t r = (uint32_t)(rec >> 32) >> (lo - 32);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (p < passes) {
        const uint32_t m = p == passes - 1 ? last_mask : 0xffu;
        atomicAdd(&s_hist[p * RADIX + ((r >> (8 * p)) & m)], 1u);
      }
    }
    return;
  }
  const uint64_t r = rec >> lo;
#pragma unroll
  for (int p = 0; p < MAX_PASSES; ++p) {
    if (p < passes) {
      const uint32_t m = p == passes - 1 ? last_mask : 0xffu;
      atomicAdd(&s_hist[p * RADIX + ((uint32_t)(r >> (8 * p)) & m)], 1u);
    }
  }
}

static_assert((1 << MAX_BIN_BITS) <= MAX_PASSES * RADIX, "bins share the digit histogram");

// Appended records (SEL_APPEND) collect per warp in shared memory and go out
// STAGE_FLUSH or more at a time: a warp reserves output space once per
// batch, not once per round (rounds keep a record in nearly every warp
// whatever the share of bins selected, and every reservation is an atomic
// on one counter), and the stores are contiguous runs.
constexpr uint32_t STAGE_FLUSH = 128;
constexpr uint32_t STAGE_CAP = STAGE_FLUSH + 32;
struct WarpStage {
  uint64_t* buf;  // STAGE_CAP words of this warp
  uint32_t n;     // staged records (the same in every lane)
};

__device__ __forceinline__ void flush_stage(WarpStage& st, uint64_t* __restrict__ out,
                                            uint64_t n_rec, const BinSel& sel, uint32_t lane,
                                            uint32_t* __restrict__ err) {
  if (st.n == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(sel.append, (unsigned long long)st.n);
  base = __shfl_sync(FULL_MASK, base, 0);
  __syncwarp();  // every lane's staged records are visible
  for (uint32_t k = lane; k < st.n; k += 32) {
    const uint64_t slot = base + k;
    if (slot < n_rec)
      out[slot] = st.buf[k];
    else
      atomicOr(err, DERR_RANGE);
  }
  __syncwarp();  // read before the stage fills again
  st.n = 0;
}

// Where a finished record goes (all lanes of the warp call this together;
// `valid` says whether this lane holds a record):
//   SEL_ALL    out[pos], its digits counted for the sort
//   SEL_COUNT  only its fingerprint bin counted (s_hist holds the bins)
//   SEL_APPEND staged for appending when its bin lies in [sel.lo, sel.hi);
//              its digits counted
template <int SEL, bool HIW = false>
__device__ __forceinline__ void place_record(uint64_t rec, bool valid, uint64_t pos,
                                             uint64_t* __restrict__ out, uint64_t n_rec,
                                             uint32_t* s_hist, int hist_lo, int hist_passes,
                                             uint32_t last_mask, const BinSel& sel, uint32_t lane,
                                             WarpStage& st, uint32_t* __restrict__ err) {
  if constexpr (SEL == SEL_ALL) {
    if (valid) {
      out[pos] = rec;
      count_digits<HIW>(s_hist, rec, hist_lo, hist_passes, last_mask);
    }
  } else {
    const uint32_t bin = (uint32_t)(rec >> sel.shift) & sel.mask;
    if constexpr (SEL == SEL_COUNT) {
      if (valid) atomicAdd(&s_hist[bin], 1u);
    } else {
      const bool keep = valid && bin >= sel.lo && bin < sel.hi;
      const uint32_t bal = __ballot_sync(FULL_MASK, keep);
      if (keep) {
        st.buf[st.n + __popc(bal & ((1u << lane) - 1u))] = rec;  // st.n + 32 <= STAGE_CAP
        count_digits<HIW>(s_hist, rec, hist_lo, hist_passes, last_mask);
      }
      st.n += __popc(bal);
      if (st.n >= STAGE_FLUSH) flush_stage(st, out, n_rec, sel, lane, err);
    }
  }
}

// Clears n 16-byte words for a later kernel (the record sort's look-back
// status), grid-stride: the expansion is bound by instruction issue, so these
// stores cost it almost nothing and spare the sort a memset or the clearing.
__device__ __forceinline__ void zero_fill(uint4* __restrict__ p, uint64_t n) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x)
    p[k] = make_uint4(0u, 0u, 0u, 0u);
}

template <int SEL>
__global__ void __launch_bounds__(EXPAND_THREADS)
    k_expand(const Key128* __restrict__ keys, const uint8_t* __restrict__ lens,
             const uint32_t* __restrict__ eqprev, const uint64_t* __restrict__ rec_off, int64_t n,
             int d, const uint32_t* __restrict__ seq_rep, uint32_t id_bits,
             uint64_t* __restrict__ out, uint64_t n_rec, uint32_t* __restrict__ hist, int hist_lo,
             int hist_passes, int hist_hi, BinSel sel, uint32_t* __restrict__ err,
             uint4* __restrict__ zero, uint64_t n_zero) {
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  __shared__ VariantTables s_tab;
  __shared__ WarpVariants s_warp[EXPAND_THREADS / 32];
  zero_fill(zero, n_zero);
  constexpr int STAGE_WARPS = SEL == SEL_APPEND ? EXPAND_THREADS / 32 : 1;
  __shared__ uint64_t s_stage[STAGE_WARPS][SEL == SEL_APPEND ? STAGE_CAP : 1];
  WarpStage st{s_stage[SEL == SEL_APPEND ? threadIdx.x >> 5 : 0], 0u};
  const int n_hist = SEL == SEL_COUNT ? (int)sel.mask + 1 : hist_passes * RADIX;
  for (int k = threadIdx.x; k < n_hist; k += blockDim.x) s_hist[k] = 0;
  init_variant_tables(&s_tab);
  __syncthreads();
  WarpVariants* w = &s_warp[threadIdx.x >> 5];
  const uint32_t lane = lane_id();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t idmask = (id_bits >= 64) ? ~0ull : ((1ull << id_bits) - 1ull);
  const int last_bits = hist_hi - hist_lo - 8 * (hist_passes - 1);
  const uint32_t last_mask = (1u << last_bits) - 1u;
  // each warp takes 32 consecutive sequences per round: their metadata is
  // read with one coalesced load per field and handed out by shuffles
  for (int64_t s0 = warp0 * 32; s0 < n; s0 += n_warps * 32) {
    const int64_t my = s0 + lane;
    Key128 mk{0ull, 0ull};
    uint32_t mL = 0, mEq = 0, mRep = 0;
    uint64_t mBase = 0, mEnd = 0;
    if (my < n) {
      mk = keys[my];
      mL = lens[my];
      mEq = eqprev[my];
      mBase = rec_off[my];
      mEnd = rec_off[my + 1];
      if (seq_rep) mRep = seq_rep[my];
    }
    const int m = (n - s0 < 32) ? (int)(n - s0) : 32;
    for (int j = 0; j < m; ++j) {
      const int64_t s = s0 + j;
      const Key128 k{__shfl_sync(FULL_MASK, mk.lo, j), __shfl_sync(FULL_MASK, mk.hi, j)};
      const uint32_t L = __shfl_sync(FULL_MASK, mL, j);
      const uint32_t eq = __shfl_sync(FULL_MASK, mEq, j);
      const uint64_t base = __shfl_sync(FULL_MASK, mBase, j);
      uint32_t cnt = (uint32_t)(__shfl_sync(FULL_MASK, mEnd, j) - base);
      if (SEL == SEL_ALL && base + cnt > n_rec) {
        if (lane == 0) atomicOr(err, DERR_RANGE);
        cnt = 0;
      }
      const uint64_t salt = seq_rep ? rep_salt(__shfl_sync(FULL_MASK, mRep, j)) : 0ull;
      const SeqShape sh = warp_prepare(w, &s_tab, k, L, eq, lane);
      if (d <= 2) {
        uint32_t total = canonical_total_d2(sh, d);
        if (total != cnt) {
          if (lane == 0) atomicOr(err, DERR_RANGE);
          total = 0;
        }
        for (uint32_t v0 = 0; v0 < total; v0 += 32) {
          const uint32_t v = v0 + lane;
          uint64_t rec = 0;
          if (v < total)
            rec = (canonical_fingerprint_d2(w, &s_tab, sh, v, salt) & ~idmask) | (uint64_t)s;
          place_record<SEL>(rec, v < total, base + v, out, n_rec, s_hist, hist_lo, hist_passes,
                            last_mask, sel, lane, st, err);
        }
      } else {
        // every subset with <= d deletions, canonical ones kept (ballot compaction)
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
          const bool ok = keep && slot < cnt;
          uint64_t rec = 0;
          if (ok) rec = (subset_fingerprint(w, L, ss, salt) & ~idmask) | (uint64_t)s;
          place_record<SEL>(rec, ok, base + slot, out, n_rec, s_hist, hist_lo, hist_passes,
                            last_mask, sel, lane, st, err);
          written += __popc(bal);
        }
        if (written != cnt && lane == 0) atomicOr(err, DERR_RANGE);
      }
    }
  }
  if constexpr (SEL == SEL_APPEND) flush_stage(st, out, n_rec, sel, lane, err);
  __syncthreads();
  uint32_t* dst = SEL == SEL_COUNT ? sel.bin_count : hist;
  for (int k = threadIdx.x; k < n_hist; k += blockDim.x)
    if (s_hist[k]) atomicAdd(&dst[k], s_hist[k]);
}

// Packed expansion for d <= 2.  A warp takes PACK_SEQS consecutive
// sequences; lane i < PACK_SEQS first prepares sequence i alone (prefix sums
// of the polynomial fingerprint, run starts, canonical variant count), then
// the whole warp walks the batch's records as one stream: record t of the
// batch belongs to the sequence whose start (exclusive scan of the counts) is
// the largest <= t, found by a 4-step search over the lanes' starts.  Every
// lane computes a record in every round and the batch's records are
// contiguous in the output, so the stores stay coalesced; no warp-wide work
// is spent per sequence.  16 sequences a batch keep the per-warp tables at
// about 4 KB, so that enough warps fit on an SM to hide the arithmetic's
// latency.
constexpr int PACK_WARPS = 8;
constexpr int PACK_SEQS = 16;
constexpr int PACK_STRIDE = XTN_MAX_LEN + 3;  // P[0 .. L + 2]

struct PackedSeqs {
  uint64_t P[PACK_SEQS][PACK_STRIDE];
  uint8_t rs[PACK_SEQS][XTN_MAX_LEN + 1];
  uint8_t ds[PACK_SEQS][XTN_MAX_LEN / 2 + 1];
};

// PK_SALT: sequences carry a repertoire salt (seq_rep given); PK_HIW: the
// histogram's digits lie in the record's high word (hist_lo >= 32).
constexpr int PK_SALT = 1, PK_HIW = 2;

template <int SEL, int PK>
__global__ void __launch_bounds__(PACK_WARPS * 32)
    k_expand_packed(const Key128* __restrict__ keys, const uint8_t* __restrict__ lens,
                    const uint32_t* __restrict__ eqprev, const uint64_t* __restrict__ rec_off,
                    int64_t n, int d, const uint32_t* __restrict__ seq_rep, uint32_t id_bits,
                    uint64_t* __restrict__ out, uint64_t n_rec, uint32_t* __restrict__ hist,
                    int hist_lo, int hist_passes, int hist_hi, BinSel sel,
                    uint32_t* __restrict__ err, uint4* __restrict__ zero, uint64_t n_zero) {
  zero_fill(zero, n_zero);
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  __shared__ VariantTables s_tab;
  __shared__ PackedSeqs s_seq[PACK_WARPS];
  constexpr int STAGE_WARPS = SEL == SEL_APPEND ? PACK_WARPS : 1;
  __shared__ uint64_t s_stage[STAGE_WARPS][SEL == SEL_APPEND ? STAGE_CAP : 1];
  WarpStage st{s_stage[SEL == SEL_APPEND ? threadIdx.x >> 5 : 0], 0u};
  const int n_hist = SEL == SEL_COUNT ? (int)sel.mask + 1 : hist_passes * RADIX;
  for (int k = threadIdx.x; k < n_hist; k += blockDim.x) s_hist[k] = 0;
  init_variant_tables(&s_tab);
  __syncthreads();
  PackedSeqs* ps = &s_seq[threadIdx.x >> 5];
  const uint32_t lane = lane_id();
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t idmask = (id_bits >= 64) ? ~0ull : ((1ull << id_bits) - 1ull);
  const int last_bits = hist_hi - hist_lo - 8 * (hist_passes - 1);
  const uint32_t last_mask = (1u << last_bits) - 1u;
  static_assert(PACK_SEQS <= 32 && (PACK_SEQS & (PACK_SEQS - 1)) == 0, "power of two <= 32");
  for (int64_t s0 = warp0 * PACK_SEQS; s0 < n; s0 += n_warps * PACK_SEQS) {
    const int64_t my = s0 + lane;
    // ---- this lane's sequence
    uint32_t L = 0, R = 0, nD = 0, total = 0;
    uint64_t salt = 0, base = 0;
    if (lane < (uint32_t)PACK_SEQS && my < n) {
      Key128 k = keys[my];
      L = lens[my];
      const uint32_t eq = eqprev[my];
      base = rec_off[my];
      const uint64_t cnt = rec_off[my + 1] - base;
      if ((PK & PK_SALT) && seq_rep) salt = rep_salt(seq_rep[my]);
      if (L > XTN_MAX_LEN) L = XTN_MAX_LEN;  // encode rejects longer ones
      uint64_t acc = 0, pw = 1;
      ps->P[lane][0] = 0ull;
      for (uint32_t p = 0; p < L; ++p) {
        acc += (uint64_t)(uint32_t)(k.lo & 31u) * pw;
        pw *= HASH_B;
        k.lo = (k.lo >> 5) | (k.hi << 59);
        k.hi >>= 5;
        ps->P[lane][p + 1] = acc;
      }
      for (uint32_t p = L + 1; p <= L + 2; ++p) ps->P[lane][p] = acc;
      const uint32_t all = L ? (0xffffffffu >> (32 - L)) : 0u;
      uint32_t runs = ~eq & all;
      uint32_t dbl = runs & (eq >> 1);
      R = __popc(runs);
      nD = __popc(dbl);
      for (uint32_t i = 0; runs; ++i, runs &= runs - 1) ps->rs[lane][i] = (uint8_t)(__ffs(runs) - 1);
      for (uint32_t i = 0; dbl; ++i, dbl &= dbl - 1) ps->ds[lane][i] = (uint8_t)(__ffs(dbl) - 1);
      total = canonical_total_d2(SeqShape{L, R, nD}, d);
      if (total != cnt || (SEL == SEL_ALL && base + cnt > n_rec)) {
        atomicOr(err, DERR_RANGE);
        total = 0;
      }
    }
    // ---- the batch's records, 32 at a time
    uint32_t start = total;  // exclusive scan of the totals over lanes
#pragma unroll
    for (int o = 1; o < PACK_SEQS; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL_MASK, start, o);
      if (lane >= (uint32_t)o) start += t;
    }
    const uint32_t T = __shfl_sync(FULL_MASK, start, PACK_SEQS - 1);
    start -= total;
    const uint64_t base0 = __shfl_sync(FULL_MASK, base, 0);
    __syncwarp();  // the tables written above are read by every lane below
    for (uint32_t t0 = 0; t0 < T; t0 += 32) {
      const uint32_t t = t0 + lane;
      // largest j with start[j] <= t (starts do not decrease)
      uint32_t j = 0;
#pragma unroll
      for (int step = PACK_SEQS / 2; step > 0; step >>= 1) {
        const uint32_t sj = __shfl_sync(FULL_MASK, start, (int)(j + step));
        if (sj <= t) j += step;
      }
      const uint32_t sj = __shfl_sync(FULL_MASK, start, (int)j);
      const uint32_t Lj = __shfl_sync(FULL_MASK, L, (int)j);
      const uint32_t Rj = __shfl_sync(FULL_MASK, R, (int)j);
      const uint32_t Dj = __shfl_sync(FULL_MASK, nD, (int)j);
      const uint64_t saltj = (PK & PK_SALT) ? __shfl_sync(FULL_MASK, salt, (int)j) : 0ull;
      uint64_t rec = 0;
      if (t < T) {
        const uint32_t v = t - sj;
        // canonical variant v of sequence j (numbering of canonical_fingerprint_d2)
        const uint32_t u = v - 1 - Rj;
        const uint32_t c2 = Rj * (Rj - 1) / 2;
        const bool single = v >= 1 && v <= Rj;
        const bool pair = v > Rj && u < c2;
        const bool dbl = v > Rj && u >= c2;
        const uint32_t pr = s_tab.pair[pair ? u : 0u];
        const uint32_t a = ps->rs[j][single ? v - 1 : (pr & 255u)];
        const uint32_t b = ps->rs[j][pr >> 8];
        const uint32_t c = ps->ds[j][dbl ? u - c2 : 0u];
        const uint32_t p1 = single || pair ? a : (dbl ? c : Lj);
        const uint32_t p2 = pair ? b : (dbl ? c + 1 : (single ? Lj : Lj + 1));
        auto P = [&](uint32_t x) { return ps->P[j][x]; };
        const uint64_t h = P(p1) + HASH_BINV * ((P(p2) - P(p1 + 1)) +
                                                HASH_BINV * (P(Lj) - P(p2 + 1)));
        rec = (mix64((PK & PK_SALT) ? h ^ saltj : h) & ~idmask) | (uint64_t)(s0 + j);
      }
      place_record<SEL, (PK & PK_HIW) != 0>(rec, t < T, base0 + t, out, n_rec, s_hist, hist_lo,
                                            hist_passes, last_mask, sel, lane, st, err);
    }
    __syncwarp();  // the next batch overwrites the tables
  }
  if constexpr (SEL == SEL_APPEND) flush_stage(st, out, n_rec, sel, lane, err);
  __syncthreads();
  uint32_t* dst = SEL == SEL_COUNT ? sel.bin_count : hist;
  for (int k = threadIdx.x; k < n_hist; k += blockDim.x)
    if (s_hist[k]) atomicAdd(&dst[k], s_hist[k]);
}

// Match vectors: peq[i * PEQ_STRIDE + c - 1] = {positions p of sequence i with code c}.
constexpr int PEQ_THREADS = 128;

__global__ void __launch_bounds__(PEQ_THREADS)
    k_peq(const Key128* __restrict__ keys, const uint8_t* __restrict__ lens, int64_t n,
          uint32_t* __restrict__ peq) {
  __shared__ uint32_t s_peq[PEQ_THREADS * PEQ_STRIDE];
  const int64_t first = (int64_t)blockIdx.x * PEQ_THREADS;
  for (int k = threadIdx.x; k < PEQ_THREADS * PEQ_STRIDE; k += PEQ_THREADS) s_peq[k] = 0;
  __syncthreads();
  const int64_t i = first + threadIdx.x;
  if (i < n) {
    Key128 k = keys[i];
    const uint32_t L = lens[i];
    uint32_t* row = s_peq + threadIdx.x * PEQ_STRIDE;
    for (uint32_t p = 0; p < L; ++p) {
      const uint32_t c = (uint32_t)(k.lo & 31u);
      k.lo = (k.lo >> 5) | (k.hi << 59);
      k.hi >>= 5;
      if (c >= 1 && c <= 20) row[c - 1] |= 1u << p;
    }
  }
  __syncthreads();
  const int64_t rows = (n - first < PEQ_THREADS) ? (n - first) : PEQ_THREADS;
  for (int64_t k = threadIdx.x; k < rows * PEQ_STRIDE; k += PEQ_THREADS)
    peq[first * PEQ_STRIDE + k] = s_peq[k];
}

// seq_rep[i] = repertoire of sequence i: the last r with rep_off[r] <= i.
__global__ void k_seq_rep(const int64_t* __restrict__ rep_off, int64_t n_rep,
                          uint32_t* __restrict__ seq_rep, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t lo = 0, hi = n_rep;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (rep_off[mid] <= i) lo = mid; else hi = mid;
  }
  seq_rep[i] = (uint32_t)lo;
}

void launch_seq_rep(const int64_t* rep_off, int64_t n_rep, uint32_t* seq_rep, int64_t n,
                    cudaStream_t s) {
  if (n <= 0) return;
  prof_begin(s, "k_seq_rep", (double)n * 4.0);
  k_seq_rep<<<div_up_u32(n, 256), 256, 0, s>>>(rep_off, n_rep, seq_rep, n);
  prof_end(s);
}

void launch_encode(const uint8_t* seqs, const int64_t* off, int64_t n, int d, Key128* keys,
                   uint8_t* lens, uint32_t* eqprev, uint32_t* vcount, uint32_t* err,
                   cudaStream_t s) {
  if (n <= 0) return;
  prof_begin(s, "k_encode", (double)n * (16 + 16 + 1 + 4 + 4 + 8));
  k_encode<<<div_up_u32(n, ENCODE_WARPS * 32), ENCODE_WARPS * 32, 0, s>>>(seqs, off, n, d, keys,
                                                                           lens, eqprev, vcount,
                                                                           err);
  prof_end(s);
}

template <int SEL>
static void expand_launch(const Key128* keys, const uint8_t* lens, const uint32_t* eqprev,
                          const uint64_t* rec_off, int64_t n, int d, const uint32_t* seq_rep,
                          uint32_t id_bits, uint64_t* out, uint64_t n_rec, uint32_t* hist,
                          int hist_lo, int passes, int hist_hi, const BinSel& sel, int sms,
                          uint32_t* err, cudaStream_t s, uint4* zero, uint64_t n_zero) {
  if (d <= 2) {
    const int pblocks = (int)std::min<int64_t>(
        (n + PACK_WARPS * PACK_SEQS - 1) / (PACK_WARPS * PACK_SEQS), (int64_t)sms * 8);
    // the plain expansion picks its variant; the bin passes take the general one
    auto f = k_expand_packed<SEL, PK_SALT>;
    if (SEL == SEL_ALL) {
      const bool hiw = hist_lo >= 32 && hist_hi <= 64;
      f = seq_rep ? (hiw ? k_expand_packed<SEL, PK_SALT | PK_HIW> : k_expand_packed<SEL, PK_SALT>)
                  : (hiw ? k_expand_packed<SEL, PK_HIW> : k_expand_packed<SEL, 0>);
    }
    f<<<pblocks > 0 ? pblocks : 1, PACK_WARPS * 32, 0, s>>>(keys, lens, eqprev, rec_off, n, d,
                                                              seq_rep, id_bits, out, n_rec, hist,
                                                              hist_lo, passes, hist_hi, sel, err,
                                                              zero, n_zero);
  } else {
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    if (blocks < 1) blocks = 1;
    k_expand<SEL><<<blocks, EXPAND_THREADS, 0, s>>>(keys, lens, eqprev, rec_off, n, d, seq_rep,
                                                    id_bits, out, n_rec, hist, hist_lo, passes,
                                                    hist_hi, sel, err, zero, n_zero);
  }
}

void launch_expand(const Key128* keys, const uint8_t* lens, const uint32_t* eqprev,
                   const uint64_t* rec_off, int64_t n, int d, const uint32_t* seq_rep,
                   uint32_t id_bits, uint64_t* out, uint64_t n_rec, uint32_t* hist, int hist_lo,
                   int hist_hi, int sms, uint32_t* err, cudaStream_t s, const BinSel* sel,
                   void* zero, size_t zero_bytes) {
  uint4* z = static_cast<uint4*>(zero);
  const uint64_t nz = z ? zero_bytes / 16 : 0;
  if (n <= 0) return;
  const int passes = (hist_hi - hist_lo + 7) / 8;
  const BinSel none{};
  if (!sel) {
    prof_begin(s, "k_expand", (double)n_rec * 8.0 + (double)n * 29.0);
    expand_launch<SEL_ALL>(keys, lens, eqprev, rec_off, n, d, seq_rep, id_bits, out, n_rec, hist,
                           hist_lo, passes, hist_hi, none, sms, err, s, z, nz);
  } else if (sel->append) {
    prof_begin(s, "k_expand_bins", (double)n_rec * 8.0 + (double)n * 29.0);
    expand_launch<SEL_APPEND>(keys, lens, eqprev, rec_off, n, d, seq_rep, id_bits, out, n_rec,
                              hist, hist_lo, passes, hist_hi, *sel, sms, err, s, z, nz);
  } else {
    prof_begin(s, "k_expand_count", (double)n * 29.0);
    expand_launch<SEL_COUNT>(keys, lens, eqprev, rec_off, n, d, seq_rep, id_bits, out, n_rec,
                             hist, hist_lo, passes, hist_hi, *sel, sms, err, s, z, nz);
  }
  prof_end(s);
}

void launch_peq(const Key128* keys, const uint8_t* lens, int64_t n, uint32_t* peq,
                cudaStream_t s) {
  if (n <= 0) return;
  prof_begin(s, "k_peq", (double)n * (17.0 + 4.0 * PEQ_STRIDE));
  k_peq<<<div_up_u32(n, PEQ_THREADS), PEQ_THREADS, 0, s>>>(keys, lens, n, peq);
  prof_end(s);
}

}  // namespace xtn
