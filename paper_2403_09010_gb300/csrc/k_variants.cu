// Encoding and deletion-variant expansion (Appendix A, XTNeighbor steps 1-3;
// the `expand` primitive of Sec. 2.2: each input chunk writes a disjoint
// output chunk whose size is known ahead of time).
//
//   k_encode : ASCII sequence -> 128-bit key of 5-bit residue codes
//              (Appendix "Compression of TCR sequences"), its length, and its
//              number of deletion variants sum_{k<=min(d,L)} C(L, k).
//   k_expand : one warp per sequence; lane v builds variant v (0 deletions,
//              then every single deletion, then every pair, then every
//              triple, subsets in colexicographic order), fingerprints it and
//              writes the 64-bit record  fingerprint[63:b] | id[b-1:0]  at
//              rec_off[s] + v.  Consecutive lanes write consecutive records,
//              so every warp store is one contiguous 256-byte run.  The same
//              kernel accumulates the digit histograms of every radix pass
//              that will sort these records (one read of the data saved).
#include <algorithm>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

// 'A'..'Z' -> residue code (alphabetical order of the 20 one-letter codes),
// 0 for letters outside the alphabet.
__constant__ uint8_t c_letter_code[26] = {
    1,  0,  2,  3,  4,  5,  6,  7,  8, 0, 9,  10, 11,   // A B C D E F G H I J K L M
    12, 0, 13, 14, 15, 16, 17, 0, 18, 19, 0, 20, 0};     // N O P Q R S T U V W X Y Z

__global__ void k_encode(const uint8_t* __restrict__ seqs, const int64_t* __restrict__ off,
                         int64_t n, int d, Key128* __restrict__ keys, uint8_t* __restrict__ lens,
                         uint32_t* __restrict__ vcount, uint32_t* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t a = off[i], b = off[i + 1], total = off[n];
  Key128 k{0ull, 0ull};
  uint32_t L = 0;
  if (a < 0 || b < a || b > total) {
    atomicOr(err, DERR_RANGE);
  } else if (b - a > XTN_MAX_LEN) {
    atomicOr(err, DERR_TOO_LONG);
  } else {
    L = (uint32_t)(b - a);
    for (uint32_t p = 0; p < L; ++p) {
      const uint32_t ch = seqs[a + p];
      const uint32_t c = (ch >= 'A' && ch <= 'Z') ? c_letter_code[ch - 'A'] : 0u;
      if (c == 0) atomicOr(err, DERR_BAD_RESIDUE);
      const uint32_t m = 5 * p;
      if (m < 64) {
        k.lo |= (uint64_t)c << m;
        if (m > 59) k.hi |= (uint64_t)c >> (64 - m);
      } else {
        k.hi |= (uint64_t)c << (m - 64);
      }
    }
  }
  keys[i] = k;
  lens[i] = (uint8_t)L;
  vcount[i] = variant_count(L, (uint32_t)d);
}

constexpr int EXPAND_THREADS = 256;

__global__ void __launch_bounds__(EXPAND_THREADS)
    k_expand(const Key128* __restrict__ keys, const uint8_t* __restrict__ lens,
             const uint64_t* __restrict__ rec_off, int64_t n, const uint32_t* __restrict__ seq_rep,
             uint32_t id_bits, uint64_t* __restrict__ out, uint64_t n_rec,
             uint32_t* __restrict__ hist, int hist_lo, int hist_passes, int hist_hi,
             uint32_t* __restrict__ err) {
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  for (int k = threadIdx.x; k < hist_passes * RADIX; k += blockDim.x) s_hist[k] = 0;
  __syncthreads();
  const uint32_t lane = lane_id();
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t idmask = (id_bits >= 64) ? ~0ull : ((1ull << id_bits) - 1ull);
  for (int64_t s = warp0; s < n; s += n_warps) {
    const Key128 k = keys[s];
    const uint32_t L = lens[s];
    const uint64_t base = rec_off[s];
    uint32_t cnt = (uint32_t)(rec_off[s + 1] - base);
    if (base + cnt > n_rec) {
      if (lane == 0) atomicOr(err, DERR_RANGE);
      cnt = 0;
    }
    const uint64_t salt = seq_rep ? rep_salt(seq_rep[s]) : 0ull;
    for (uint32_t v = lane; v < cnt; v += 32) {
      const Key128 var = variant_of(k, L, v);
      const uint64_t rec = (fingerprint(var, salt) & ~idmask) | (uint64_t)s;
      out[base + v] = rec;
      for (int p = 0; p < hist_passes; ++p) {
        const int sh = hist_lo + 8 * p;
        const int bits = min(8, hist_hi - sh);
        atomicAdd(&s_hist[p * RADIX + (uint32_t)((rec >> sh) & ((1u << bits) - 1u))], 1u);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < hist_passes * RADIX; k += blockDim.x)
    if (s_hist[k]) atomicAdd(&hist[k], s_hist[k]);
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
                   uint8_t* lens, uint32_t* vcount, uint32_t* err, cudaStream_t s) {
  if (n <= 0) return;
  prof_begin(s, "k_encode", (double)n * (16 + 16 + 1 + 4 + 8));
  k_encode<<<div_up_u32(n, 256), 256, 0, s>>>(seqs, off, n, d, keys, lens, vcount, err);
  prof_end(s);
}

void launch_expand(const Key128* keys, const uint8_t* lens, const uint64_t* rec_off, int64_t n,
                   const uint32_t* seq_rep, uint32_t id_bits, uint64_t* out, uint64_t n_rec,
                   uint32_t* hist, int hist_lo, int hist_hi, int sms, uint32_t* err,
                   cudaStream_t s) {
  if (n <= 0) return;
  const int passes = (hist_hi - hist_lo + 7) / 8;
  const int64_t warps_needed = n;
  int blocks = (int)std::min<int64_t>((warps_needed + 7) / 8, (int64_t)sms * 8);
  if (blocks < 1) blocks = 1;
  prof_begin(s, "k_expand", (double)n_rec * 8.0 + (double)n * 25.0);
  k_expand<<<blocks, EXPAND_THREADS, 0, s>>>(keys, lens, rec_off, n, seq_rep, id_bits, out, n_rec,
                                             hist, hist_lo, passes, hist_hi, err);
  prof_end(s);
}

}  // namespace xtn
