// Paired chains (Discussion: the CDR3s of both chains joined by a
// non-deletable token).  A receptor is the string alpha + token + beta; its
// deletion variants delete up to d residues of either chain and never the
// token, and two receptors' distance is the edit distance of those strings
// with the token never deleted, inserted or substituted -- the two tokens
// always face each other, so the distance is Lev(alpha_i, alpha_j) +
// Lev(beta_i, beta_j) (computed in k_verify.cu, metric 2).
//
//   k_paired_counts : canonical variants per receptor (d <= 2): the token
//                     separates the chains, so the runs of equal residues
//                     are those of alpha plus those of beta, and the count
//                     is 1 + R + C(R, 2) + nD over both chains together.
//   k_expand_paired : one warp per receptor.  The lanes lay out the
//                     concatenated residue codes (token code 21), take the
//                     prefix sums of the polynomial fingerprint over all
//                     positions up to 51, list the run starts of both chains
//                     (never the token's position) and compute the canonical
//                     variants' fingerprints exactly as for one chain: the
//                     fingerprint is that of the variant string, token
//                     included, so equal receptor variants meet in one group.
#include <algorithm>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

namespace {

constexpr uint32_t TOKEN_CODE = 21;  // outside the residue codes 1..20
constexpr int PAIRED_MAX = 2 * XTN_MAX_LEN + 1;  // longest joined string
constexpr int PAIRED_WARPS = 8;

__device__ __forceinline__ uint32_t runs_of(uint32_t L, uint32_t eq) {
  const uint32_t all = L ? (0xffffffffu >> (32 - L)) : 0u;
  return ~eq & all;
}

// Canonical variants with at most d <= 2 deletions of a receptor.
__device__ __forceinline__ uint32_t paired_count(uint32_t La, uint32_t eqa, uint32_t Lb,
                                                 uint32_t eqb, int d) {
  const uint32_t ra = runs_of(La, eqa), rb = runs_of(Lb, eqb);
  const uint32_t R = (uint32_t)(__popc(ra) + __popc(rb));
  const uint32_t nD = (uint32_t)(__popc(ra & (eqa >> 1)) + __popc(rb & (eqb >> 1)));
  if (d <= 0) return 1u;
  if (d == 1) return 1u + R;
  return 1u + R + R * (R - 1) / 2 + nD;
}

__global__ void k_paired_counts(const uint8_t* __restrict__ lens_a,
                                const uint32_t* __restrict__ eq_a,
                                const uint8_t* __restrict__ lens_b,
                                const uint32_t* __restrict__ eq_b, int64_t n, int d,
                                uint32_t* __restrict__ vcount) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  vcount[i] = paired_count(min((uint32_t)lens_a[i], (uint32_t)XTN_MAX_LEN), eq_a[i],
                           min((uint32_t)lens_b[i], (uint32_t)XTN_MAX_LEN), eq_b[i], d);
}

struct PairedWarp {
  uint64_t P[PAIRED_MAX + 3];    // P[0 .. Lt + 2]
  uint8_t rs[PAIRED_MAX + 1];    // run starts (positions in the joined string)
  uint8_t ds[PAIRED_MAX + 1];    // starts of runs of length >= 2
};

// HIW: the histogram's digits lie in the record's high word (hist_lo >= 32).
// zero / n_zero: 16-byte words cleared for the record sort's status.
template <bool HIW>
__global__ void __launch_bounds__(PAIRED_WARPS * 32)
    k_expand_paired(const Key128* __restrict__ keys_a, const uint8_t* __restrict__ lens_a,
                    const uint32_t* __restrict__ eq_a, const Key128* __restrict__ keys_b,
                    const uint8_t* __restrict__ lens_b, const uint32_t* __restrict__ eq_b,
                    const uint64_t* __restrict__ rec_off, int64_t n, int d, uint32_t id_bits,
                    uint64_t* __restrict__ out, uint64_t n_rec, uint32_t* __restrict__ hist,
                    int hist_lo, int hist_passes, int hist_hi, uint32_t* __restrict__ err,
                    uint4* __restrict__ zero, uint64_t n_zero) {
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_zero;
       k += (uint64_t)gridDim.x * blockDim.x)
    zero[k] = make_uint4(0u, 0u, 0u, 0u);
  __shared__ uint64_t s_pow[64];
  __shared__ PairedWarp s_w[PAIRED_WARPS];
  for (int k = threadIdx.x; k < hist_passes * RADIX; k += blockDim.x) s_hist[k] = 0;
  for (int k = threadIdx.x; k < 64; k += blockDim.x) {
    uint64_t p = 1;
    for (int e = 0; e < k; ++e) p *= HASH_B;
    s_pow[k] = p;
  }
  __syncthreads();
  PairedWarp* w = &s_w[threadIdx.x >> 5];
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t idmask = (1ull << id_bits) - 1ull;
  const int last_bits = hist_hi - hist_lo - 8 * (hist_passes - 1);
  const uint32_t last_mask = (1u << last_bits) - 1u;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp0; r < n; r += n_warps) {
    const Key128 ka = keys_a[r], kb = keys_b[r];
    const uint32_t La = min((uint32_t)lens_a[r], (uint32_t)XTN_MAX_LEN);
    const uint32_t Lb = min((uint32_t)lens_b[r], (uint32_t)XTN_MAX_LEN);
    const uint32_t ea = eq_a[r], eb = eq_b[r];
    const uint32_t Lt = La + 1 + Lb;  // <= 51
    const uint64_t base = rec_off[r];
    const uint64_t cnt = rec_off[r + 1] - base;
    __syncwarp();  // the previous receptor's readers are done with w
    // residue code of joined position q
    auto code = [&](uint32_t q) -> uint32_t {
      if (q < La) return code_at(ka, (int)q);
      if (q == La) return TOKEN_CODE;
      return code_at(kb, (int)(q - La - 1));
    };
    // prefix sums over positions q = lane and q = 32 + lane
    const uint64_t t0 = lane < Lt ? (uint64_t)code(lane) * s_pow[lane] : 0ull;
    const uint64_t t1 = 32 + lane < Lt ? (uint64_t)code(32 + lane) * s_pow[32 + lane] : 0ull;
    const uint64_t i0 = warp_incl_scan_u64(t0);
    const uint64_t s0 = __shfl_sync(FULL_MASK, i0, 31);
    const uint64_t i1 = warp_incl_scan_u64(t1) + s0;
    const uint64_t PL = Lt <= 32 ? __shfl_sync(FULL_MASK, i0, (int)Lt - 1)
                                 : __shfl_sync(FULL_MASK, i1, (int)Lt - 33);
    // P[q + 1] for q < Lt, P[x] = P[Lt] up to Lt + 2
    for (uint32_t q = lane; q < Lt + 2; q += 32) {
      w->P[q + 1] = q < Lt ? (q < 32 ? i0 : i1) : PL;
    }
    if (lane == 0) w->P[0] = 0ull;
    // run starts of both chains as joined positions (alpha at q, beta at
    // La + 1 + q); the token is never a deletion
    const uint32_t ra = runs_of(La, ea), rb = runs_of(Lb, eb);
    const uint32_t da = ra & (ea >> 1), db = rb & (eb >> 1);
    const uint32_t Ra = (uint32_t)__popc(ra), Da = (uint32_t)__popc(da);
    if ((ra >> lane) & 1u) w->rs[__popc(ra & lt)] = (uint8_t)lane;
    if ((rb >> lane) & 1u) w->rs[Ra + __popc(rb & lt)] = (uint8_t)(La + 1 + lane);
    if ((da >> lane) & 1u) w->ds[__popc(da & lt)] = (uint8_t)lane;
    if ((db >> lane) & 1u) w->ds[Da + __popc(db & lt)] = (uint8_t)(La + 1 + lane);
    __syncwarp();
    const uint32_t R = Ra + (uint32_t)__popc(rb);
    uint32_t total = paired_count(La, ea, Lb, eb, d);
    if (total != cnt || base + cnt > n_rec) {
      if (lane == 0) atomicOr(err, DERR_RANGE);
      total = 0;
    }
    const uint32_t c2 = R * (R - 1) / 2;
    auto P = [&](uint32_t x) { return w->P[x]; };
    for (uint32_t v = lane; v < total; v += 32) {
      // canonical variant v: none, one run start, two run starts (colex
      // rank u = b(b-1)/2 + a, a < b), or the first two of a long run
      uint32_t p1 = Lt, p2 = Lt + 1;
      if (v >= 1 && v <= R) {
        p1 = w->rs[v - 1];
        p2 = Lt;
      } else if (v > R) {
        const uint32_t u = v - 1 - R;
        if (u < c2) {
          uint32_t b = (uint32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)u)) * 0.5f);
          while (b * (b - 1) / 2 > u) --b;
          while ((b + 1) * b / 2 <= u) ++b;
          const uint32_t a = u - b * (b - 1) / 2;
          p1 = w->rs[a];
          p2 = w->rs[b];
        } else {
          p1 = w->ds[u - c2];
          p2 = p1 + 1;
        }
      }
      const uint64_t h = P(p1) + HASH_BINV * ((P(p2) - P(p1 + 1)) + HASH_BINV * (P(Lt) - P(p2 + 1)));
      const uint64_t rec = (mix64(h) & ~idmask) | (uint64_t)r;
      out[base + v] = rec;
      if (HIW) {
        const uint32_t rr = (uint32_t)(rec >> 32) >> (hist_lo - 32);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (p < hist_passes) {
            const uint32_t m = p == hist_passes - 1 ? last_mask : 0xffu;
            atomicAdd(&s_hist[p * RADIX + ((rr >> (8 * p)) & m)], 1u);
          }
        }
      } else {
        const uint64_t rr = rec >> hist_lo;
#pragma unroll
        for (int p = 0; p < MAX_PASSES; ++p) {
          if (p < hist_passes) {
            const uint32_t m = p == hist_passes - 1 ? last_mask : 0xffu;
            atomicAdd(&s_hist[p * RADIX + ((uint32_t)(rr >> (8 * p)) & m)], 1u);
          }
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < hist_passes * RADIX; k += blockDim.x)
    if (s_hist[k]) atomicAdd(&hist[k], s_hist[k]);
}

}  // namespace

void launch_paired_counts(const uint8_t* lens_a, const uint32_t* eq_a, const uint8_t* lens_b,
                          const uint32_t* eq_b, int64_t n, int d, uint32_t* vcount,
                          cudaStream_t s) {
  if (n <= 0) return;
  prof_begin(s, "k_paired_counts", (double)n * 14.0);
  k_paired_counts<<<div_up_u32(n, 256), 256, 0, s>>>(lens_a, eq_a, lens_b, eq_b, n, d, vcount);
  prof_end(s);
}

void launch_expand_paired(const Key128* keys_a, const uint8_t* lens_a, const uint32_t* eq_a,
                          const Key128* keys_b, const uint8_t* lens_b, const uint32_t* eq_b,
                          const uint64_t* rec_off, int64_t n, int d, uint32_t id_bits,
                          uint64_t* out, uint64_t n_rec, uint32_t* hist, int hist_lo, int hist_hi,
                          int sms, uint32_t* err, cudaStream_t s, void* zero,
                          size_t zero_bytes) {
  if (n <= 0) return;
  const int passes = (hist_hi - hist_lo + 7) / 8;
  const int blocks = (int)std::min<int64_t>((n + PAIRED_WARPS - 1) / PAIRED_WARPS,
                                            (int64_t)sms * 8);
  prof_begin(s, "k_expand_paired", (double)n_rec * 8.0 + (double)n * 58.0);
  auto f = hist_lo >= 32 && hist_hi <= 64 ? k_expand_paired<true> : k_expand_paired<false>;
  f<<<blocks > 0 ? blocks : 1, PAIRED_WARPS * 32, 0, s>>>(
      keys_a, lens_a, eq_a, keys_b, lens_b, eq_b, rec_off, n, d, id_bits, out, n_rec, hist,
      hist_lo, passes, hist_hi, err, static_cast<uint4*>(zero), zero ? zero_bytes / 16 : 0);
  prof_end(s);
}

}  // namespace xtn
