// Host-side launchers of the sm_103a kernels (one translation unit each) and
// the constants they share.  All launches are asynchronous on stream `s`.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <stdint.h>

#include "xtn.h"

namespace xtn {

struct Key128;

constexpr int RADIX = 256;       // 8-bit digits
constexpr int MAX_PASSES = 8;    // 64-bit keys
constexpr int PEQ_STRIDE = 20;   // match vectors per sequence (one per residue code)

// api.cu: tuning knobs
std::atomic<int>& cfg_records();
std::atomic<int>& cfg_pairs();

// k_variants.cu ------------------------------------------------------------
void launch_encode(const uint8_t* seqs, const int64_t* off, int64_t n, int d, Key128* keys,
                   uint8_t* lens, uint32_t* eqprev, uint32_t* vcount, uint32_t* err,
                   cudaStream_t s);
// Record selection by fingerprint bin, bin = (record >> shift) & mask, for
// searches that take the records in several passes.  With `append` null the
// expand kernel only counts records per bin into bin_count[0 .. mask] (mask
// < 2048) and writes nothing; otherwise it appends the records whose bin lies
// in [lo, hi) to out[0, n_rec), counting them in *append.
enum { SEL_ALL = 0, SEL_COUNT = 1, SEL_APPEND = 2 };
struct BinSel {
  uint32_t shift = 0, mask = 0;
  uint32_t lo = 0, hi = 0;
  uint32_t* bin_count = nullptr;
  unsigned long long* append = nullptr;
};
constexpr int MAX_BIN_BITS = 11;

// sel null: every record of sequence i goes to out[rec_off[i] ...].
// zero: when not null, zero_bytes (a multiple of 16, 16-byte aligned) are
// cleared there as well (the record sort's look-back status).
void launch_expand(const Key128* keys, const uint8_t* lens, const uint32_t* eqprev,
                   const uint64_t* rec_off, int64_t n, int d, const uint32_t* seq_rep,
                   uint32_t id_bits, uint64_t* out, uint64_t n_rec, uint32_t* hist, int hist_lo,
                   int hist_hi, int sms, uint32_t* err, cudaStream_t s,
                   const BinSel* sel = nullptr, void* zero = nullptr, size_t zero_bytes = 0);
void launch_peq(const Key128* keys, const uint8_t* lens, int64_t n, uint32_t* peq,
                cudaStream_t s);
void launch_seq_rep(const int64_t* rep_off, int64_t n_rep, uint32_t* seq_rep, int64_t n,
                    cudaStream_t s);

// k_radix.cu ---------------------------------------------------------------
int onesweep_tile(int cfg);
int onesweep_configs();
size_t radix_status_bytes(int64_t n, int cfg);
void launch_histogram(const uint64_t* keys, int64_t n, int lo, int hi, uint32_t* hist, int sms,
                      cudaStream_t s);
// Sorts a[0:n) on bits [lo, hi) using b as the second buffer; `hist` holds the
// digit histograms of every pass.  *sorted receives a or b.
// hist_in_passes: `hist` holds only pass 0's digit counts; every pass counts
// the next pass's digits itself (zeroed hist rows 1.. expected).
// n_dev: when not null the key count is read on the device (n is then a
// capacity that sizes the grid and the look-back status).
// bucket_start: when not null (2^(hi-lo) entries, all bits set on entry), the
// last pass leaves in bucket_start[b] the first sorted position whose bits
// [lo, hi) equal b; buckets without records keep all bits set.
// first_cfg: configuration of the first pass (>= 0), e.g. the unstable one;
// LSD order needs only the later passes to be stable.  Ignored when its tile
// differs from cfg's.
// status_zeroed: the whole status area (radix_status_bytes) is zero on entry,
// so the first two passes need no clearing.
cudaError_t radix_sort_passes(uint64_t* a, uint64_t* b, int64_t n, int lo, int hi, uint32_t* hist,
                              uint64_t* digit_base, uint64_t* status, int cfg, uint32_t* err,
                              uint64_t** sorted, const char* tag, cudaStream_t s,
                              bool hist_in_passes = false, const uint64_t* n_dev = nullptr,
                              uint64_t* bucket_start = nullptr, int first_cfg = -1,
                              bool status_zeroed = false);
// Unstable configuration with the same tile as cfg, for a sort's first pass.
int onesweep_unstable_config(int cfg);

// k_bucket.cu --------------------------------------------------------------
// Positions per flag tile of the group-bound kernels (head/tail counts are
// kept per tile of this many sorted records).
constexpr int GROUP_FLAG_TILE = 32768;
// Split of the hs group-key bits: the top G are sorted by global radix
// passes (bucket = those bits), the low L = hs - G in shared memory, 2^kbits
// buckets per block.  G depends only on (n_rec, hs); kbits also on the
// shared-memory step (hash grouping or sort).
struct GroupingShape {
  int G = 0, L = 0, kbits = 0;
};
GroupingShape choose_grouping(uint64_t n_rec, int hs, bool hash);
int bucket_capacity(bool hash);
// A holds n records sorted on their top G group-key bits (bits [lo + L, 64)),
// bucket_start as left by radix_sort_passes (unused when G == 0).  Writes the
// records to Y (A is scratch afterwards): with `hash`, every group's records
// contiguous in arbitrary order; without, sorted on all group-key bits.
// With `flags` (zeroed, group_flag_words(n)) and `tile_counts` (zeroed, one
// per GROUP_FLAG_TILE positions) also the head/tail flags k_group_write
// reads.  cap: records per shared-memory segment (0 = the full capacity).
// With `cand` (hash only): buckets that fit a segment write no records and no
// flags but append their candidate pair words (min id << id_bits | max id)
// to cand[0, cand_cap), counting them in cand_count[0] (DERR_CAPACITY past
// the capacity); larger buckets go the flag route as before and add their
// record count to cand_count[1].
// seg_list / seg_count: when given, only the *seg_count blocks of buckets
// listed (the ones k_bucket_filter left), by a grid of sms x 5 blocks.
void launch_bucket(bool hash, uint64_t* A, uint64_t* Y, int64_t n, const uint64_t* n_dev,
                   const uint64_t* bucket_start, const GroupingShape& g, int lo, int cap,
                   uint64_t* flags, uint64_t* tile_counts, uint64_t* cand, uint64_t cand_cap,
                   uint64_t* cand_count, int id_bits, uint32_t* err, cudaStream_t s,
                   const uint32_t* seg_list = nullptr, const uint32_t* seg_count = nullptr,
                   int sms = 0);
// k_filter.cu --------------------------------------------------------------
// Candidate mode of the grouping for the buckets of shape g (G global bits):
// each block takes 2^(kbits + fx) buckets, keeps only the records whose group
// key occurs twice or more (two bitmaps), groups those exactly in shared
// memory and appends their pairs to cand as k_bucket does.  A block whose
// kept records overflow appends the k_bucket blocks it covers to seg_list
// (counted in *seg_count, zeroed; room for every k_bucket block), for
// launch_bucket(..., seg_list, seg_count).
void launch_bucket_filter(const uint64_t* A, int64_t n, const uint64_t* n_dev,
                          const uint64_t* bucket_start, const GroupingShape& g, int fx, int lo,
                          uint64_t* cand, uint64_t cand_cap, uint64_t* cand_count, int id_bits,
                          uint32_t* seg_list, uint32_t* seg_count, uint32_t* err, cudaStream_t s);
// k_pairs.cu ---------------------------------------------------------------
size_t scan_status_bytes(int64_t n);
size_t group_status_bytes(int64_t n);
void launch_scan_counts(const uint32_t* counts, int64_t n, uint64_t* out, uint64_t* status,
                        uint32_t* err, cudaStream_t s);
void launch_scan_group_pairs(const uint32_t* S, const uint32_t* E, int64_t n_groups,
                             const uint64_t* n_groups_dev, uint64_t* out, uint64_t* status,
                             uint32_t* err, cudaStream_t s);
size_t group_flag_words(int64_t n);
// Group bounds = flags (k_group_flags, or k_bucket_sort) + finish (tile
// prefix, k_group_write, group count).  `status` holds group_status_bytes(n).
void launch_group_bounds(const uint64_t* keys, int64_t n, const uint64_t* n_dev, int gshift,
                         uint32_t* S, uint32_t* E, uint64_t cap, uint64_t* flags,
                         uint64_t* status, uint32_t* err, uint64_t* n_groups, cudaStream_t s);
uint64_t* group_tile_counts(uint64_t* status, int64_t n);
void launch_group_flags(const uint64_t* keys, int64_t n, const uint64_t* n_dev, int gshift,
                        uint64_t* flags, uint64_t* status, cudaStream_t s);
void launch_group_finish(const uint64_t* flags, int64_t n, const uint64_t* n_dev, uint32_t* S,
                         uint32_t* E, uint64_t cap, uint64_t* status, uint32_t* err,
                         uint64_t* n_groups, cudaStream_t s);
// Candidate words of the groups [S, E] into out[base + t], t < pairs of the
// groups, base = *out_base (0 when null); *n_pairs_out = base + pairs.
void launch_emit_pairs(const uint64_t* keys, uint64_t n_keys, const uint32_t* S,
                       const uint64_t* pair_off, int64_t n_groups, const uint64_t* n_groups_dev,
                       uint64_t pair_cap, uint32_t id_bits, uint64_t* out,
                       const uint64_t* out_base, uint64_t* n_pairs_out, int sms, uint32_t* err,
                       cudaStream_t s);

// k_verify.cu --------------------------------------------------------------
// Rows per tile of the verify, dedup and TCRdist kernels, and the look-back
// status those kernels need for n rows (one word per tile plus a tile counter).
constexpr int VERIFY_TILE = 2048;
constexpr size_t verify_status_bytes_for(int64_t n) {
  return (size_t)((n + VERIFY_TILE - 1) / VERIFY_TILE) * 8 + 16;
}
// Second chains of paired receptors (metric 2, the sum of the two chains'
// edit distances): match vectors of the i side, keys of the j side and both
// sides' lengths.  All null for one chain.
struct SecondChain {
  const uint32_t* peq_i = nullptr;
  const uint8_t* lens_i = nullptr;
  const Key128* keys_j = nullptr;
  const uint8_t* lens_j = nullptr;
};
// metric: 0 = Levenshtein, 1 = Hamming (pairs of equal length only), 2 =
// paired chains (Levenshtein of the first chains plus that of the second,
// which `sc` describes).  Verify writes a survivor's distance into bits
// [hist_hi, hist_hi + 8) of its word when they exist (hist_hi + 8 <= 64);
// the dedup then reads it there (dist_shift = hist_hi) instead of computing
// it again (dist_shift = 0).
// self_mode: 0 = query vs reference, 1 = self-search (pairs within a
// repertoire when seq_rep is given), 2 = self-search keeping only pairs
// between different repertoires.
size_t verify_status_bytes(int64_t n);
void launch_verify_candidates(const uint64_t* cand, uint64_t n, const uint64_t* n_dev,
                              uint32_t j_bits,
                              const uint32_t* peq_i, const uint8_t* lens_i, uint64_t n_i,
                              const Key128* keys_j, const uint8_t* lens_j, uint64_t n_j,
                              const uint32_t* seq_rep, int self_mode, int d, int metric,
                              uint64_t* surv, uint64_t surv_cap, uint64_t* n_surv, uint32_t* hist,
                              int hist_hi, int sms, uint32_t* err, cudaStream_t s,
                              const SecondChain& sc = SecondChain());
void launch_unique_finalize(const uint64_t* pairs, int64_t n, const uint64_t* n_dev,
                            uint32_t j_bits,
                            const uint32_t* peq_i, const uint8_t* lens_i, uint64_t n_i,
                            const Key128* keys_j, const uint8_t* lens_j, uint64_t n_j,
                            int metric, xtn_triple* out, int64_t cap, uint64_t* status,
                            uint32_t* err, uint64_t* total, cudaStream_t s,
                            const SecondChain& sc = SecondChain(), int dist_shift = 0);
void launch_tcrdist_filter(const xtn_triple* in, int64_t n, const Key128* keys,
                           const uint8_t* lens, int64_t n_seq, int max_score, xtn_triple* out,
                           uint64_t* status, uint32_t* err, uint64_t* total, cudaStream_t s);

// k_paired.cu --------------------------------------------------------------
// Canonical deletion variants (d <= 2) of receptors alpha + token + beta,
// the token never deleted: counts per receptor, and the expansion into
// records fingerprint | receptor id at rec_off (digit histograms of the sort
// passes over bits [hist_lo, hist_hi) on the way).
void launch_paired_counts(const uint8_t* lens_a, const uint32_t* eq_a, const uint8_t* lens_b,
                          const uint32_t* eq_b, int64_t n, int d, uint32_t* vcount,
                          cudaStream_t s);
void launch_expand_paired(const Key128* keys_a, const uint8_t* lens_a, const uint32_t* eq_a,
                          const Key128* keys_b, const uint8_t* lens_b, const uint32_t* eq_b,
                          const uint64_t* rec_off, int64_t n, int d, uint32_t id_bits,
                          uint64_t* out, uint64_t n_rec, uint32_t* hist, int hist_lo, int hist_hi,
                          int sms, uint32_t* err, cudaStream_t s, void* zero = nullptr,
                          size_t zero_bytes = 0);

// k_query.cu ---------------------------------------------------------------
// Directory of the sorted index (entry t = first record whose top dir_bits
// bits are >= t) and, added into *n_groups, the number of distinct group keys
// (bits from gshift up).
void launch_build_dir(const uint64_t* rec, uint64_t n_rec, int dir_bits, int gshift,
                      uint32_t* dir, uint64_t* n_groups, cudaStream_t s);
void launch_query_lookup(const Key128* qkeys, const uint8_t* qlens, const uint32_t* qeqprev,
                         const uint64_t* q_rec_off, int64_t n_q, uint64_t n_qv, int d,
                         const uint64_t* rec, uint64_t n_rec, const uint32_t* dir,
                         int dir_bits, int gshift, uint32_t* qv_start, uint32_t* qv_cnt,
                         uint32_t* qv_q, int sms, uint32_t* err, cudaStream_t s);
void launch_query_emit(const uint64_t* rec, uint64_t n_rec, uint32_t ref_bits,
                       const uint32_t* qv_start, const uint32_t* qv_q, const uint64_t* cand_off,
                       uint64_t n_qv, uint64_t n_cand, uint64_t* out, int sms, uint32_t* err,
                       cudaStream_t s);

}  // namespace xtn
