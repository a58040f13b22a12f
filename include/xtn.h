/*
 * xtn.h -- C ABI of the GB300 (sm_103a) symmetric-deletion neighbour search.
 *
 * The library finds every pair of amino-acid sequences within Levenshtein
 * distance d by symmetric deletion lookup (XTNeighbor, arXiv 2403.09010):
 * expand each sequence into its deletion variants with up to d deletions
 * (Appendix A, "XTNeighbor algorithm step-by-step", steps 1-3), group equal
 * variants (step 4), emit the index pairs that share a variant (step 5),
 * remove duplicate pairs (step 6) and keep the pairs whose exact edit
 * distance is <= d (step 7).  Every step runs in the library's own CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Sequences are passed packed: `seqs` holds the ASCII letters of all
 *   sequences back to back (no separators, no terminator) and `offsets[k]`
 *   .. `offsets[k+1]` delimit sequence k (`offsets` has n+1 entries,
 *   offsets[0] = 0, non-decreasing).  Letters must be upper-case one-letter
 *   amino-acid codes from "ACDEFGHIKLMNPQRSTVWY"; sequence lengths must be in
 *   [0, XTN_MAX_LEN].  The paper packs 5 bits per residue into 12 bytes
 *   (<= 18 residues, Appendix "Compression of TCR sequences"); this library
 *   packs them into 16 bytes and so admits up to 25.
 * - Every pointer argument except `n_out` and the index handle may be a host
 *   pointer or a device pointer of the current CUDA device; the library
 *   inspects it (cudaPointerGetAttributes) and copies pageable host data to
 *   and from the device itself.  The xtn_search_* calls read pinned host
 *   sequences and offsets (cudaHostAlloc / cudaHostRegister) in place from
 *   their first kernel and write rows into a pinned host buffer in place,
 *   without a staging copy.  The caller owns all buffers it passes.
 *   `n_out` is always a host pointer.
 * - `stream` is a cudaStream_t (NULL = the legacy default stream).  Kernels
 *   and copies are issued on it; every call returns only after the stream has
 *   finished the call's work, because the result count is read back.
 *   Scratch memory is carved from a per-device cache of device blocks that
 *   calls take and give back (see xtn_scratch_trim); only a call that needs
 *   more than its block holds allocates the rest from the device's
 *   stream-ordered pool (cudaMallocAsync), and the block grows to that size
 *   the next time it is taken.
 * - Output rows are `xtn_triple {i, j, dist}` sorted ascending by (i, j),
 *   without duplicates.  `*n_out` always receives the exact number of rows of
 *   the full result.  If it exceeds `cap`, the first `cap` rows are written
 *   and XTN_ERR_BUFFER_TOO_SMALL is returned; call again with a larger buffer.
 * - Every function returns XTN_OK (0) or a negative status; see
 *   xtn_status_string().  On an error no output row is guaranteed.
 */
#ifndef XTN_H_
#define XTN_H_

#include <stdint.h>

#if defined(__GNUC__)
#define XTN_API __attribute__((visibility("default")))
#else
#define XTN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream. */
typedef struct CUstream_st* xtn_stream_t;

/* One neighbour pair.  Self-search: i < j are sequence indices.  Batched
 * self-search: i < j index the concatenation of all repertoires and always
 * fall in the same repertoire.  Query search: i is the query index, j the
 * reference index.  dist is the Levenshtein distance, 0 <= dist <= d. */
typedef struct {
  uint32_t i;
  uint32_t j;
  uint32_t dist;
} xtn_triple;

/* Device-resident deletion-variant index of a reference set (opaque). */
typedef struct xtn_index xtn_index;

#define XTN_MAX_LEN 25 /* longest admissible sequence */
#define XTN_MAX_D 3    /* largest admissible distance threshold */

enum {
  XTN_OK = 0,
  XTN_ERR_INVALID_ARG = -1,      /* bad size, pointer or d */
  XTN_ERR_BAD_RESIDUE = -2,      /* a letter outside the 20-letter alphabet */
  XTN_ERR_SEQ_TOO_LONG = -3,     /* a sequence longer than XTN_MAX_LEN */
  XTN_ERR_OOM = -4,              /* device memory could not be allocated */
  XTN_ERR_BUFFER_TOO_SMALL = -5, /* *n_out > cap; first cap rows written */
  XTN_ERR_CUDA = -6,             /* a CUDA runtime call failed */
  XTN_ERR_DEVICE_TIMEOUT = -7,   /* a bounded device-side wait gave up */
  XTN_ERR_TOO_LARGE = -8,        /* more than 2^32-1 variant records or pairs */
  XTN_ERR_CAPACITY = -9          /* a plan's candidate-pair capacity was exceeded */
};

/* Human-readable name of a status code (static string, never NULL). */
XTN_API const char* xtn_status_string(int status);

/* Library version as 10000*major + 100*minor + patch. */
XTN_API int xtn_version(void);

/*
 * All-pairs self-search (Appendix A, XTNeighbor steps 0-7).
 *   seqs, offsets, n : the n input sequences (see conventions above).
 *   d                : distance threshold, 0 <= d <= XTN_MAX_D.
 *   rep_offsets      : NULL for one repertoire.  Otherwise n_rep+1
 *                      non-decreasing int64 entries with rep_offsets[0] = 0
 *                      and rep_offsets[n_rep] = n: the sequences
 *                      [rep_offsets[r], rep_offsets[r+1]) form repertoire r
 *                      and pairs are only reported within a repertoire
 *                      (batched mode; indices stay global).
 *   n_rep            : number of repertoires (ignored when rep_offsets is
 *                      NULL; must be >= 1 otherwise).
 *   out, cap         : output rows and their capacity (out may be NULL when
 *                      cap == 0, to learn the count).
 *   n_out            : host; receives the exact number of result rows.
 * Scratch comes from the scratch cache (see xtn_scratch_trim) and is given
 * back before the call returns; the call synchronises the stream three times
 * (record count, candidate count, row count).  With the default grouping the
 * candidate buffer is sized at half the record count before grouping; an
 * input that needs more (thousands of copies of one sequence) is searched
 * again with all-global grouping, which sizes it exactly, so the result is
 * the same, only slower.
 * Errors: INVALID_ARG, BAD_RESIDUE, SEQ_TOO_LONG, OOM, BUFFER_TOO_SMALL,
 * CUDA, DEVICE_TIMEOUT, TOO_LARGE.  An input with 2^32 variant records or more,
 * or 2^32 candidate pairs or more, is searched in passes as
 * xtn_search_self_streaming does with max_pass_records = 0.
 */
XTN_API int xtn_search_self(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                    const int64_t* rep_offsets, int64_t n_rep, xtn_triple* out, int64_t cap,
                    int64_t* n_out, xtn_stream_t stream);

/*
 * The Hamming variant of the self-search (Results, comparison with
 * CompAIRR): the same symmetric-deletion candidates, the last step filtering
 * by Hamming distance instead.  Rows are {i, j, dist} with i < j, equal
 * lengths and dist = the number of differing positions <= d, sorted by
 * (i, j); sequences of different lengths are never neighbours.  Two
 * sequences with h <= d differing positions share the string left after
 * deleting those positions, so no neighbour is missed.  Arguments, batched
 * mode and errors as xtn_search_self.
 */
XTN_API int xtn_search_self_hamming(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                                    const int64_t* rep_offsets, int64_t n_rep, xtn_triple* out,
                                    int64_t cap, int64_t* n_out, xtn_stream_t stream);

/*
 * Pairs between repertoires (Results, comparison with CompAIRR: the
 * repertoire-overlap workload).  Rows are {i, j, dist} with i < j global
 * indices, i and j in different repertoires, dist = Levenshtein distance
 * (metric XTN_METRIC_LEVENSHTEIN) or Hamming distance (XTN_METRIC_HAMMING,
 * equal lengths only) <= d, sorted by (i, j).  The search is the self-search
 * of the concatenated repertoires (Appendix A, XTNeighbor steps 0-7) whose
 * last step keeps a pair only when its repertoires differ: together with the
 * rows of xtn_search_self's batched mode these are exactly the rows of one
 * self-search over all sequences.  rep_offsets (required, n_rep >= 1) as in
 * xtn_search_self; other arguments and errors as xtn_search_self, plus
 * INVALID_ARG for a NULL rep_offsets or an unknown metric.
 */
#define XTN_METRIC_LEVENSHTEIN 0
#define XTN_METRIC_HAMMING 1
XTN_API int xtn_search_between(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                               const int64_t* rep_offsets, int64_t n_rep, int metric,
                               xtn_triple* out, int64_t cap, int64_t* n_out, xtn_stream_t stream);

/*
 * Paired-chain self-search (Discussion: the CDR3s of both chains joined by a
 * non-deletable token).  Receptor k is the pair (alpha_k, beta_k): alpha_k
 * delimited by a_offsets[k] .. a_offsets[k+1] in a_seqs, beta_k by b_offsets
 * in b_seqs (both offset arrays have n+1 entries; either chain may be empty;
 * each at most XTN_MAX_LEN residues).  Each receptor stands for the string
 * alpha + token + beta whose deletion variants delete up to d residues and
 * never the token; the distance of two receptors is the edit distance of
 * those strings with the token never deleted, inserted or substituted, which
 * equals Lev(alpha_i, alpha_j) + Lev(beta_i, beta_j).  Rows are {i, j, dist}
 * with i < j and dist <= d, sorted by (i, j).  0 <= d <= 2.
 * Other arguments as xtn_search_self (one repertoire).  Errors: as
 * xtn_search_self; INVALID_ARG for d > 2 or a NULL b_offsets; TOO_LARGE
 * for 2^32 variant records or candidate pairs or more (no search in passes).
 */
XTN_API int xtn_search_paired(const uint8_t* a_seqs, const int64_t* a_offsets,
                              const uint8_t* b_seqs, const int64_t* b_offsets, int64_t n, int d,
                              xtn_triple* out, int64_t cap, int64_t* n_out, xtn_stream_t stream);

/*
 * The self-search in passes, for inputs whose variant records do not fit the
 * device at once (Sec. 2.3, "Overcoming memory bottlenecks"; Appendix A,
 * XTNeighbor-streaming).  A first expansion only counts the records of each
 * of 2048 bins of the variant fingerprint.  Next-Fit packs consecutive bins
 * into passes of at most max_pass_records records (a bin larger than that is
 * a pass of its own).  Each pass expands only its bins' records, groups them,
 * and emits and verifies their candidate pairs.  Equal variants fall in one
 * bin, so no neighbour is missed.  Verified pairs of all passes are kept and
 * sorted once at the end, which drops pairs found in several passes.  A pass
 * whose candidate pairs exceed 2^32 words or device memory is split in two.
 * The rows are those of xtn_search_self (metric 0), xtn_search_self_hamming
 * (metric 1) or xtn_search_between (between != 0).
 *   max_pass_records : records per pass; <= 0 takes what fits in half the
 *                      free device memory (about 32 bytes per record).
 *   n_passes         : host, may be NULL; receives the passes run.
 * Other arguments as xtn_search_self.  Device memory: the sequences and
 * their match vectors, buffers for the largest pass, and the verified pairs.
 * Errors: as xtn_search_self; INVALID_ARG for an unknown metric, or for
 * between != 0 without rep_offsets.
 */
XTN_API int xtn_search_self_streaming(const uint8_t* seqs, const int64_t* offsets, int64_t n,
                                      int d, const int64_t* rep_offsets, int64_t n_rep, int metric,
                                      int between, int64_t max_pass_records, xtn_triple* out,
                                      int64_t cap, int64_t* n_out, int64_t* n_passes,
                                      xtn_stream_t stream);

/*
 * Build a device-resident index of a reference set: its encoded sequences
 * and its deletion variants, grouped by sorting (Appendix A, XTNeighbor steps
 * 1-4; the paper's multi-value hash map of the SymDel step list, realised as a
 * sorted array as Sec. 2.2 describes).  The index owns its device memory
 * until xtn_index_free(); it is tied to the current device and may be used
 * from any stream of it.  *out receives the handle.
 * Errors: INVALID_ARG, BAD_RESIDUE, SEQ_TOO_LONG, OOM, CUDA, DEVICE_TIMEOUT,
 * TOO_LARGE.
 */
XTN_API int xtn_index_build(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                    xtn_stream_t stream, xtn_index** out);

/* Release an index (NULL is accepted). */
XTN_API int xtn_index_free(xtn_index* idx);

/* Host-side facts about an index; any output pointer may be NULL. */
XTN_API int xtn_index_info(const xtn_index* idx, int64_t* n, int* d, int64_t* n_records,
                   int64_t* device_bytes);

/*
 * Query-vs-reference search (SymDel step 3 with the queries' own variants,
 * the fuzzy database lookup of the Discussion): every (q, r) with
 * Lev(query q, reference r) <= d, the d the index was built with.
 * Rows are {i = q, j = r, dist}, sorted by (q, r).  Several calls may run
 * concurrently on different streams against the same index.
 * Errors: INVALID_ARG, BAD_RESIDUE, SEQ_TOO_LONG, OOM, BUFFER_TOO_SMALL,
 * CUDA, DEVICE_TIMEOUT, TOO_LARGE.
 */
XTN_API int xtn_search_query(const xtn_index* idx, const uint8_t* q_seqs, const int64_t* q_offsets,
                     int64_t n_q, xtn_triple* out, int64_t cap, int64_t* n_out,
                     xtn_stream_t stream);

/*
 * Scratch estimate of a query search, for admission control of query
 * batches: *bytes receives the device bytes xtn_search_query (or its Hamming
 * variant) takes for n_q queries with these offsets (a host pointer, n_q+1
 * entries; the letters are not needed), counting host input and output
 * buffers.  The part set by the queries' lengths is an upper bound (every
 * deletion subset of at most d positions); the candidate part is estimated
 * from the candidates per query variant this index has produced in the
 * searches so far (before any: its mean number of records per variant
 * fingerprint), with a margin of 1.5x.  The call only reads host memory.
 * Errors: INVALID_ARG, SEQ_TOO_LONG.
 */
XTN_API int xtn_search_query_scratch(const xtn_index* idx, const int64_t* q_offsets, int64_t n_q,
                                     int64_t* bytes);

/*
 * The Hamming variant of the query search (Results, comparison with
 * CompAIRR): the same candidates from the index, the last step filtering by
 * Hamming distance.  Rows are {q, r, dist} with equal lengths and dist = the
 * number of differing positions <= d (the index's d), sorted by (q, r).
 * Arguments and errors as xtn_search_query.
 */
XTN_API int xtn_search_query_hamming(const xtn_index* idx, const uint8_t* q_seqs,
                                     const int64_t* q_offsets, int64_t n_q, xtn_triple* out,
                                     int64_t cap, int64_t* n_out, xtn_stream_t stream);

/*
 * TCRdist post-filter of neighbour rows (Results, "SymDel lookup can be
 * combined with more advanced similarity metrics").  For each input row
 * {i, j, dist} the score of sequences i and j is computed as: with m the
 * shorter length and g = |len_i - len_j|, the g gaps sit in the shorter
 * sequence after its first floor(m/2) residues; each aligned position costs
 * 0 if the residues agree, else min(4, 4 - BLOSUM62[a][b]); each gap costs
 * 4; the sum is multiplied by 3.  Rows with score <= max_score are written
 * to `out` in input order (out must hold n_in rows).
 *   seqs, offsets, n : the sequences the row indices refer to.
 *   in, n_in         : input rows (i, j < n).
 * Errors: INVALID_ARG, BAD_RESIDUE, SEQ_TOO_LONG, OOM, CUDA.
 */
XTN_API int xtn_tcrdist_filter(const uint8_t* seqs, const int64_t* offsets, int64_t n,
                       const xtn_triple* in, int64_t n_in, int max_score, xtn_triple* out,
                       int64_t* n_out, xtn_stream_t stream);

/*
 * Planned self-search: all device memory is allocated once, so that running
 * the search issues only kernels and memsets on one stream, with no host
 * synchronisation -- the sequence a CUDA graph can capture and replay.  This
 * is the batched mode of the library: any number of repertoires of uneven
 * size (rep_offsets as in xtn_search_self) go through one launch of each
 * kernel (Appendix A, XTNeighbor steps 0-7, over all repertoires at once).
 *
 * xtn_plan_create: plan for inputs with exactly these offsets (host or
 *   device, n+1 entries) and repertoire offsets (NULL for one repertoire).
 *   Record buffers are sized for every deletion subset of every sequence, an
 *   upper bound whatever the letters.  pair_capacity bounds the candidate
 *   pairs of one run (<= 0: one eighth of the record bound, at least 65,536).
 * xtn_plan_run: search the n sequences at `seqs` (a device pointer; letters
 *   laid out as the plan's offsets say) on `stream`; returns once the work is
 *   queued.  Runs on one plan must not overlap.
 * xtn_plan_result: wait for the stream and copy the rows of the last run to
 *   out (host or device, capacity cap); *n_out = number of rows.  If the run
 *   produced more candidate pairs than the plan holds, returns
 *   XTN_ERR_CAPACITY with *n_out = the capacity needed; create a plan with at
 *   least that pair_capacity.
 * Errors: INVALID_ARG, SEQ_TOO_LONG, OOM, CUDA, TOO_LARGE at creation;
 *   BAD_RESIDUE, DEVICE_TIMEOUT, CAPACITY, BUFFER_TOO_SMALL at result.
 */
typedef struct xtn_plan xtn_plan;
XTN_API int xtn_plan_create(const int64_t* offsets, int64_t n, int d, const int64_t* rep_offsets,
                    int64_t n_rep, int64_t pair_capacity, xtn_plan** out);
XTN_API int xtn_plan_run(xtn_plan* plan, const uint8_t* seqs, xtn_stream_t stream);
XTN_API int xtn_plan_result(xtn_plan* plan, xtn_triple* out, int64_t cap, int64_t* n_out,
                    xtn_stream_t stream);
XTN_API int xtn_plan_info(const xtn_plan* plan, int64_t* record_capacity, int64_t* pair_capacity,
                  int64_t* device_bytes);
/* Counts of the last run (waits for `stream`): variant records, groups of
 * two or more records, candidate pairs, verified pair words (before dedup);
 * any output pointer may be NULL. */
XTN_API int xtn_plan_stats(xtn_plan* plan, int64_t* records, int64_t* groups, int64_t* candidates,
                   int64_t* survivors, xtn_stream_t stream);
XTN_API int xtn_plan_free(xtn_plan* plan);

/*
 * xtn_tcrdist_filter_noalloc: xtn_tcrdist_filter for callers that cannot
 * allocate device memory -- a process that must stay inside a fixed
 * device-memory budget, or a library loaded into a host application whose
 * own allocator owns the device memory, where an allocation of ours could
 * fail or take memory the host application counted on.  The paper has no
 * counterpart to this entry point; it computes exactly what
 * xtn_tcrdist_filter computes.
 *   - It allocates nothing: its scratch (encoded sequences, look-back status,
 *     counters) lives in one fixed array of about 6.3 MiB of device memory
 *     that every GPU loading the library holds until the process exits.
 *   - Limits: n <= XTN_NOALLOC_MAX_SEQS sequences and n_in <=
 *     XTN_NOALLOC_MAX_ROWS rows; larger inputs return XTN_ERR_TOO_LARGE.
 *   - seqs, offsets, in and out must be device pointers of the current
 *     device, or managed memory (a host buffer would need a device copy);
 *     otherwise XTN_ERR_INVALID_ARG.  n_out is a host pointer.
 *   - The call reads the row count back, so it returns only after its stream
 *     has finished the call's work.
 *   - The first call on a device looks the array's device address up (once
 *     per device); make that first call before any stream capture.
 *   - All calls share the one array, which keeps the last call's contents
 *     (the call clears its counters itself): calls that overlap on the GPU
 *     (other streams, other host threads) race and must be serialised by
 *     the caller.
 * Errors: as xtn_tcrdist_filter, plus TOO_LARGE.
 */
#define XTN_NOALLOC_MAX_SEQS (1 << 18)
#define XTN_NOALLOC_MAX_ROWS (1 << 22)
XTN_API int xtn_tcrdist_filter_noalloc(const uint8_t* seqs, const int64_t* offsets, int64_t n,
                               const xtn_triple* in, int64_t n_in, int max_score, xtn_triple* out,
                               int64_t* n_out, xtn_stream_t stream);

/*
 * Tuning knobs (process-wide, take effect for calls that start afterwards).
 *   XTN_TUNE_SORT_RECORDS : tile configuration of the radix sort of variant
 *                           records (0 .. xtn_tune_count(knob)-1): 0-19 rank
 *                           keys stably with ranks held in registers (the
 *                           first pass of a sort unstably); 20 and up count
 *                           and place keys with shared-memory atomics by
 *                           digit and run of already-sorted bits (default 22)
 *   XTN_TUNE_SORT_PAIRS   : tile configuration of the radix sort of verified
 *                           pair words, the same range (default 21)
 *   XTN_TUNE_RECORD_HISTOGRAM : where the record sort's digit counts are
 *                           taken: 0 = the expand kernel counts the digits
 *                           of every pass, 1 = expand counts the first pass
 *                           and each sort pass counts the next
 *   XTN_TUNE_GROUPING     : how records are grouped: 0 = global radix passes
 *                           on the top bits only, then one shared-memory pass
 *                           per block of buckets that finishes the sort and
 *                           writes the group flags (default); 1 = global
 *                           passes on every bit, then a flag pass; 2 = as 0
 *                           with 512-record shared-memory segments (slower;
 *                           more buckets take the large-bucket path)
 *   XTN_TUNE_FILTER_SEGMENT : grouping mode 0 groups each block of buckets
 *                           with a singleton filter first; its blocks hold
 *                           2^value times the buckets of the shared-memory
 *                           pass (0..3)
 * Every value gives the same result; they differ in threads per block, keys
 * per thread, ranking method and counting, hence in speed per GPU and size.
 * xtn_tune_set returns XTN_ERR_INVALID_ARG for an unknown knob or value.
 */
enum {
  XTN_TUNE_SORT_RECORDS = 0,
  XTN_TUNE_SORT_PAIRS = 1,
  XTN_TUNE_RECORD_HISTOGRAM = 2,
  XTN_TUNE_GROUPING = 3,
  XTN_TUNE_FILTER_SEGMENT = 4
};
XTN_API int xtn_tune_set(int knob, int value);
XTN_API int xtn_tune_get(int knob);
XTN_API int xtn_tune_count(int knob);

/*
 * Scratch cache.  Each search, index build or filter call carves its scratch
 * out of one device block taken from a per-device cache and gives it back
 * when it returns (stream-ordered: the next call that takes the block waits,
 * on its own stream, for the work of the call before); a call that needs more
 * takes the rest from the stream-ordered allocator, and the block grows to
 * that size the next time it is taken.  So calls in steady state allocate
 * nothing, and the cache holds about as much device memory as the largest
 * calls that ran at the same time needed.  xtn_scratch_trim() waits for and
 * frees the cached blocks of the current device that no call holds, and
 * returns the allocator's unused memory to the device.
 * Errors: CUDA.
 */
XTN_API int xtn_scratch_trim(void);

/*
 * Bounded device waits.  A kernel that waits for another block's status word
 * (the decoupled look-back of the scans, sorts and row compaction) polls it
 * at most 2^20 times, about a second, and then gives up: the call returns
 * XTN_ERR_DEVICE_TIMEOUT instead of waiting without bound, and every index a
 * kernel computes from the incomplete sums is range-checked before use.
 * xtn_set_wait_limit(polls) sets that limit for the calls that start
 * afterwards (process-wide; 0 restores the default).  A small limit makes a
 * wait give up while its predecessors are still working, which exercises the
 * give-up path; the search results of such a call are not defined.
 * Errors: INVALID_ARG for polls < 0 or > 2^20.
 */
XTN_API int xtn_set_wait_limit(int64_t polls);

/*
 * Kernel timing.  While enabled, every kernel the library launches is
 * bracketed by CUDA events on its stream and tagged with the algorithmic
 * bytes it must move.  xtn_profile_report() synchronises those events and
 * writes one line per kernel name, "name launches total_ms total_bytes\n",
 * into buf (NUL-terminated, truncated to buf_len); it returns the number of
 * lines, and clears the records.  Enabling costs two event records per launch.
 * Host-side spans are reported the same way, with zero bytes and wall-clock
 * milliseconds: host_call_search_self / _between / _paired / _query /
 * _query_hamming (the whole call),
 * host_scratch_alloc (each scratch allocation outside the cache) and
 * host_stream_wait (each wait for the stream to drain).
 * xtn_profile_only(name) restricts the timing to launches and spans with
 * that name (NULL or "" = all again), so that a timed loop carries only the
 * events of the kernel it is after; XTN_ERR_INVALID_ARG for a name of 64
 * characters or more.
 */
XTN_API int xtn_profile_enable(int on);
XTN_API int xtn_profile_only(const char* name);
XTN_API int xtn_profile_report(char* buf, int64_t buf_len);

#ifdef __cplusplus
}
#endif

#endif /* XTN_H_ */
