// C ABI (include/xtn.h): argument checks, host/device buffer handling,
// stream-ordered scratch, and the order of kernel launches for the
// self-search, index build, query search and TCRdist filter.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {

// ------------------------------------------------------------- profiler ---
namespace {
struct ProfRec {
  const char* name;
  double bytes;
  cudaEvent_t a, b;  // null for a host-side span
  double host_ms;    // wall-clock length of a host-side span
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::atomic<bool> g_prof_filtered{false};  // only launches named g_prof_only
char g_prof_only[64] = "";                 // guarded by g_prof_mu
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_ev_pool;
thread_local ProfRec t_pending{nullptr, 0.0, nullptr, nullptr, 0.0};

bool prof_wanted(const char* name) {
  if (!g_prof_filtered.load(std::memory_order_relaxed)) return true;
  std::lock_guard<std::mutex> g(g_prof_mu);
  return std::strcmp(name, g_prof_only) == 0;
}

cudaEvent_t ev_get() {
  {
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_ev_pool.empty()) {
      cudaEvent_t e = g_ev_pool.back();
      g_ev_pool.pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void prof_begin(cudaStream_t s, const char* name, double bytes) {
  if (!g_prof_on.load(std::memory_order_relaxed) || !prof_wanted(name)) return;
  t_pending.name = name;
  t_pending.bytes = bytes;
  t_pending.a = ev_get();
  t_pending.b = ev_get();
  cudaEventRecord(t_pending.a, s);
}

void prof_end(cudaStream_t s) {
  if (!t_pending.name) return;
  cudaEventRecord(t_pending.b, s);
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof.push_back(t_pending);
  t_pending.name = nullptr;
}

namespace {
// Host-side span for the profiler: the wall-clock time of a scope (a whole
// call, a scratch allocation, a wait for the stream), reported like a kernel.
class HostSpan {
 public:
  explicit HostSpan(const char* name)
      : name_(name), on_(g_prof_on.load(std::memory_order_relaxed) && prof_wanted(name)) {
    if (on_) t0_ = std::chrono::steady_clock::now();
  }
  ~HostSpan() {
    if (!on_) return;
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0_).count();
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.push_back(ProfRec{name_, 0.0, nullptr, nullptr, ms});
  }

 private:
  const char* name_;
  bool on_;
  std::chrono::steady_clock::time_point t0_;
};

cudaError_t host_sync(cudaStream_t s) {
  HostSpan span("host_stream_wait");
  return cudaStreamSynchronize(s);
}

}  // namespace

// --------------------------------------------------------------- device ---
namespace {

struct DevInfo {
  int sms = 0;
  bool pool_ready = false;
};
std::mutex g_dev_mu;
std::map<int, DevInfo> g_dev;

int current_device_info(int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return XTN_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_dev_mu);
  DevInfo& di = g_dev[dev];
  if (!di.pool_ready) {
    if (cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return XTN_ERR_CUDA;
    // keep freed scratch cached in the pool between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    di.pool_ready = true;
  }
  *sms = di.sms;
  return XTN_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Pinned host memory that this device's kernels can read and write in place
// (over the chip-to-chip link of a Grace-Blackwell node): its device address,
// else null (pageable memory is copied instead).
void* mapped_host_ptr(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost) return nullptr;
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, const_cast<void*>(p), 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return d;
}

// Cached scratch.  Each call carves its buffers out of one workspace, a
// device block taken from a per-device cache and given back when the call
// returns, so that a call in steady state allocates nothing: the stream-
// ordered allocator's own per-call cost grows with the process's history of
// streams and allocations.  Reuse is stream-ordered through an event: the
// call that takes a workspace makes its stream wait for the event the
// previous user recorded on its own stream when it gave the block back.  A
// call that needs more than the block holds takes the rest from the stream-
// ordered allocator; the block is grown to the call's total when it is next
// taken.
struct Workspace {
  char* base = nullptr;
  size_t cap = 0;              // bytes at base
  size_t want = 0;             // the largest total a call carved from it
  cudaEvent_t done = nullptr;  // recorded where its last user finished
};
struct WorkspaceCache {
  std::vector<Workspace*> idle;
};
std::mutex g_ws_mu;
std::map<int, WorkspaceCache> g_ws;

constexpr size_t SCRATCH_ALIGN = 256;

// Stream-ordered scratch owned by one call; given back at scope exit.
class Arena {
 public:
  explicit Arena(cudaStream_t s) : s_(s) {}
  ~Arena() { release(); }
  template <class T>
  T* get(size_t count) {
    if (count == 0) count = 1;
    // 64 spare bytes behind every buffer, 256-byte aligned starts
    const size_t bytes = (count * sizeof(T) + 64 + SCRATCH_ALIGN - 1) & ~(SCRATCH_ALIGN - 1);
    if (!taken_) take();
    total_ += bytes;
    if (ws_ && off_ + bytes <= ws_->cap) {
      void* p = ws_->base + off_;
      off_ += bytes;
      return static_cast<T*>(p);
    }
    void* p = nullptr;
    HostSpan span("host_scratch_alloc");
    if (cudaMallocAsync(&p, bytes, s_) != cudaSuccess) {
      cudaGetLastError();
      failed_ = true;
      return nullptr;
    }
    ptrs_.push_back(p);
    return static_cast<T*>(p);
  }
  bool failed() const { return failed_; }
  // Gives everything back now (stream-ordered), e.g. before a retry that
  // takes scratch again.
  void release() {
    for (void* p : ptrs_) cudaFreeAsync(p, s_);
    ptrs_.clear();
    if (ws_) {
      ws_->want = std::max(ws_->want, total_);
      cudaEventRecord(ws_->done, s_);
      std::lock_guard<std::mutex> g(g_ws_mu);
      g_ws[dev_].idle.push_back(ws_);
      ws_ = nullptr;
    }
    taken_ = false;
    off_ = total_ = 0;
  }

 private:
  void take() {
    taken_ = true;
    if (cudaGetDevice(&dev_) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    {
      std::lock_guard<std::mutex> g(g_ws_mu);
      auto& idle = g_ws[dev_].idle;
      if (!idle.empty()) {
        ws_ = idle.back();
        idle.pop_back();
      }
    }
    if (!ws_) {
      ws_ = new Workspace;
      if (cudaEventCreateWithFlags(&ws_->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete ws_;
        ws_ = nullptr;
        return;
      }
    }
    // the previous user's kernels are done with the block before ours start
    if (cudaStreamWaitEvent(s_, ws_->done, 0) != cudaSuccess) cudaGetLastError();
    if (ws_->want > ws_->cap) {
      if (ws_->base) cudaFreeAsync(ws_->base, s_);
      ws_->base = nullptr;
      ws_->cap = 0;
      HostSpan span("host_scratch_alloc");
      void* p = nullptr;
      if (cudaMallocAsync(&p, ws_->want, s_) == cudaSuccess) {
        ws_->base = static_cast<char*>(p);
        ws_->cap = ws_->want;
      } else {
        cudaGetLastError();  // the call takes its buffers one by one instead
      }
    }
  }

  cudaStream_t s_;
  int dev_ = 0;
  Workspace* ws_ = nullptr;
  bool taken_ = false;
  size_t off_ = 0, total_ = 0;
  std::vector<void*> ptrs_;
  bool failed_ = false;
};

// Frees the cached workspaces of the current device that no call holds.
int trim_scratch() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return XTN_ERR_CUDA;
  std::vector<Workspace*> idle;
  {
    std::lock_guard<std::mutex> g(g_ws_mu);
    idle.swap(g_ws[dev].idle);
  }
  bool ok = true;
  for (Workspace* w : idle) {
    ok &= cudaEventSynchronize(w->done) == cudaSuccess;  // its last user is done
    if (w->base) ok &= cudaFreeAsync(w->base, 0) == cudaSuccess;
    cudaEventDestroy(w->done);
    delete w;
  }
  ok &= cudaStreamSynchronize(0) == cudaSuccess;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  if (!ok) {
    cudaGetLastError();
    return XTN_ERR_CUDA;
  }
  return XTN_OK;
}

int map_device_err(uint32_t e) {
  if (e & DERR_TIMEOUT) return XTN_ERR_DEVICE_TIMEOUT;
  if (e & DERR_BAD_RESIDUE) return XTN_ERR_BAD_RESIDUE;
  if (e & DERR_TOO_LONG) return XTN_ERR_SEQ_TOO_LONG;
  if (e & DERR_CAPACITY) return XTN_ERR_CAPACITY;
  if (e & DERR_RANGE) return XTN_ERR_INVALID_ARG;
  return XTN_OK;
}

#define XTN_CK(call)                         \
  do {                                       \
    if ((call) != cudaSuccess) {             \
      cudaGetLastError();                    \
      return XTN_ERR_CUDA;                   \
    }                                        \
  } while (0)
#define XTN_ALLOC_OK(ar) \
  do {                   \
    if ((ar).failed()) return XTN_ERR_OOM; \
  } while (0)
#define XTN_RC(call)         \
  do {                       \
    const int rc_ = (call);  \
    if (rc_) return rc_;     \
  } while (0)

// Counts read back in the middle of a call (a few words) go through pinned
// host memory, one block per thread and device, and one wait: a pageable
// destination would turn every copy into a staged transfer that waits for
// the stream by itself.  wait() can queue work that needs none of the values
// (`overlap`) between the copies and the wait, so the GPU has it to run
// while the host takes the values and queues what follows.
class ReadBack {
 public:
  explicit ReadBack(cudaStream_t s) : s_(s) {}
  template <class T>
  int add(T* host, const T* dev) {
    static_assert(sizeof(T) <= 8, "one word per value");
    if (n_ == kSlots) return XTN_ERR_CUDA;
    Slot& m = slot();
    if (!m.buf) return XTN_ERR_CUDA;
    XTN_CK(cudaMemcpyAsync(m.buf + n_, dev, sizeof(T), cudaMemcpyDeviceToHost, s_));
    dst_[n_] = host;
    size_[n_] = sizeof(T);
    ++n_;
    return XTN_OK;
  }
  template <class F>
  int wait(F&& overlap) {
    Slot& m = slot();
    if (!m.buf) return XTN_ERR_CUDA;
    XTN_CK(cudaEventRecord(m.ev, s_));
    overlap();
    XTN_CK(cudaGetLastError());
    {
      HostSpan span("host_stream_wait");
      XTN_CK(cudaEventSynchronize(m.ev));
    }
    for (int k = 0; k < n_; ++k) std::memcpy(dst_[k], m.buf + k, size_[k]);
    n_ = 0;
    return XTN_OK;
  }
  int wait() {
    return wait([] {});
  }

 private:
  static constexpr int kSlots = 8;
  struct Slot {
    uint64_t* buf = nullptr;
    cudaEvent_t ev = nullptr;
  };
  static Slot& slot() {
    thread_local std::map<int, Slot> per_device;
    int dev = 0;
    cudaGetDevice(&dev);
    Slot& m = per_device[dev];
    if (!m.buf) {
      void* p = nullptr;
      if (cudaHostAlloc(&p, kSlots * sizeof(uint64_t), cudaHostAllocPortable) != cudaSuccess)
        return m;
      if (cudaEventCreateWithFlags(&m.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaFreeHost(p);
        return m;
      }
      m.buf = static_cast<uint64_t*>(p);
    }
    return m;
  }
  cudaStream_t s_;
  int n_ = 0;
  void* dst_[kSlots] = {};
  size_t size_[kSlots] = {};
};

// Poll limit of bounded device waits for calls that start from now on (0 =
// the kernels' default); see xtn_set_wait_limit.
std::atomic<uint32_t> g_wait_limit{0};

__global__ void k_set_word(uint32_t* p, uint32_t v) { *p = v; }

// Zero a call's error words (4 x u32) and, when a wait limit is set, put it
// in the second word, where the look-back waits read it.
int init_err(uint32_t* err, cudaStream_t s) {
  XTN_CK(cudaMemsetAsync(err, 0, 16, s));
  const uint32_t lim = g_wait_limit.load();
  if (lim) {
    k_set_word<<<1, 1, 0, s>>>(err + 1, lim);
    XTN_CK(cudaGetLastError());
  }
  return XTN_OK;
}

// Read n elements of device memory into host memory and wait for the stream.
template <class T>
int read_back(T* host, const T* dev, size_t n, cudaStream_t s) {
  XTN_CK(cudaMemcpyAsync(host, dev, n * sizeof(T), cudaMemcpyDeviceToHost, s));
  XTN_CK(host_sync(s));
  return XTN_OK;
}

uint32_t bits_for(uint64_t n) {  // bits to hold every value in [0, n)
  uint32_t b = 1;
  while (b < 64 && (1ull << b) < n) ++b;
  return b;
}

// Fingerprint bits used for grouping: the smallest multiple of 8 with
// 2^hs >= 32 * n_rec (expected colliding pairs <= n_rec / 64), at least 16
// and at most what the id field leaves free.
int choose_hash_bits(uint64_t n_rec, uint32_t id_bits) {
  int hs = 16;
  while (hs < 64 && std::ldexp(1.0, hs) < 32.0 * (double)n_rec) hs += 8;
  return std::min<int>(hs, 64 - (int)id_bits);
}

// Tunables (set by the autotuner through xtn_tune_set).
std::atomic<int> g_cfg_records{22};
std::atomic<int> g_cfg_pairs{21};
// Where the record sort's digit counts come from: 0 = the expand kernel
// counts every pass's digit, 1 = expand counts the first and each sort pass
// counts the next one.
std::atomic<int> g_record_hist{0};
// How records are grouped: 0 = global radix passes on the top bucket bits,
// then k_bucket_sort (shared-memory finish + group flags); 1 = global passes
// on every group-key bit, then k_group_flags; 2 = as 0 with 512-record
// shared-memory segments (more buckets take the large-bucket path).
std::atomic<int> g_grouping{0};
}  // namespace
// Buckets per block of the singleton filter: 2^fx of k_bucket's blocks.
std::atomic<int> g_filter_fx{1};
std::atomic<int>& cfg_records() { return g_cfg_records; }
std::atomic<int>& cfg_pairs() { return g_cfg_pairs; }
namespace {

// Sequences resident on the device for one call.
struct DevSeqs {
  const uint8_t* seqs = nullptr;
  const int64_t* off = nullptr;
  int64_t n = 0;
};

// Host-side check of host offsets: starts at 0, non-decreasing, lengths <= max.
int check_host_offsets(const int64_t* off, int64_t n) {
  if (off[0] != 0) return XTN_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t L = off[i + 1] - off[i];
    if (L < 0) return XTN_ERR_INVALID_ARG;
    if (L > XTN_MAX_LEN) return XTN_ERR_SEQ_TOO_LONG;
  }
  return XTN_OK;
}

int stage_seqs(const uint8_t* seqs, const int64_t* offsets, int64_t n, Arena& ar, cudaStream_t s,
               DevSeqs* out) {
  out->n = n;
  int64_t total = 0;
  const bool seqs_on_device = is_device_ptr(seqs);
  if (is_device_ptr(offsets)) {
    out->off = offsets;
    if (seqs_on_device) {
      // nothing to copy: k_encode checks the offsets (first 0, none past the
      // last, none decreasing) without a wait for the stream here
      out->seqs = seqs;
      return XTN_OK;
    }
    // host letters: their count is the last offset
    int64_t first = 0;
    XTN_CK(cudaMemcpyAsync(&first, offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    XTN_CK(cudaMemcpyAsync(&total, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    XTN_CK(host_sync(s));
    if (first != 0 || total < 0) return XTN_ERR_INVALID_ARG;
  } else {
    // O(1) on the host: the letters copied are offsets[n] bytes, at most 25
    // per sequence; a decreasing offset or a sequence longer than 25 inside
    // that total is found by k_encode on the device (error word).  Past the
    // total bound, the full host check names the error.
    total = offsets[n];
    if (offsets[0] != 0 || total < 0) return XTN_ERR_INVALID_ARG;
    if (total > (int64_t)XTN_MAX_LEN * n) {
      const int rc = check_host_offsets(offsets, n);
      return rc ? rc : XTN_ERR_INVALID_ARG;
    }
    // pinned host offsets and letters are read in place by k_encode, the
    // only kernel that reads them; pageable ones are copied first
    if (void* m = mapped_host_ptr(offsets)) {
      out->off = static_cast<const int64_t*>(m);
    } else {
      int64_t* d = ar.get<int64_t>(n + 1);
      XTN_ALLOC_OK(ar);
      XTN_CK(cudaMemcpyAsync(d, offsets, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      out->off = d;
    }
  }
  if (total > 0 && !seqs) return XTN_ERR_INVALID_ARG;
  if (seqs_on_device) {
    out->seqs = seqs;
  } else if (void* m = total > 0 ? mapped_host_ptr(seqs) : nullptr) {
    out->seqs = static_cast<const uint8_t*>(m);
  } else {
    uint8_t* d = ar.get<uint8_t>(total);
    XTN_ALLOC_OK(ar);
    if (total > 0) XTN_CK(cudaMemcpyAsync(d, seqs, total, cudaMemcpyHostToDevice, s));
    out->seqs = d;
  }
  return XTN_OK;
}

// Encoded sequences plus their variant-record offsets.
struct Encoded {
  Key128* keys = nullptr;
  uint8_t* lens = nullptr;
  uint32_t* eqprev = nullptr;
  uint64_t* rec_off = nullptr;
  uint64_t n_rec = 0;
  // paired receptors: the second chains (keys, lens, eqprev above are the
  // first chains); null for one chain
  Key128* keys_b = nullptr;
  uint8_t* lens_b = nullptr;
  uint32_t* eq_b = nullptr;
};

// allow_large: return the count even when it is 2^32 or more (the caller
// then searches in passes); otherwise that is TOO_LARGE.
int encode_and_count(const DevSeqs& in, int d, Arena& ar, uint32_t* err, cudaStream_t s,
                     Encoded* e, bool allow_large = false, uint32_t* peq = nullptr) {
  const int64_t n = in.n;
  e->keys = ar.get<Key128>(n);
  e->lens = ar.get<uint8_t>(n);
  e->eqprev = ar.get<uint32_t>(n);
  uint32_t* vcount = ar.get<uint32_t>(n);
  e->rec_off = ar.get<uint64_t>(n + 1);
  uint64_t* status = ar.get<uint64_t>(scan_status_bytes(n) / 8 + 1);
  XTN_ALLOC_OK(ar);
  launch_encode(in.seqs, in.off, n, d, e->keys, e->lens, e->eqprev, vcount, err, s);
  launch_scan_counts(vcount, n, e->rec_off, status, err, s);
  XTN_CK(cudaGetLastError());
  struct {
    uint64_t n_rec;
    uint32_t err;
  } h{0, 0};
  ReadBack rb(s);
  XTN_RC(rb.add(&h.n_rec, e->rec_off + n));
  XTN_RC(rb.add(&h.err, err));
  // the match vectors need only the encoded keys: they run during the wait
  XTN_RC(rb.wait([&] {
    if (peq) launch_peq(e->keys, e->lens, n, peq, s);
  }));
  if (h.err) return map_device_err(h.err);
  e->n_rec = h.n_rec;
  if (!allow_large && h.n_rec >= (1ull << 32)) return XTN_ERR_TOO_LARGE;
  return XTN_OK;
}

// Paired receptors: both chains encoded, the canonical variant counts of the
// joined strings (the token never deleted) and their record offsets.
int encode_and_count_paired(const DevSeqs& a, const DevSeqs& b, int d, Arena& ar, uint32_t* err,
                            cudaStream_t s, Encoded* e, uint32_t* peq = nullptr,
                            uint32_t* peq_b = nullptr) {
  const int64_t n = a.n;
  e->keys = ar.get<Key128>(n);
  e->lens = ar.get<uint8_t>(n);
  e->eqprev = ar.get<uint32_t>(n);
  e->keys_b = ar.get<Key128>(n);
  e->lens_b = ar.get<uint8_t>(n);
  e->eq_b = ar.get<uint32_t>(n);
  uint32_t* vcount = ar.get<uint32_t>(n);
  e->rec_off = ar.get<uint64_t>(n + 1);
  uint64_t* status = ar.get<uint64_t>(scan_status_bytes(n) / 8 + 1);
  XTN_ALLOC_OK(ar);
  launch_encode(a.seqs, a.off, n, d, e->keys, e->lens, e->eqprev, vcount, err, s);
  launch_encode(b.seqs, b.off, n, d, e->keys_b, e->lens_b, e->eq_b, vcount, err, s);
  launch_paired_counts(e->lens, e->eqprev, e->lens_b, e->eq_b, n, d, vcount, s);
  launch_scan_counts(vcount, n, e->rec_off, status, err, s);
  XTN_CK(cudaGetLastError());
  struct {
    uint64_t n_rec;
    uint32_t err;
  } h{0, 0};
  ReadBack rb(s);
  XTN_RC(rb.add(&h.n_rec, e->rec_off + n));
  XTN_RC(rb.add(&h.err, err));
  XTN_RC(rb.wait([&] {
    if (peq) launch_peq(e->keys, e->lens, n, peq, s);
    if (peq_b) launch_peq(e->keys_b, e->lens_b, n, peq_b, s);
  }));
  if (h.err) return map_device_err(h.err);
  e->n_rec = h.n_rec;
  if (h.n_rec >= (1ull << 32)) return XTN_ERR_TOO_LARGE;
  return XTN_OK;
}

// Expand + sort variant records: returns the sorted buffer and the other one.
struct Sorted {
  uint64_t* rec = nullptr;
  uint64_t* spare = nullptr;
  uint64_t* flags = nullptr;    // group flags (when asked for)
  uint64_t* gstatus = nullptr;  // group-bound scratch holding the flag tile counts
  uint32_t id_bits = 0;
  int hs = 0;
};

// Scratch of the grouping sort.  bucket_start: 2^G + 1 entries (bucket
// modes); flags + gstatus: group flags and group-bound scratch (when null, no
// flags are made: the caller only wants sorted records).
struct GroupScratch {
  uint64_t* bucket_start = nullptr;
  uint64_t* flags = nullptr;
  uint64_t* gstatus = nullptr;
  // bucket mode with flags: candidate words of the buckets that fit shared
  // memory go straight to cand[0, cand_cap); cand_count[0] counts them,
  // cand_count[1] the records of larger buckets (zeroed by the caller)
  uint64_t* cand = nullptr;
  uint64_t cand_cap = 0;
  uint64_t* cand_count = nullptr;
  // with cand (grouping mode 0): seg_area_bytes() for the singleton filter's
  // segment counter (first 16 bytes) and one flag byte per block of buckets
  uint8_t* seg_area = nullptr;
};

size_t seg_area_bytes(uint64_t rec_cap, int hs) {
  const GroupingShape g = choose_grouping(rec_cap, hs, true);
  return 16 + 4 * (((size_t)1 << g.G) >> g.kbits);
}

size_t bucket_start_words(uint64_t rec_cap, int hs, int mode) {
  if (mode == 1) return 1;
  return ((size_t)1 << choose_grouping(rec_cap, hs, true).G) + 1;
}

// Which of A / B receives the grouped records for this mode and size.
bool sorted_in_b(uint64_t rec_cap, int hs, int mode) {
  if (mode == 1) return ((hs + 7) / 8) % 2 == 1;
  return ((choose_grouping(rec_cap, hs, true).G / 8) % 2) == 0;
}

// Expand records into A and group them on their hs group-key bits
// (lo = 64 - hs).  With gs.flags (self-search) the records of each group end
// up contiguous and the group flags are written; without (reference index)
// the records end up sorted.  `hist_mode` is the record histogram placement
// (see g_record_hist), `mode` the grouping mode (see g_grouping).  *sorted
// receives A or B.
int expand_sort_launch(const Key128* keys, const uint8_t* lens, const uint32_t* eqprev,
                       const uint64_t* rec_off, int64_t n, int d, const uint32_t* seq_rep,
                       int id_bits, uint64_t* A, uint64_t* B, uint64_t rec_cap, int lo,
                       uint32_t* hist, uint64_t* digit_base, uint64_t* status, int cfg,
                       int hist_mode, int mode, const GroupScratch& gs, int sms, uint32_t* err,
                       cudaStream_t s, const uint64_t* n_rec_dev, uint64_t** sorted,
                       const BinSel* sel = nullptr, const Encoded* paired = nullptr) {
  // the expansion: one chain, or paired receptors (no bin selection); it
  // also clears the record sort's status area
  const bool zeroed = true;
  auto expand = [&](int hist_lo, int hist_hi) {
    if (paired)
      launch_expand_paired(paired->keys, paired->lens, paired->eqprev, paired->keys_b,
                           paired->lens_b, paired->eq_b, rec_off, n, d, id_bits, A, rec_cap, hist,
                           hist_lo, hist_hi, sms, err, s, status,
                           radix_status_bytes((int64_t)rec_cap, cfg));
    else
      launch_expand(keys, lens, eqprev, rec_off, n, d, seq_rep, id_bits, A, rec_cap, hist, hist_lo,
                    hist_hi, sms, err, s, sel, status, radix_status_bytes((int64_t)rec_cap, cfg));
  };
  if (mode == 1) {
    const bool in_passes = hist_mode == 1;
    expand(lo, in_passes ? std::min(64, lo + 8) : 64);
    XTN_CK(cudaGetLastError());
    XTN_CK(radix_sort_passes(A, B, (int64_t)rec_cap, lo, 64, hist, digit_base, status, cfg, err,
                             sorted, "k_onesweep_records", s, in_passes, n_rec_dev, nullptr,
                             onesweep_unstable_config(cfg), zeroed));
    if (gs.flags) {
      XTN_CK(cudaMemsetAsync(gs.gstatus, 0, group_status_bytes((int64_t)rec_cap), s));
      launch_group_flags(*sorted, (int64_t)rec_cap, n_rec_dev, lo, gs.flags, gs.gstatus, s);
    }
    return XTN_OK;
  }
  const bool hash = gs.flags != nullptr;
  const GroupingShape g = choose_grouping(rec_cap, 64 - lo, hash);
  const int glo = 64 - g.G;  // global passes sort bits [glo, 64)
  const bool in_passes = hist_mode == 1 && g.G > 8;
  if (g.G > 0)
    XTN_CK(cudaMemsetAsync(gs.bucket_start, 0xFF, ((size_t)1 << g.G) * 8, s));
  expand(glo, g.G == 0 ? glo : (in_passes ? glo + 8 : 64));
  XTN_CK(cudaGetLastError());
  uint64_t* X = A;
  XTN_CK(radix_sort_passes(A, B, (int64_t)rec_cap, glo, 64, hist, digit_base, status, cfg, err,
                           &X, "k_onesweep_records", s, in_passes, n_rec_dev, gs.bucket_start,
                           onesweep_unstable_config(cfg), zeroed));
  uint64_t* Y = X == A ? B : A;
  uint64_t* tile_counts = nullptr;
  if (gs.flags) {
    XTN_CK(cudaMemsetAsync(gs.flags, 0, group_flag_words((int64_t)rec_cap) * 8, s));
    XTN_CK(cudaMemsetAsync(gs.gstatus, 0, group_status_bytes((int64_t)rec_cap), s));
    tile_counts = group_tile_counts(gs.gstatus, (int64_t)rec_cap);
  }
  if (hash && gs.cand && gs.seg_area && mode == 0) {
    // the singleton filter groups and emits nearly every block of buckets;
    // k_bucket takes only the blocks it lists
    uint32_t* seg_count = reinterpret_cast<uint32_t*>(gs.seg_area);
    uint32_t* seg_list = reinterpret_cast<uint32_t*>(gs.seg_area + 16);
    XTN_CK(cudaMemsetAsync(seg_count, 0, 16, s));
    launch_bucket_filter(X, (int64_t)rec_cap, n_rec_dev, gs.bucket_start, g,
                         g_filter_fx.load(), lo, gs.cand, gs.cand_cap, gs.cand_count, id_bits,
                         seg_list, seg_count, err, s);
    launch_bucket(hash, X, Y, (int64_t)rec_cap, n_rec_dev, gs.bucket_start, g, lo, 0, gs.flags,
                  tile_counts, gs.cand, gs.cand_cap, gs.cand_count, id_bits, err, s, seg_list,
                  seg_count, sms);
  } else {
    launch_bucket(hash, X, Y, (int64_t)rec_cap, n_rec_dev, gs.bucket_start, g, lo,
                  mode == 2 ? 512 : 0, gs.flags, tile_counts, hash ? gs.cand : nullptr,
                  gs.cand_cap, gs.cand_count, id_bits, err, s);
  }
  XTN_CK(cudaGetLastError());
  *sorted = Y;
  return XTN_OK;
}

// want_flags: also make the group flags (out->flags, out->gstatus, the latter
// sized for the group-bound and group-pair scans of up to g_cap groups).
int expand_and_sort(const Encoded& e, int64_t n, int d, const uint32_t* seq_rep, int sms,
                    Arena& ar, uint32_t* err, cudaStream_t s, Sorted* out,
                    bool want_flags = false, uint64_t g_cap = 0, int mode = -1,
                    const GroupScratch* direct = nullptr) {
  const uint64_t n_rec = e.n_rec;
  out->id_bits = bits_for((uint64_t)n);
  out->hs = choose_hash_bits(n_rec, out->id_bits);
  const int lo = 64 - out->hs;
  const int cfg = g_cfg_records.load();
  uint64_t* A = ar.get<uint64_t>(n_rec + 8);
  uint64_t* B = ar.get<uint64_t>(n_rec + 8);
  uint32_t* hist = ar.get<uint32_t>(MAX_PASSES * RADIX);
  uint64_t* digit_base = ar.get<uint64_t>(MAX_PASSES * RADIX);
  uint64_t* status = ar.get<uint64_t>(radix_status_bytes(n_rec, cfg) / 8 + 1);
  if (mode < 0) mode = g_grouping.load();
  GroupScratch gs;
  if (direct) {
    gs.cand = direct->cand;
    gs.cand_cap = direct->cand_cap;
    gs.cand_count = direct->cand_count;
    if (mode == 0) gs.seg_area = ar.get<uint8_t>(seg_area_bytes(n_rec, out->hs));
  }
  gs.bucket_start = ar.get<uint64_t>(bucket_start_words(n_rec, out->hs, mode));
  if (want_flags) {
    gs.flags = ar.get<uint64_t>(group_flag_words((int64_t)n_rec));
    gs.gstatus = ar.get<uint64_t>(
        std::max(group_status_bytes((int64_t)n_rec), scan_status_bytes((int64_t)g_cap)) / 8 + 1);
  }
  XTN_ALLOC_OK(ar);
  XTN_CK(cudaMemsetAsync(hist, 0, MAX_PASSES * RADIX * 4, s));
  uint64_t* sorted = nullptr;
  XTN_CK(expand_sort_launch(e.keys, e.lens, e.eqprev, e.rec_off, n, d, seq_rep, out->id_bits, A,
                            B, n_rec, lo, hist, digit_base, status, cfg, g_record_hist.load(), mode,
                            gs, sms, err, s, nullptr, &sorted, nullptr,
                            e.keys_b ? &e : nullptr));
  out->flags = gs.flags;
  out->gstatus = gs.gstatus;
  out->rec = sorted;
  out->spare = sorted == A ? B : A;
  return XTN_OK;
}

// Back stage, asynchronous: verify candidate words P1 (count cand_cap, or
// the device count *n_cand_dev when given), append survivors to P2, sort
// them (P1 reused as the second buffer), drop duplicates and write rows.
// counters[0] receives the survivor count, counters[1] the row count.
struct BackStage {
  uint64_t* P1 = nullptr;
  uint64_t* P2 = nullptr;
  uint32_t* hist = nullptr;        // MAX_PASSES * RADIX
  uint64_t* digit_base = nullptr;  // MAX_PASSES * RADIX
  uint64_t* status = nullptr;      // back_status_bytes(cand_cap)
  uint64_t* counters = nullptr;    // 2
};

size_t back_status_bytes(uint64_t cand_cap, int cfg) {
  return std::max(radix_status_bytes((int64_t)cand_cap, cfg),
                  verify_status_bytes((int64_t)cand_cap));
}

// Sort the verified words surv[0, n) (n = *n_dev when given, else cap; tmp
// is the second buffer, both hold cap words) by their pair_bits low bits
// with the digit counts in hist, drop repeated words and write the rows;
// *n_rows receives the row count.
int launch_sort_unique(uint64_t* surv, uint64_t* tmp, uint64_t cap, const uint64_t* n_dev,
                       uint32_t pair_bits, uint32_t j_bits, uint32_t* hist, uint64_t* digit_base,
                       uint64_t* status, const uint32_t* peq_i, const uint8_t* lens_i,
                       uint64_t n_i, const Key128* keys_j, const uint8_t* lens_j, uint64_t n_j,
                       int metric, xtn_triple* rows, int64_t row_cap, uint32_t* err,
                       uint64_t* n_rows, cudaStream_t s, int cfg,
                       const SecondChain& sc = SecondChain()) {
  uint64_t* sorted = nullptr;
  XTN_CK(radix_sort_passes(surv, tmp, (int64_t)cap, 0, (int)pair_bits, hist, digit_base, status,
                           cfg, err, &sorted, "k_onesweep_pairs", s, false, n_dev, nullptr,
                           onesweep_unstable_config(cfg)));
  launch_unique_finalize(sorted, (int64_t)cap, n_dev, j_bits, peq_i, lens_i, n_i, keys_j, lens_j,
                         n_j, metric, rows, row_cap, status, err, n_rows, s, sc,
                         pair_bits + 8 <= 64 ? (int)pair_bits : 0);
  XTN_CK(cudaGetLastError());
  return XTN_OK;
}

int launch_back(const BackStage& b, uint64_t cand_cap, const uint64_t* n_cand_dev,
                uint32_t pair_bits, uint32_t j_bits, const uint32_t* peq_i, const uint8_t* lens_i,
                uint64_t n_i, const Key128* keys_j, const uint8_t* lens_j, uint64_t n_j,
                const uint32_t* seq_rep, int self_mode, int d, xtn_triple* rows, int64_t row_cap,
                int sms, uint32_t* err, cudaStream_t s, int cfg, int metric = 0,
                const SecondChain& sc = SecondChain()) {
  XTN_CK(cudaMemsetAsync(b.hist, 0, MAX_PASSES * RADIX * 4, s));
  XTN_CK(cudaMemsetAsync(b.counters, 0, 16, s));
  launch_verify_candidates(b.P1, cand_cap, n_cand_dev, j_bits, peq_i, lens_i, n_i, keys_j, lens_j,
                           n_j, seq_rep, self_mode, d, metric, b.P2, cand_cap, b.counters, b.hist,
                           (int)pair_bits, sms, err, s, sc);
  return launch_sort_unique(b.P2, b.P1, cand_cap, b.counters, pair_bits, j_bits, b.hist,
                            b.digit_base, b.status, peq_i, lens_i, n_i, keys_j, lens_j, n_j, metric,
                            rows, row_cap, err, b.counters + 1, s, cfg, sc);
}

// Result rows go to `out` directly when it is device memory; otherwise into
// scratch and then to the host.
struct OutRows {
  xtn_triple* dev = nullptr;
  int64_t dev_cap = 0;
  bool host = false;
};

int prepare_out(xtn_triple* out, int64_t cap, uint64_t max_rows, Arena& ar, OutRows* o) {
  if (cap > 0 && !out) return XTN_ERR_INVALID_ARG;
  if (cap <= 0) {
    o->dev = nullptr;
    o->dev_cap = 0;
    return XTN_OK;
  }
  if (is_device_ptr(out)) {
    o->dev = out;
    o->dev_cap = cap;
  } else if (void* m = mapped_host_ptr(out)) {  // pinned host rows: written in place
    o->dev = static_cast<xtn_triple*>(m);
    o->dev_cap = cap;
  } else {
    o->host = true;
    o->dev_cap = (int64_t)std::min<uint64_t>((uint64_t)cap, max_rows);
    o->dev = ar.get<xtn_triple>(o->dev_cap);
    XTN_ALLOC_OK(ar);
  }
  return XTN_OK;
}

int finish_out(const OutRows& o, xtn_triple* out, int64_t cap, uint64_t n_rows, cudaStream_t s,
               int64_t* n_out) {
  *n_out = (int64_t)n_rows;
  const int64_t w = std::min<int64_t>(cap, (int64_t)n_rows);
  if (o.host && w > 0) {
    XTN_CK(cudaMemcpyAsync(out, o.dev, w * sizeof(xtn_triple), cudaMemcpyDeviceToHost, s));
    XTN_CK(host_sync(s));
  }
  return (int64_t)n_rows > cap ? XTN_ERR_BUFFER_TOO_SMALL : XTN_OK;
}

// Repertoire of every sequence (batched mode), checked on the host.
int stage_reps(const int64_t* rep_offsets, int64_t n_rep, int64_t n, Arena* ar, cudaStream_t s,
               uint32_t* seq_rep) {
  std::vector<int64_t> h(n_rep + 1);
  if (is_device_ptr(rep_offsets)) {
    int rc = read_back(h.data(), rep_offsets, n_rep + 1, s);
    if (rc) return rc;
  } else {
    std::memcpy(h.data(), rep_offsets, (n_rep + 1) * sizeof(int64_t));
  }
  if (h[0] != 0 || h[n_rep] != n) return XTN_ERR_INVALID_ARG;
  for (int64_t r = 0; r < n_rep; ++r)
    if (h[r + 1] < h[r]) return XTN_ERR_INVALID_ARG;
  int64_t* d_rep = ar->get<int64_t>(n_rep + 1);
  XTN_ALLOC_OK(*ar);
  XTN_CK(cudaMemcpyAsync(d_rep, h.data(), (n_rep + 1) * 8, cudaMemcpyHostToDevice, s));
  launch_seq_rep(d_rep, n_rep, seq_rep, n, s);
  return XTN_OK;
}

// pair_count[0] = pair_off[n_groups] once n_groups is known on the device.
__global__ void k_pair_total(const uint64_t* __restrict__ pair_off,
                             const uint64_t* __restrict__ n_groups, uint64_t* __restrict__ out) {
  *out = pair_off[*n_groups];
}

// A device buffer of 64-bit words that a multi-pass call grows as it goes
// (stream-ordered, outside the scratch cache: its size is not known ahead).
struct GrowBuf {
  explicit GrowBuf(cudaStream_t st) : s(st) {}
  ~GrowBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  // At least `need` words; the first `keep` words survive a move.
  bool reserve(uint64_t need, uint64_t keep) {
    if (need <= cap) return true;
    const uint64_t c = std::max(need, cap + cap / 2);
    void* q = nullptr;
    HostSpan span("host_scratch_alloc");
    if (cudaMallocAsync(&q, (c + 8) * 8, s) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (keep && cudaMemcpyAsync(q, p, keep * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeAsync(q, s);
      return false;
    }
    if (p) cudaFreeAsync(p, s);
    p = static_cast<uint64_t*>(q);
    cap = c;
    return true;
  }
  cudaStream_t s;
  uint64_t* p = nullptr;
  uint64_t cap = 0;
};

// Records one pass may hold when the caller sets no budget: what a pass needs
// (two record buffers, candidate words, flags: about 32 bytes per record) in
// half the free device memory, below 2^32.
uint64_t default_pass_records() {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 1ull << 28;
  }
  return std::max<uint64_t>(1ull << 20, (uint64_t)free_b / 2 / 32);
}

// The self-search in passes over fingerprint bins, for inputs whose variant
// records do not fit at once (Sec. 2.3, "Overcoming memory bottlenecks";
// Appendix A, XTNeighbor-streaming).  A counting expansion gives the records
// of every bin (the MAX_BIN_BITS lowest bits of the fingerprint field);
// Next-Fit packs consecutive bins into passes of at most max_pass records;
// each pass expands only its bins' records, groups them and emits and
// verifies their candidate pairs.  Equal variants share their fingerprint
// and so their bin, so every candidate of the one-pass search is a candidate
// of some pass.  A pair that shares variants in several bins is found in
// several passes: the verified words of all passes are kept and sorted once
// at the end, which drops those repeats.  (The paper bins candidate pairs by
// min(i, j) instead, so that it can remove repeats before verifying; here
// verification comes first, and only its survivors are kept.)  A pass whose
// candidates exceed 2^32 words or device memory is split in two at its
// middle bin.  Arguments as search_self_impl; max_pass <= 0 takes
// default_pass_records(); *n_passes receives the passes run.
int search_stream_impl(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                       const int64_t* rep_offsets, int64_t n_rep, int metric, bool between,
                       int64_t max_pass, xtn_triple* out, int64_t cap, int64_t* n_out,
                       int64_t* n_passes, cudaStream_t s) {
  if (!n_out) return XTN_ERR_INVALID_ARG;
  *n_out = 0;
  if (n_passes) *n_passes = 0;
  if (n < 0 || d < 0 || d > XTN_MAX_D || cap < 0 || !offsets) return XTN_ERR_INVALID_ARG;
  if (metric != XTN_METRIC_LEVENSHTEIN && metric != XTN_METRIC_HAMMING) return XTN_ERR_INVALID_ARG;
  if (n >= (1ll << 32)) return XTN_ERR_TOO_LARGE;
  if (rep_offsets && n_rep < 1) return XTN_ERR_INVALID_ARG;
  if (between && !rep_offsets) return XTN_ERR_INVALID_ARG;
  if (n == 0) return XTN_OK;
  int sms = 0;
  int rc = current_device_info(&sms);
  if (rc) return rc;
  Arena ar(s);
  constexpr uint32_t NB = 1u << MAX_BIN_BITS;
  uint32_t* err = ar.get<uint32_t>(4);
  // [0] groups [1] pairs [2] direct candidates [3] large-bucket records
  // [4] records appended [5] survivors [6] rows
  uint64_t* ctr = ar.get<uint64_t>(8);
  uint32_t* bins = ar.get<uint32_t>(NB);
  XTN_ALLOC_OK(ar);
  XTN_CK(init_err(err, s));
  XTN_CK(cudaMemsetAsync(ctr, 0, 64, s));
  XTN_CK(cudaMemsetAsync(bins, 0, NB * 4, s));
  DevSeqs in;
  rc = stage_seqs(seqs, offsets, n, ar, s, &in);
  if (rc) return rc;
  uint32_t* seq_rep = nullptr;
  if (rep_offsets) {
    seq_rep = ar.get<uint32_t>(n);
    XTN_ALLOC_OK(ar);
    rc = stage_reps(rep_offsets, n_rep, n, &ar, s, seq_rep);
    if (rc) return rc;
  }
  Encoded e;
  rc = encode_and_count(in, d, ar, err, s, &e, true);
  if (rc) return rc;
  const uint32_t id_bits = bits_for((uint64_t)n);
  const uint32_t* salt_rep = between ? nullptr : seq_rep;

  // records per bin
  BinSel sel;
  sel.shift = id_bits;
  sel.mask = NB - 1u;
  sel.bin_count = bins;
  launch_expand(e.keys, e.lens, e.eqprev, e.rec_off, n, d, salt_rep, id_bits, nullptr, e.n_rec,
                nullptr, 0, 8, sms, err, s, &sel);
  XTN_CK(cudaGetLastError());
  std::vector<uint32_t> hb(NB);
  uint32_t herr = 0;
  XTN_CK(cudaMemcpyAsync(hb.data(), bins, NB * 4, cudaMemcpyDeviceToHost, s));
  XTN_CK(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
  XTN_CK(host_sync(s));
  if (herr) return map_device_err(herr);
  std::vector<uint64_t> pre(NB + 1, 0);  // records of bins [0, b)
  for (uint32_t b = 0; b < NB; ++b) pre[b + 1] = pre[b] + hb[b];
  if (pre[NB] != e.n_rec) return XTN_ERR_CUDA;  // the two expansions disagree

  // Next-Fit over consecutive bins
  const uint64_t limit = (1ull << 32) - (1ull << 20);
  const uint64_t R = std::min<uint64_t>(max_pass > 0 ? (uint64_t)max_pass : default_pass_records(),
                                        limit);
  std::vector<std::pair<uint32_t, uint32_t>> work;  // bin ranges, run from the back
  for (uint32_t b0 = 0, b = 0; b <= NB; ++b) {
    if (b == NB || (pre[b] > pre[b0] && pre[b + 1] - pre[b0] > R)) {
      if (pre[b] > pre[b0]) work.emplace_back(b0, b);
      b0 = b;
    }
  }
  std::reverse(work.begin(), work.end());
  uint64_t P = 0;  // records of the largest pass
  for (auto& w : work) P = std::max(P, pre[w.second] - pre[w.first]);
  if (P >= limit) return XTN_ERR_TOO_LARGE;  // one bin beyond a pass

  // buffers for the largest pass
  const int hs = choose_hash_bits(P, id_bits);
  const int lo = 64 - hs;
  const int cfg = g_cfg_records.load();
  const int cfg_pairs = g_cfg_pairs.load();
  const int mode0 = g_grouping.load();
  const uint64_t g_cap = P / 2 + 1;
  uint64_t* A = ar.get<uint64_t>(P + 8);
  uint64_t* B = ar.get<uint64_t>(P + 8);
  uint32_t* hist = ar.get<uint32_t>(MAX_PASSES * RADIX);
  uint32_t* phist = ar.get<uint32_t>(MAX_PASSES * RADIX);  // survivors, over all passes
  uint64_t* digit_base = ar.get<uint64_t>(MAX_PASSES * RADIX);
  uint64_t* status = ar.get<uint64_t>(radix_status_bytes(P, cfg) / 8 + 1);
  GroupScratch gs0;
  gs0.bucket_start = ar.get<uint64_t>(bucket_start_words(P, hs, 0));
  gs0.seg_area = ar.get<uint8_t>(seg_area_bytes(P, hs));
  gs0.flags = ar.get<uint64_t>(group_flag_words((int64_t)P));
  gs0.gstatus = ar.get<uint64_t>(
      std::max(group_status_bytes((int64_t)P), scan_status_bytes((int64_t)g_cap)) / 8 + 1);
  uint32_t* peq = ar.get<uint32_t>((size_t)n * PEQ_STRIDE);
  XTN_ALLOC_OK(ar);
  GrowBuf cand(s), surv(s);
  if (!cand.reserve(std::max<uint64_t>(P / 2, 1u << 20), 0) ||
      !surv.reserve(std::max<uint64_t>((uint64_t)n, 1u << 20), 0))
    return XTN_ERR_OOM;
  XTN_CK(cudaMemsetAsync(phist, 0, MAX_PASSES * RADIX * 4, s));
  launch_peq(e.keys, e.lens, n, peq, s);
  const uint32_t pair_bits = 2 * id_bits;

  int64_t passes_run = 0;
  while (!work.empty()) {
    const auto w = work.back();
    work.pop_back();
    const uint64_t np = pre[w.second] - pre[w.first];
    int mode = mode0;
    bool split = false;
    for (;;) {  // at most twice: the tuned grouping, then all-global
      XTN_CK(cudaMemsetAsync(ctr, 0, 40, s));
      XTN_CK(cudaMemsetAsync(hist, 0, MAX_PASSES * RADIX * 4, s));
      sel.lo = w.first;
      sel.hi = w.second;
      sel.bin_count = nullptr;
      sel.append = reinterpret_cast<unsigned long long*>(ctr + 4);
      GroupScratch gs = gs0;
      if (mode != 1) {
        gs.cand = cand.p;
        gs.cand_cap = cand.cap;
        gs.cand_count = ctr + 2;
      }
      uint64_t* sorted = nullptr;
      XTN_CK(expand_sort_launch(e.keys, e.lens, e.eqprev, e.rec_off, n, d, salt_rep, id_bits, A,
                                B, np, lo, hist, digit_base, status, cfg, g_record_hist.load(),
                                mode, gs, sms, err, s, nullptr, &sorted, &sel));
      struct {
        uint64_t direct, large, appended, survivors;
        uint64_t groups, pairs;
        uint32_t err;
      } h{0, 0, 0, 0, 0, 0, 0};
      XTN_CK(cudaMemcpyAsync(&h.direct, ctr + 2, 32, cudaMemcpyDeviceToHost, s));
      XTN_CK(cudaMemcpyAsync(&h.err, err, 4, cudaMemcpyDeviceToHost, s));
      XTN_CK(host_sync(s));
      if (mode != 1 && h.err == DERR_CAPACITY) {  // direct candidates overflowed, nothing else
        XTN_CK(cudaMemsetAsync(err, 0, 4, s));
        mode = 1;
        continue;
      }
      if (h.err) return map_device_err(h.err);
      if (h.appended != np) return XTN_ERR_CUDA;  // the two expansions disagree
      uint32_t* S = reinterpret_cast<uint32_t*>(sorted == A ? B : A);
      uint32_t* E = S + g_cap;
      uint64_t* pair_off = reinterpret_cast<uint64_t*>(E + g_cap);
      if (mode == 1 || h.large > 0) {
        launch_group_finish(gs.flags, (int64_t)np, nullptr, S, E, g_cap, gs.gstatus, err, ctr, s);
        launch_scan_group_pairs(S, E, (int64_t)g_cap, ctr, pair_off, gs.gstatus, err, s);
        k_pair_total<<<1, 1, 0, s>>>(pair_off, ctr, ctr + 1);
        XTN_CK(cudaGetLastError());
        XTN_CK(cudaMemcpyAsync(&h.groups, ctr, 16, cudaMemcpyDeviceToHost, s));
        XTN_CK(cudaMemcpyAsync(&h.err, err, 4, cudaMemcpyDeviceToHost, s));
        XTN_CK(host_sync(s));
        if (h.err) return map_device_err(h.err);
      }
      const uint64_t n_pairs = h.direct + h.pairs;
      if (mode != 1 && n_pairs > cand.cap) {
        mode = 1;
        continue;
      }
      if (n_pairs >= limit || !cand.reserve(n_pairs, 0) ||
          !surv.reserve(h.survivors + n_pairs, h.survivors)) {
        if (w.second - w.first < 2) return n_pairs >= limit ? XTN_ERR_TOO_LARGE : XTN_ERR_OOM;
        const uint32_t mid = w.first + (w.second - w.first) / 2;
        work.emplace_back(mid, w.second);
        work.emplace_back(w.first, mid);
        split = true;
        break;
      }
      if (h.pairs)
        launch_emit_pairs(sorted, np, S, pair_off, (int64_t)h.groups, nullptr, h.pairs, id_bits,
                          cand.p + h.direct, nullptr, nullptr, sms, err, s);
      if (n_pairs)
        launch_verify_candidates(cand.p, n_pairs, nullptr, id_bits, peq, e.lens, (uint64_t)n,
                                 e.keys, e.lens, (uint64_t)n, seq_rep, between ? 2 : 1, d, metric,
                                 surv.p, surv.cap, ctr + 5, phist, (int)pair_bits, sms, err, s);
      XTN_CK(cudaGetLastError());
      break;
    }
    if (!split) ++passes_run;
  }
  if (n_passes) *n_passes = passes_run;

  // the survivors of every pass: sort, drop repeats, write rows
  struct {
    uint64_t survivors;
    uint32_t err;
  } f{0, 0};
  XTN_CK(cudaMemcpyAsync(&f.survivors, ctr + 5, 8, cudaMemcpyDeviceToHost, s));
  XTN_CK(cudaMemcpyAsync(&f.err, err, 4, cudaMemcpyDeviceToHost, s));
  XTN_CK(host_sync(s));
  if (f.err) return map_device_err(f.err);
  if (f.survivors == 0) return XTN_OK;
  GrowBuf tmp(s);
  if (!tmp.reserve(f.survivors, 0)) return XTN_ERR_OOM;
  uint64_t* pstatus = ar.get<uint64_t>(back_status_bytes(f.survivors, cfg_pairs) / 8 + 1);
  XTN_ALLOC_OK(ar);
  OutRows o;
  rc = prepare_out(out, cap, f.survivors, ar, &o);
  if (rc) return rc;
  rc = launch_sort_unique(surv.p, tmp.p, f.survivors, nullptr, pair_bits, id_bits, phist,
                          digit_base, pstatus, peq, e.lens, (uint64_t)n, e.keys, e.lens,
                          (uint64_t)n, metric, o.dev, o.dev_cap, err, ctr + 6, s, cfg_pairs);
  if (rc) return rc;
  uint64_t rows = 0;
  XTN_CK(cudaMemcpyAsync(&rows, ctr + 6, 8, cudaMemcpyDeviceToHost, s));
  XTN_CK(cudaMemcpyAsync(&f.err, err, 4, cudaMemcpyDeviceToHost, s));
  XTN_CK(host_sync(s));
  if (f.err) return map_device_err(f.err);
  return finish_out(o, out, cap, rows, s, n_out);
}

// mode: grouping mode (see g_grouping), -1 = the tuned one.  metric: 0 =
// Levenshtein, 1 = Hamming (the Hamming variant: the same candidates, the
// last step filters by Hamming distance).  between: report the pairs between
// different repertoires instead of those within one; the variants then carry
// no repertoire salt, so that equal variants of different repertoires meet.
// b_seqs / b_offsets (paired receptors, the paired-chain search): the second
// chains; seqs / offsets then hold the first chains, d <= 2, one repertoire,
// and the last step takes metric 2 (the sum of the two chains' distances).
int search_self_impl(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                     const int64_t* rep_offsets, int64_t n_rep, xtn_triple* out, int64_t cap,
                     int64_t* n_out, cudaStream_t s, int mode = -1, int metric = 0,
                     bool between = false, const uint8_t* b_seqs = nullptr,
                     const int64_t* b_offsets = nullptr) {
  if (!n_out) return XTN_ERR_INVALID_ARG;
  *n_out = 0;
  if (n < 0 || d < 0 || d > XTN_MAX_D || cap < 0 || !offsets) return XTN_ERR_INVALID_ARG;
  const bool paired = b_offsets != nullptr;
  if (paired && (d > 2 || rep_offsets)) return XTN_ERR_INVALID_ARG;
  if (paired) metric = 2;
  if (n >= (1ll << 32)) return XTN_ERR_TOO_LARGE;
  if (rep_offsets && n_rep < 1) return XTN_ERR_INVALID_ARG;
  if (between && !rep_offsets) return XTN_ERR_INVALID_ARG;
  if (n == 0) return XTN_OK;
  int sms = 0;
  int rc = current_device_info(&sms);
  if (rc) return rc;
  Arena ar(s);
  uint32_t* err = ar.get<uint32_t>(4);
  uint64_t* counters = ar.get<uint64_t>(4);
  XTN_ALLOC_OK(ar);
  XTN_CK(init_err(err, s));
  XTN_CK(cudaMemsetAsync(counters, 0, 32, s));
  DevSeqs in, in_b;
  rc = stage_seqs(seqs, offsets, n, ar, s, &in);
  if (rc) return rc;
  if (paired) {
    rc = stage_seqs(b_seqs, b_offsets, n, ar, s, &in_b);
    if (rc) return rc;
  }
  uint32_t* seq_rep = nullptr;
  if (rep_offsets) {
    seq_rep = ar.get<uint32_t>(n);
    XTN_ALLOC_OK(ar);
    rc = stage_reps(rep_offsets, n_rep, n, &ar, s, seq_rep);
    if (rc) return rc;
  }

  // front: encode (read back the record count; the match vectors are
  // computed meanwhile), expand, sort, group, offsets
  uint32_t* peq = ar.get<uint32_t>((size_t)n * PEQ_STRIDE);
  uint32_t* peq_b = paired ? ar.get<uint32_t>((size_t)n * PEQ_STRIDE) : nullptr;
  XTN_ALLOC_OK(ar);
  Encoded e;
  rc = paired ? encode_and_count_paired(in, in_b, d, ar, err, s, &e, peq, peq_b)
              : encode_and_count(in, d, ar, err, s, &e, false, peq);
  if (rc == XTN_ERR_TOO_LARGE && !paired) {  // 2^32 records or more: search in passes
    ar.release();
    return search_stream_impl(seqs, offsets, n, d, rep_offsets, n_rep, metric, between, 0, out,
                              cap, n_out, nullptr, s);
  }
  if (rc) return rc;
  Sorted so;
  const uint64_t g_cap = e.n_rec / 2 + 1;
  if (mode < 0) mode = g_grouping.load();
  // Bucket modes emit the candidates of every bucket that fits shared memory
  // during grouping, into a buffer sized by a guess; past it, the search runs
  // again with all-global grouping, which sizes its buffers exactly.
  GroupScratch direct;
  if (mode != 1) {
    direct.cand_cap = std::max<uint64_t>(e.n_rec / 2, 1u << 20);
    direct.cand = ar.get<uint64_t>(direct.cand_cap + 8);
    direct.cand_count = counters + 2;
    XTN_ALLOC_OK(ar);
  }
  rc = expand_and_sort(e, n, d, between ? nullptr : seq_rep, sms, ar, err, s, &so, true, g_cap,
                       mode, mode != 1 ? &direct : nullptr);
  if (rc) return rc;
  uint32_t* S = reinterpret_cast<uint32_t*>(so.spare);  // groups live in the spare buffer
  uint32_t* E = S + g_cap;
  uint64_t* pair_off = reinterpret_cast<uint64_t*>(E + g_cap);  // 8-byte aligned
  struct {
    uint64_t groups, pairs, direct, large;
    uint32_t err;
  } h{0, 0, 0, 0, 0};
  bool flagged = mode == 1;  // groups to emit through flags and S/E
  if (mode != 1) {
    ReadBack rb(s);
    XTN_RC(rb.add(&h.direct, counters + 2));
    XTN_RC(rb.add(&h.large, counters + 3));
    XTN_RC(rb.add(&h.err, err));
    XTN_RC(rb.wait());
    if (h.err == DERR_CAPACITY) {  // candidate overflow alone: regroup sized exactly
      ar.release();
      return search_self_impl(seqs, offsets, n, d, rep_offsets, n_rep, out, cap, n_out, s, 1,
                              metric, between, b_seqs, b_offsets);
    }
    if (h.err) return map_device_err(h.err);
    flagged = h.large > 0;
  }
  if (flagged) {
    launch_group_finish(so.flags, (int64_t)e.n_rec, nullptr, S, E, g_cap, so.gstatus, err,
                        counters, s);
    launch_scan_group_pairs(S, E, (int64_t)g_cap, counters, pair_off, so.gstatus, err, s);
    k_pair_total<<<1, 1, 0, s>>>(pair_off, counters, counters + 1);
    XTN_CK(cudaGetLastError());
    ReadBack rb(s);
    XTN_RC(rb.add(&h.groups, counters));
    XTN_RC(rb.add(&h.pairs, counters + 1));
    XTN_RC(rb.add(&h.err, err));
    XTN_RC(rb.wait());
    if (h.err) return map_device_err(h.err);
  }
  const uint64_t n_pairs = h.direct + h.pairs;
  if (n_pairs == 0) return XTN_OK;
  if (n_pairs >= (1ull << 32)) {  // candidate words past 2^32: search in passes
    if (paired) return XTN_ERR_TOO_LARGE;
    ar.release();
    return search_stream_impl(seqs, offsets, n, d, rep_offsets, n_rep, metric, between, 0, out,
                              cap, n_out, nullptr, s);
  }
  if (mode != 1 && n_pairs > direct.cand_cap) {
    ar.release();
    return search_self_impl(seqs, offsets, n, d, rep_offsets, n_rep, out, cap, n_out, s, 1,
                            metric, between, b_seqs, b_offsets);
  }

  // back: the remaining candidates, verify, sort survivors, dedup
  BackStage b;
  b.P1 = mode != 1 ? direct.cand : ar.get<uint64_t>(n_pairs + 8);
  b.P2 = ar.get<uint64_t>(n_pairs + 8);
  b.hist = ar.get<uint32_t>(MAX_PASSES * RADIX);
  b.digit_base = ar.get<uint64_t>(MAX_PASSES * RADIX);
  const int cfg_pairs = g_cfg_pairs.load();
  b.status = ar.get<uint64_t>(back_status_bytes(n_pairs, cfg_pairs) / 8 + 1);
  b.counters = ar.get<uint64_t>(2);
  XTN_ALLOC_OK(ar);
  if (h.pairs)
    launch_emit_pairs(so.rec, e.n_rec, S, pair_off, (int64_t)h.groups, nullptr, h.pairs,
                      so.id_bits, b.P1 + h.direct, nullptr, nullptr, sms, err, s);
  SecondChain sc;
  if (paired) {
    sc.peq_i = peq_b;
    sc.lens_i = e.lens_b;
    sc.keys_j = e.keys_b;
    sc.lens_j = e.lens_b;
  }
  OutRows o;
  rc = prepare_out(out, cap, n_pairs, ar, &o);
  if (rc) return rc;
  rc = launch_back(b, n_pairs, nullptr, 2 * so.id_bits, so.id_bits, peq, e.lens, n, e.keys, e.lens,
                   n, seq_rep, between ? 2 : 1, d, o.dev, o.dev_cap, sms, err, s, cfg_pairs,
                   metric, sc);
  if (rc) return rc;
  ReadBack rb(s);
  XTN_RC(rb.add(&h.pairs, b.counters + 1));
  XTN_RC(rb.add(&h.err, err));
  XTN_RC(rb.wait());
  if (h.err) return map_device_err(h.err);
  return finish_out(o, out, cap, h.pairs, s, n_out);
}

}  // namespace
}  // namespace xtn

// ======================================================================
// Query index
// ======================================================================
struct xtn_index {
  int device = 0;
  int d = 0;
  int64_t n = 0;
  uint64_t n_rec = 0;
  uint32_t id_bits = 0;
  int hs = 0;
  int dir_bits = 0;
  xtn::Key128* keys = nullptr;
  uint8_t* lens = nullptr;
  uint64_t* rec = nullptr;
  uint32_t* dir = nullptr;
  int64_t bytes = 0;
  uint64_t n_groups = 0;  // distinct variant fingerprints in the index
  // candidates and query variants of the searches so far (scratch estimates)
  mutable std::atomic<uint64_t> seen_cand{0}, seen_qv{0};
};

namespace xtn {
namespace {

int index_build_impl(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d, cudaStream_t s,
                     xtn_index** out) {
  if (!out) return XTN_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || d < 0 || d > XTN_MAX_D || !offsets) return XTN_ERR_INVALID_ARG;
  if (n >= (1ll << 32)) return XTN_ERR_TOO_LARGE;
  int sms = 0;
  int rc = current_device_info(&sms);
  if (rc) return rc;
  Arena ar(s);
  uint32_t* err = ar.get<uint32_t>(4);
  XTN_ALLOC_OK(ar);
  XTN_CK(init_err(err, s));
  DevSeqs in;
  rc = stage_seqs(seqs, offsets, n, ar, s, &in);
  if (rc) return rc;
  Encoded e;
  rc = encode_and_count(in, d, ar, err, s, &e);
  if (rc) return rc;
  Sorted so;
  rc = expand_and_sort(e, n, d, nullptr, sms, ar, err, s, &so);
  if (rc) return rc;

  xtn_index* idx = new xtn_index;
  cudaGetDevice(&idx->device);
  idx->d = d;
  idx->n = n;
  idx->n_rec = e.n_rec;
  idx->id_bits = so.id_bits;
  idx->hs = so.hs;
  // about one directory entry per 4 records (at most 2^28 entries, 1 GiB):
  // a lookup's range then spans a cache line or two instead of a binary
  // search through hundreds of records
  {
    int db = 10;
    while (db < 28 && db < so.hs && ((uint64_t)1 << (db + 2)) < e.n_rec) ++db;
    idx->dir_bits = db;
  }
  const size_t b_keys = n * sizeof(Key128), b_lens = n, b_rec = e.n_rec * 8,
               b_dir = ((size_t(1) << idx->dir_bits) + 1) * 4;
  bool ok = cudaMalloc(&idx->keys, b_keys) == cudaSuccess &&
            cudaMalloc(&idx->lens, b_lens + 16) == cudaSuccess &&
            cudaMalloc(&idx->rec, b_rec + 8) == cudaSuccess &&
            cudaMalloc(&idx->dir, b_dir) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    xtn_index_free(idx);
    return XTN_ERR_OOM;
  }
  idx->bytes = (int64_t)(b_keys + b_lens + b_rec + b_dir);
  bool cp = cudaMemcpyAsync(idx->keys, e.keys, b_keys, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(idx->lens, e.lens, b_lens, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(idx->rec, so.rec, b_rec, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
  uint64_t* groups = ar.get<uint64_t>(1);
  if (!groups) cp = false;
  if (cp) cp = cudaMemsetAsync(groups, 0, 8, s) == cudaSuccess;
  if (cp)
    launch_build_dir(idx->rec, idx->n_rec, idx->dir_bits, 64 - idx->hs, idx->dir, groups, s);
  struct {
    uint64_t groups;
    uint32_t err;
  } h{0, 0};
  if (!cp || cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&h.groups, groups, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&h.err, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      host_sync(s) != cudaSuccess) {
    cudaGetLastError();
    xtn_index_free(idx);
    return XTN_ERR_CUDA;
  }
  if (h.err) {
    xtn_index_free(idx);
    return map_device_err(h.err);
  }
  idx->n_groups = h.groups;
  *out = idx;
  return XTN_OK;
}

// metric: 0 = Levenshtein, 1 = Hamming (the index's candidates serve both:
// Hamming neighbours within d share the string left after deleting the
// differing positions).
int search_query_impl(const xtn_index* idx, const uint8_t* q_seqs, const int64_t* q_offsets,
                      int64_t n_q, xtn_triple* out, int64_t cap, int64_t* n_out, cudaStream_t s,
                      int metric = 0) {
  if (!n_out) return XTN_ERR_INVALID_ARG;
  *n_out = 0;
  if (!idx || n_q < 0 || cap < 0 || !q_offsets) return XTN_ERR_INVALID_ARG;
  if (n_q >= (1ll << 31)) return XTN_ERR_TOO_LARGE;
  if (n_q == 0) return XTN_OK;
  int sms = 0;
  int rc = current_device_info(&sms);
  if (rc) return rc;
  Arena ar(s);
  uint32_t* err = ar.get<uint32_t>(4);
  XTN_ALLOC_OK(ar);
  XTN_CK(init_err(err, s));
  DevSeqs in;
  rc = stage_seqs(q_seqs, q_offsets, n_q, ar, s, &in);
  if (rc) return rc;
  Encoded e;
  rc = encode_and_count(in, idx->d, ar, err, s, &e);
  if (rc) return rc;
  const uint64_t n_qv = e.n_rec;
  uint32_t* qv_start = ar.get<uint32_t>(n_qv);
  uint32_t* qv_cnt = ar.get<uint32_t>(n_qv);
  uint32_t* qv_q = ar.get<uint32_t>(n_qv);
  uint64_t* cand_off = ar.get<uint64_t>(n_qv + 1);
  uint64_t* status = ar.get<uint64_t>(scan_status_bytes(n_qv) / 8 + 1);
  XTN_ALLOC_OK(ar);
  launch_query_lookup(e.keys, e.lens, e.eqprev, e.rec_off, n_q, n_qv, idx->d, idx->rec,
                      idx->n_rec, idx->dir, idx->dir_bits, 64 - idx->hs, qv_start, qv_cnt, qv_q,
                      sms, err, s);
  launch_scan_counts(qv_cnt, (int64_t)n_qv, cand_off, status, err, s);
  XTN_CK(cudaGetLastError());
  struct {
    uint64_t cand;
    uint32_t err;
  } hc{0, 0};
  {
    ReadBack rb(s);
    XTN_RC(rb.add(&hc.cand, cand_off + n_qv));
    XTN_RC(rb.add(&hc.err, err));
    XTN_RC(rb.wait());
  }
  if (hc.err) return map_device_err(hc.err);
  const uint64_t n_cand = hc.cand;
  idx->seen_cand += n_cand;
  idx->seen_qv += n_qv;
  if (n_cand == 0) return XTN_OK;
  if (n_cand >= (1ull << 32)) return XTN_ERR_TOO_LARGE;
  const uint32_t q_bits = bits_for((uint64_t)n_q);
  const uint32_t pair_bits = q_bits + idx->id_bits;
  if (pair_bits > 64) return XTN_ERR_TOO_LARGE;
  BackStage b;
  b.P1 = ar.get<uint64_t>(n_cand + 8);
  b.P2 = ar.get<uint64_t>(n_cand + 8);
  b.hist = ar.get<uint32_t>(MAX_PASSES * RADIX);
  b.digit_base = ar.get<uint64_t>(MAX_PASSES * RADIX);
  const int cfg_pairs = g_cfg_pairs.load();
  b.status = ar.get<uint64_t>(back_status_bytes(n_cand, cfg_pairs) / 8 + 1);
  b.counters = ar.get<uint64_t>(2);
  uint32_t* peq = ar.get<uint32_t>((size_t)n_q * PEQ_STRIDE);
  XTN_ALLOC_OK(ar);
  launch_query_emit(idx->rec, idx->n_rec, idx->id_bits, qv_start, qv_q, cand_off, n_qv, n_cand,
                    b.P1, sms, err, s);
  launch_peq(e.keys, e.lens, n_q, peq, s);
  XTN_CK(cudaGetLastError());
  OutRows o;
  rc = prepare_out(out, cap, n_cand, ar, &o);
  if (rc) return rc;
  rc = launch_back(b, n_cand, nullptr, pair_bits, idx->id_bits, peq, e.lens, (uint64_t)n_q,
                   idx->keys, idx->lens, (uint64_t)idx->n, nullptr, 0, idx->d, o.dev, o.dev_cap,
                   sms, err, s, cfg_pairs, metric);
  if (rc) return rc;
  struct {
    uint64_t rows;
    uint32_t err;
  } h{0, 0};
  {
    ReadBack rb(s);
    XTN_RC(rb.add(&h.rows, b.counters + 1));
    XTN_RC(rb.add(&h.err, err));
    XTN_RC(rb.wait());
  }
  if (h.err) return map_device_err(h.err);
  const uint64_t n_rows = h.rows;
  return finish_out(o, out, cap, n_rows, s, n_out);
}

int tcrdist_impl(const uint8_t* seqs, const int64_t* offsets, int64_t n, const xtn_triple* in_rows,
                 int64_t n_in, int max_score, xtn_triple* out, int64_t* n_out, cudaStream_t s) {
  if (!n_out) return XTN_ERR_INVALID_ARG;
  *n_out = 0;
  if (n < 0 || n_in < 0 || !offsets || (n_in > 0 && (!in_rows || !out))) return XTN_ERR_INVALID_ARG;
  if (n >= (1ll << 32)) return XTN_ERR_TOO_LARGE;
  if (n_in == 0 || n == 0) return n_in == 0 ? XTN_OK : XTN_ERR_INVALID_ARG;
  int sms = 0;
  int rc = current_device_info(&sms);
  if (rc) return rc;
  Arena ar(s);
  uint32_t* err = ar.get<uint32_t>(4);
  XTN_ALLOC_OK(ar);
  XTN_CK(init_err(err, s));
  DevSeqs in;
  rc = stage_seqs(seqs, offsets, n, ar, s, &in);
  if (rc) return rc;
  Encoded e;
  rc = encode_and_count(in, 0, ar, err, s, &e);
  if (rc) return rc;
  const xtn_triple* d_in = in_rows;
  if (!is_device_ptr(in_rows)) {
    xtn_triple* t = ar.get<xtn_triple>(n_in);
    XTN_ALLOC_OK(ar);
    XTN_CK(cudaMemcpyAsync(t, in_rows, n_in * sizeof(xtn_triple), cudaMemcpyHostToDevice, s));
    d_in = t;
  }
  const bool host_out = !is_device_ptr(out);
  xtn_triple* d_out = host_out ? ar.get<xtn_triple>(n_in) : out;
  uint64_t* status = ar.get<uint64_t>(verify_status_bytes(n_in) / 8 + 1);
  uint64_t* d_total = ar.get<uint64_t>(1);
  XTN_ALLOC_OK(ar);
  launch_tcrdist_filter(d_in, n_in, e.keys, e.lens, n, max_score, d_out, status, err, d_total, s);
  XTN_CK(cudaGetLastError());
  uint64_t total = 0;
  rc = read_back(&total, d_total, 1, s);
  if (rc) return rc;
  uint32_t herr = 0;
  rc = read_back(&herr, err, 1, s);
  if (rc) return rc;
  if (herr) return map_device_err(herr);
  if (host_out && total > 0) {
    XTN_CK(cudaMemcpyAsync(out, d_out, total * sizeof(xtn_triple), cudaMemcpyDeviceToHost, s));
    XTN_CK(host_sync(s));
  }
  *n_out = (int64_t)total;
  return XTN_OK;
}

}  // namespace
}  // namespace xtn

// ======================================================================
// Plans (sync-free self-search, batched mode)
// ======================================================================
struct xtn_plan {
  int device = 0;
  int d = 0;
  int64_t n = 0;
  uint64_t rec_cap = 0, pair_cap = 0, g_cap = 0;
  uint32_t id_bits = 0;
  int hs = 0, cfg_rec = 0, cfg_pair = 0, hist_mode = 0, group_mode = 0, sms = 0;
  uint64_t* bucket_start = nullptr;
  uint8_t* seg_area = nullptr;  // singleton filter's segment counter and flags
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int64_t* off = nullptr;
  uint32_t* seq_rep = nullptr;
  xtn::Key128* keys = nullptr;
  uint8_t* lens = nullptr;
  uint32_t *eqprev = nullptr, *vcount = nullptr, *hist = nullptr, *peq = nullptr, *err = nullptr;
  uint64_t *rec_off = nullptr, *A = nullptr, *B = nullptr, *digit_base = nullptr;
  uint64_t *status = nullptr, *flags = nullptr, *counters = nullptr;
  uint32_t *S = nullptr, *E = nullptr;
  uint64_t* pair_off = nullptr;
  uint64_t* sorted = nullptr;
  xtn::BackStage back;
  xtn_triple* rows = nullptr;

  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    const size_t b = (count ? count : 1) * sizeof(T) + 64;
    if (cudaMalloc(&p, b) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    allocs.push_back(p);
    bytes += (int64_t)b;
    return static_cast<T*>(p);
  }
  ~xtn_plan() {
    for (void* p : allocs) cudaFree(p);
  }
};

namespace xtn {
namespace {

int plan_create_impl(const int64_t* offsets, int64_t n, int d, const int64_t* rep_offsets,
                     int64_t n_rep, int64_t pair_capacity, xtn_plan** out) {
  if (!out) return XTN_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || d < 0 || d > XTN_MAX_D || !offsets) return XTN_ERR_INVALID_ARG;
  if (n >= (1ll << 32)) return XTN_ERR_TOO_LARGE;
  if (rep_offsets && n_rep < 1) return XTN_ERR_INVALID_ARG;
  int sms = 0;
  int rc = current_device_info(&sms);
  if (rc) return rc;
  std::vector<int64_t> h(n + 1);
  if (is_device_ptr(offsets)) {
    if (cudaMemcpy(h.data(), offsets, (n + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return XTN_ERR_CUDA;
    }
  } else {
    std::memcpy(h.data(), offsets, (n + 1) * 8);
  }
  rc = check_host_offsets(h.data(), n);
  if (rc) return rc;
  uint64_t rec_cap = 0;  // every deletion subset: canonical ones are a subset
  for (int64_t i = 0; i < n; ++i) rec_cap += variant_count((uint32_t)(h[i + 1] - h[i]), (uint32_t)d);
  if (rec_cap >= (1ull << 32)) return XTN_ERR_TOO_LARGE;
  xtn_plan* p = new xtn_plan;
  cudaGetDevice(&p->device);
  p->d = d;
  p->n = n;
  p->sms = sms;
  p->rec_cap = rec_cap;
  p->g_cap = rec_cap / 2 + 1;
  p->pair_cap = pair_capacity > 0 ? (uint64_t)pair_capacity
                                  : std::max<uint64_t>(rec_cap / 8, 65536);
  if (p->pair_cap >= (1ull << 32)) p->pair_cap = (1ull << 32) - 1;
  p->id_bits = bits_for((uint64_t)n);
  p->hs = choose_hash_bits(rec_cap, p->id_bits);
  p->cfg_rec = g_cfg_records.load();
  p->cfg_pair = g_cfg_pairs.load();
  p->hist_mode = g_record_hist.load();
  p->group_mode = g_grouping.load();
  const size_t st = std::max({radix_status_bytes((int64_t)rec_cap, p->cfg_rec),
                              group_status_bytes((int64_t)rec_cap),
                              scan_status_bytes((int64_t)p->g_cap), scan_status_bytes(n)});
  p->off = p->alloc<int64_t>(n + 1);
  p->keys = p->alloc<Key128>(n);
  p->lens = p->alloc<uint8_t>(n);
  p->eqprev = p->alloc<uint32_t>(n);
  p->vcount = p->alloc<uint32_t>(n);
  p->rec_off = p->alloc<uint64_t>(n + 1);
  p->A = p->alloc<uint64_t>(rec_cap + 8);
  p->B = p->alloc<uint64_t>(rec_cap + 8);
  p->hist = p->alloc<uint32_t>(MAX_PASSES * RADIX);
  p->digit_base = p->alloc<uint64_t>(MAX_PASSES * RADIX);
  p->status = p->alloc<uint64_t>(st / 8 + 1);
  p->flags = p->alloc<uint64_t>(group_flag_words((int64_t)rec_cap));
  p->bucket_start = p->alloc<uint64_t>(bucket_start_words(rec_cap, p->hs, p->group_mode));
  p->seg_area = p->alloc<uint8_t>(seg_area_bytes(rec_cap, p->hs));
  p->counters = p->alloc<uint64_t>(4);
  p->err = p->alloc<uint32_t>(4);
  p->peq = p->alloc<uint32_t>((size_t)n * PEQ_STRIDE);
  p->back.P1 = p->alloc<uint64_t>(p->pair_cap + 8);
  p->back.P2 = p->alloc<uint64_t>(p->pair_cap + 8);
  p->back.hist = p->alloc<uint32_t>(MAX_PASSES * RADIX);
  p->back.digit_base = p->alloc<uint64_t>(MAX_PASSES * RADIX);
  p->back.status = p->alloc<uint64_t>(back_status_bytes(p->pair_cap, p->cfg_pair) / 8 + 1);
  p->back.counters = p->alloc<uint64_t>(2);
  p->rows = p->alloc<xtn_triple>(p->pair_cap);
  if (rep_offsets) p->seq_rep = p->alloc<uint32_t>(n);
  bool ok = p->rows && p->back.counters && p->back.status && p->back.digit_base && p->back.hist &&
            p->back.P2 && p->back.P1 && p->peq && p->err && p->counters && p->flags && p->status &&
            p->bucket_start && p->seg_area &&
            p->digit_base && p->hist && p->B && p->A && p->rec_off && p->vcount && p->eqprev &&
            p->lens && p->keys && p->off && (!rep_offsets || p->seq_rep);
  if (!ok) {
    delete p;
    return XTN_ERR_OOM;
  }
  // which buffer ends up sorted depends on the pass count; groups live in the other
  const bool in_b = sorted_in_b(rec_cap, p->hs, p->group_mode);
  p->sorted = in_b ? p->B : p->A;
  uint64_t* spare = in_b ? p->A : p->B;
  p->S = reinterpret_cast<uint32_t*>(spare);
  p->E = p->S + p->g_cap;
  p->pair_off = reinterpret_cast<uint64_t*>(p->E + p->g_cap);
  cudaStream_t s = nullptr;
  if (cudaMemcpy(p->off, h.data(), (n + 1) * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return XTN_ERR_CUDA;
  }
  if (rep_offsets) {
    Arena ar(s);
    rc = stage_reps(rep_offsets, n_rep, n, &ar, s, p->seq_rep);
    if (rc == XTN_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = XTN_ERR_CUDA;
    if (rc) {
      delete p;
      return rc;
    }
  }
  *out = p;
  return XTN_OK;
}

int plan_run_impl(xtn_plan* p, const uint8_t* seqs, cudaStream_t s) {
  if (!p || !seqs) return XTN_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return XTN_ERR_INVALID_ARG;
  const int64_t n = p->n;
  const int lo = 64 - p->hs;
  XTN_CK(init_err(p->err, s));
  XTN_CK(cudaMemsetAsync(p->counters, 0, 32, s));
  XTN_CK(cudaMemsetAsync(p->hist, 0, MAX_PASSES * RADIX * 4, s));
  launch_encode(seqs, p->off, n, p->d, p->keys, p->lens, p->eqprev, p->vcount, p->err, s);
  launch_scan_counts(p->vcount, n, p->rec_off, p->status, p->err, s);
  uint64_t* sorted = nullptr;
  const uint64_t* n_rec = p->rec_off + n;  // known on the device only
  GroupScratch gs;
  gs.bucket_start = p->bucket_start;
  gs.flags = p->flags;
  gs.gstatus = p->status;
  const bool direct = p->group_mode != 1;  // bucket modes emit most candidates while grouping
  if (direct) {
    gs.cand = p->back.P1;
    gs.cand_cap = p->pair_cap;
    gs.cand_count = p->counters + 2;
    gs.seg_area = p->seg_area;
  }
  XTN_CK(expand_sort_launch(p->keys, p->lens, p->eqprev, p->rec_off, n, p->d, p->seq_rep,
                            p->id_bits, p->A, p->B, p->rec_cap, lo, p->hist, p->digit_base,
                            p->status, p->cfg_rec, p->hist_mode, p->group_mode, gs, p->sms, p->err,
                            s, n_rec, &sorted));
  if (sorted != p->sorted) return XTN_ERR_CUDA;
  launch_group_finish(p->flags, (int64_t)p->rec_cap, n_rec, p->S, p->E, p->g_cap, p->status,
                      p->err, p->counters, s);
  launch_scan_group_pairs(p->S, p->E, (int64_t)p->g_cap, p->counters, p->pair_off, p->status,
                          p->err, s);
  launch_emit_pairs(sorted, p->rec_cap, p->S, p->pair_off, (int64_t)p->g_cap, p->counters,
                    p->pair_cap, p->id_bits, p->back.P1, direct ? p->counters + 2 : nullptr,
                    p->counters + 1, p->sms, p->err, s);
  launch_peq(p->keys, p->lens, n, p->peq, s);
  XTN_CK(cudaGetLastError());
  return launch_back(p->back, p->pair_cap, p->counters + 1, 2 * p->id_bits, p->id_bits, p->peq,
                     p->lens, (uint64_t)n, p->keys, p->lens, (uint64_t)n, p->seq_rep, 1, p->d,
                     p->rows, (int64_t)p->pair_cap, p->sms, p->err, s, p->cfg_pair);
}

int plan_result_impl(xtn_plan* p, xtn_triple* out, int64_t cap, int64_t* n_out, cudaStream_t s) {
  if (!n_out) return XTN_ERR_INVALID_ARG;
  *n_out = 0;
  if (!p || cap < 0 || (cap > 0 && !out)) return XTN_ERR_INVALID_ARG;
  struct {
    uint64_t pairs, rows;
    uint32_t err;
  } h{0, 0, 0};
  XTN_CK(cudaMemcpyAsync(&h.pairs, p->counters + 1, 8, cudaMemcpyDeviceToHost, s));
  XTN_CK(cudaMemcpyAsync(&h.rows, p->back.counters + 1, 8, cudaMemcpyDeviceToHost, s));
  XTN_CK(cudaMemcpyAsync(&h.err, p->err, 4, cudaMemcpyDeviceToHost, s));
  XTN_CK(host_sync(s));
  if (h.err & DERR_CAPACITY) {
    *n_out = (int64_t)h.pairs;
    return XTN_ERR_CAPACITY;
  }
  if (h.err) return map_device_err(h.err);
  *n_out = (int64_t)h.rows;
  const int64_t w = std::min<int64_t>(cap, (int64_t)h.rows);
  if (w > 0) {
    XTN_CK(cudaMemcpyAsync(out, p->rows, w * sizeof(xtn_triple), cudaMemcpyDefault, s));
    XTN_CK(host_sync(s));
  }
  return (int64_t)h.rows > cap ? XTN_ERR_BUFFER_TOO_SMALL : XTN_OK;
}

}  // namespace
}  // namespace xtn

// ======================================================================
// extern "C"
// ======================================================================
extern "C" {

const char* xtn_status_string(int status) {
  switch (status) {
    case XTN_OK: return "ok";
    case XTN_ERR_INVALID_ARG: return "invalid argument";
    case XTN_ERR_BAD_RESIDUE: return "residue outside the 20-letter amino-acid alphabet";
    case XTN_ERR_SEQ_TOO_LONG: return "sequence longer than XTN_MAX_LEN";
    case XTN_ERR_OOM: return "out of device memory";
    case XTN_ERR_BUFFER_TOO_SMALL: return "output buffer too small";
    case XTN_ERR_CUDA: return "CUDA runtime error";
    case XTN_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case XTN_ERR_TOO_LARGE: return "problem exceeds 2^32-1 records or pairs";
    case XTN_ERR_CAPACITY: return "more candidate pairs than the plan's capacity";
  }
  return "unknown status";
}

int xtn_version(void) { return 10000; }

int xtn_search_self(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                    const int64_t* rep_offsets, int64_t n_rep, xtn_triple* out, int64_t cap,
                    int64_t* n_out, xtn_stream_t stream) {
  xtn::HostSpan span("host_call_search_self");
  return xtn::search_self_impl(seqs, offsets, n, d, rep_offsets, n_rep, out, cap, n_out,
                               reinterpret_cast<cudaStream_t>(stream));
}

int xtn_search_self_hamming(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                            const int64_t* rep_offsets, int64_t n_rep, xtn_triple* out,
                            int64_t cap, int64_t* n_out, xtn_stream_t stream) {
  xtn::HostSpan span("host_call_search_self");
  return xtn::search_self_impl(seqs, offsets, n, d, rep_offsets, n_rep, out, cap, n_out,
                               reinterpret_cast<cudaStream_t>(stream), -1, 1);
}

int xtn_search_between(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                       const int64_t* rep_offsets, int64_t n_rep, int metric, xtn_triple* out,
                       int64_t cap, int64_t* n_out, xtn_stream_t stream) {
  if (n_out) *n_out = 0;
  if (metric != XTN_METRIC_LEVENSHTEIN && metric != XTN_METRIC_HAMMING)
    return XTN_ERR_INVALID_ARG;
  xtn::HostSpan span("host_call_search_between");
  return xtn::search_self_impl(seqs, offsets, n, d, rep_offsets, n_rep, out, cap, n_out,
                               reinterpret_cast<cudaStream_t>(stream), -1, metric, true);
}

int xtn_search_self_streaming(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                              const int64_t* rep_offsets, int64_t n_rep, int metric, int between,
                              int64_t max_pass_records, xtn_triple* out, int64_t cap,
                              int64_t* n_out, int64_t* n_passes, xtn_stream_t stream) {
  xtn::HostSpan span("host_call_search_streaming");
  return xtn::search_stream_impl(seqs, offsets, n, d, rep_offsets, n_rep, metric, between != 0,
                                 max_pass_records, out, cap, n_out, n_passes,
                                 reinterpret_cast<cudaStream_t>(stream));
}

int xtn_index_build(const uint8_t* seqs, const int64_t* offsets, int64_t n, int d,
                    xtn_stream_t stream, xtn_index** out) {
  return xtn::index_build_impl(seqs, offsets, n, d, reinterpret_cast<cudaStream_t>(stream), out);
}

int xtn_index_free(xtn_index* idx) {
  if (!idx) return XTN_OK;
  cudaFree(idx->keys);
  cudaFree(idx->lens);
  cudaFree(idx->rec);
  cudaFree(idx->dir);
  delete idx;
  return XTN_OK;
}

int xtn_index_info(const xtn_index* idx, int64_t* n, int* d, int64_t* n_records,
                   int64_t* device_bytes) {
  if (!idx) return XTN_ERR_INVALID_ARG;
  if (n) *n = idx->n;
  if (d) *d = idx->d;
  if (n_records) *n_records = (int64_t)idx->n_rec;
  if (device_bytes) *device_bytes = idx->bytes;
  return XTN_OK;
}

int xtn_search_paired(const uint8_t* a_seqs, const int64_t* a_offsets, const uint8_t* b_seqs,
                      const int64_t* b_offsets, int64_t n, int d, xtn_triple* out, int64_t cap,
                      int64_t* n_out, xtn_stream_t stream) {
  xtn::HostSpan span("host_call_search_paired");
  if (!b_offsets) {
    if (n_out) *n_out = 0;
    return XTN_ERR_INVALID_ARG;
  }
  return xtn::search_self_impl(a_seqs, a_offsets, n, d, nullptr, 0, out, cap, n_out,
                               reinterpret_cast<cudaStream_t>(stream), -1, 2, false, b_seqs,
                               b_offsets);
}

int xtn_search_query(const xtn_index* idx, const uint8_t* q_seqs, const int64_t* q_offsets,
                     int64_t n_q, xtn_triple* out, int64_t cap, int64_t* n_out,
                     xtn_stream_t stream) {
  xtn::HostSpan span("host_call_search_query");
  return xtn::search_query_impl(idx, q_seqs, q_offsets, n_q, out, cap, n_out,
                                reinterpret_cast<cudaStream_t>(stream));
}

int xtn_search_query_scratch(const xtn_index* idx, const int64_t* q_offsets, int64_t n_q,
                             int64_t* bytes) {
  using namespace xtn;
  if (!bytes) return XTN_ERR_INVALID_ARG;
  *bytes = 0;
  if (!idx || n_q < 0 || (n_q > 0 && !q_offsets)) return XTN_ERR_INVALID_ARG;
  if (n_q == 0) return XTN_OK;
  if (q_offsets[0] != 0) return XTN_ERR_INVALID_ARG;
  // query variants: every deletion subset of <= d positions (the canonical
  // ones the search expands are at most that many)
  uint64_t n_qv = 0;
  for (int64_t q = 0; q < n_q; ++q) {
    const int64_t L = q_offsets[q + 1] - q_offsets[q];
    if (L < 0) return XTN_ERR_INVALID_ARG;
    if (L > XTN_MAX_LEN) return XTN_ERR_SEQ_TOO_LONG;
    n_qv += variant_count((uint32_t)L, (uint32_t)idx->d);
  }
  const uint64_t letters = (uint64_t)q_offsets[n_q];
  // candidates per query variant: what this index has given so far, else
  // its mean group size; 1.5x margin
  const uint64_t sc = idx->seen_cand.load(), sq = idx->seen_qv.load();
  double rate = sq ? (double)sc / (double)sq
                   : (idx->n_groups ? (double)idx->n_rec / (double)idx->n_groups : 1.0);
  const uint64_t n_cand = (uint64_t)(1.5 * rate * (double)n_qv) + 1024;
  const int cfg = g_cfg_pairs.load();
  const uint64_t n = (uint64_t)n_q;
  const uint64_t per_buffer = 64 + 256;  // arena spare bytes and alignment
  uint64_t b = 0;
  b += 16 + letters + 8 * (n + 1);                                   // errors, staging
  b += n * (16 + 1 + 4 + 4) + 8 * (n + 1) + scan_status_bytes((int64_t)n);  // encode
  b += n_qv * 12 + 8 * (n_qv + 1) + scan_status_bytes((int64_t)n_qv);      // lookup
  b += 16 * (n_cand + 8) + MAX_PASSES * RADIX * 12 + 16;             // candidate words
  b += back_status_bytes(n_cand, cfg) + n * 4 * PEQ_STRIDE;          // sort, match vectors
  b += 12 * n_cand;                                                  // rows for host output
  b += 24 * per_buffer;
  *bytes = (int64_t)b;
  return XTN_OK;
}

int xtn_search_query_hamming(const xtn_index* idx, const uint8_t* q_seqs,
                             const int64_t* q_offsets, int64_t n_q, xtn_triple* out, int64_t cap,
                             int64_t* n_out, xtn_stream_t stream) {
  xtn::HostSpan span("host_call_search_query_hamming");
  return xtn::search_query_impl(idx, q_seqs, q_offsets, n_q, out, cap, n_out,
                                reinterpret_cast<cudaStream_t>(stream), 1);
}

int xtn_tcrdist_filter(const uint8_t* seqs, const int64_t* offsets, int64_t n,
                       const xtn_triple* in, int64_t n_in, int max_score, xtn_triple* out,
                       int64_t* n_out, xtn_stream_t stream) {
  return xtn::tcrdist_impl(seqs, offsets, n, in, n_in, max_score, out, n_out,
                           reinterpret_cast<cudaStream_t>(stream));
}

int xtn_plan_create(const int64_t* offsets, int64_t n, int d, const int64_t* rep_offsets,
                    int64_t n_rep, int64_t pair_capacity, xtn_plan** out) {
  return xtn::plan_create_impl(offsets, n, d, rep_offsets, n_rep, pair_capacity, out);
}

int xtn_plan_run(xtn_plan* plan, const uint8_t* seqs, xtn_stream_t stream) {
  return xtn::plan_run_impl(plan, seqs, reinterpret_cast<cudaStream_t>(stream));
}

int xtn_plan_result(xtn_plan* plan, xtn_triple* out, int64_t cap, int64_t* n_out,
                    xtn_stream_t stream) {
  return xtn::plan_result_impl(plan, out, cap, n_out, reinterpret_cast<cudaStream_t>(stream));
}

int xtn_plan_info(const xtn_plan* plan, int64_t* record_capacity, int64_t* pair_capacity,
                  int64_t* device_bytes) {
  if (!plan) return XTN_ERR_INVALID_ARG;
  if (record_capacity) *record_capacity = (int64_t)plan->rec_cap;
  if (pair_capacity) *pair_capacity = (int64_t)plan->pair_cap;
  if (device_bytes) *device_bytes = plan->bytes;
  return XTN_OK;
}

int xtn_plan_stats(xtn_plan* plan, int64_t* records, int64_t* groups, int64_t* candidates,
                   int64_t* survivors, xtn_stream_t stream) {
  if (!plan) return XTN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint64_t h[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(&h[0], plan->rec_off + plan->n, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&h[1], plan->counters, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&h[3], plan->back.counters, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return XTN_ERR_CUDA;
  }
  if (records) *records = (int64_t)h[0];
  if (groups) *groups = (int64_t)h[1];
  if (candidates) *candidates = (int64_t)h[2];
  if (survivors) *survivors = (int64_t)h[3];
  return XTN_OK;
}

int xtn_plan_free(xtn_plan* plan) {
  delete plan;
  return XTN_OK;
}

int xtn_tune_set(int knob, int value) {
  if (value < 0 || value >= xtn_tune_count(knob)) return XTN_ERR_INVALID_ARG;
  switch (knob) {
    case XTN_TUNE_RECORD_HISTOGRAM: xtn::g_record_hist.store(value); return XTN_OK;
    case XTN_TUNE_GROUPING: xtn::g_grouping.store(value); return XTN_OK;
    case XTN_TUNE_SORT_RECORDS: xtn::cfg_records().store(value); return XTN_OK;
    case XTN_TUNE_SORT_PAIRS: xtn::cfg_pairs().store(value); return XTN_OK;
    case XTN_TUNE_FILTER_SEGMENT: xtn::g_filter_fx.store(value); return XTN_OK;
  }
  return XTN_ERR_INVALID_ARG;
}

int xtn_tune_get(int knob) {
  switch (knob) {
    case XTN_TUNE_SORT_RECORDS: return xtn::cfg_records().load();
    case XTN_TUNE_SORT_PAIRS: return xtn::cfg_pairs().load();
    case XTN_TUNE_RECORD_HISTOGRAM: return xtn::g_record_hist.load();
    case XTN_TUNE_GROUPING: return xtn::g_grouping.load();
    case XTN_TUNE_FILTER_SEGMENT: return xtn::g_filter_fx.load();
  }
  return XTN_ERR_INVALID_ARG;
}

int xtn_tune_count(int knob) {
  switch (knob) {
    case XTN_TUNE_SORT_RECORDS:
    case XTN_TUNE_SORT_PAIRS: return xtn::onesweep_configs();
    case XTN_TUNE_RECORD_HISTOGRAM: return 2;
    case XTN_TUNE_GROUPING: return 3;
    case XTN_TUNE_FILTER_SEGMENT: return 4;
  }
  return XTN_ERR_INVALID_ARG;
}

int xtn_scratch_trim(void) { return xtn::trim_scratch(); }

int xtn_set_wait_limit(int64_t polls) {
  if (polls < 0 || polls > (int64_t)xtn::SPIN_LIMIT) return XTN_ERR_INVALID_ARG;
  xtn::g_wait_limit.store((uint32_t)polls);
  return XTN_OK;
}

int xtn_profile_enable(int on) {
  xtn::g_prof_on.store(on != 0);
  return XTN_OK;
}

int xtn_profile_only(const char* name) {
  const size_t len = name ? std::strlen(name) : 0;
  if (len >= sizeof(xtn::g_prof_only)) return XTN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(xtn::g_prof_mu);
  std::memcpy(xtn::g_prof_only, len ? name : "", len + 1);
  xtn::g_prof_filtered.store(len > 0);
  return XTN_OK;
}

int xtn_profile_report(char* buf, int64_t buf_len) {
  std::vector<xtn::ProfRec> recs;
  {
    std::lock_guard<std::mutex> g(xtn::g_prof_mu);
    recs.swap(xtn::g_prof);
  }
  struct Agg {
    int64_t launches = 0;
    double ms = 0, bytes = 0;
  };
  std::map<std::string, Agg> agg;
  for (auto& r : recs) {
    float ms = (float)r.host_ms;
    if (r.a) {
      cudaEventSynchronize(r.b);
      if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) cudaGetLastError();
    }
    Agg& a = agg[r.name];
    a.launches++;
    a.ms += ms;
    a.bytes += r.bytes;
  }
  {
    std::lock_guard<std::mutex> g(xtn::g_prof_mu);
    for (auto& r : recs) {
      if (!r.a) continue;
      xtn::g_ev_pool.push_back(r.a);
      xtn::g_ev_pool.push_back(r.b);
    }
  }
  std::string s;
  char line[256];
  for (auto& kv : agg) {
    std::snprintf(line, sizeof line, "%s %lld %.6f %.0f\n", kv.first.c_str(),
                  (long long)kv.second.launches, kv.second.ms, kv.second.bytes);
    s += line;
  }
  if (buf && buf_len > 0) {
    const size_t w = std::min<size_t>(s.size(), (size_t)buf_len - 1);
    std::memcpy(buf, s.data(), w);
    buf[w] = '\0';
  }
  return (int)agg.size();
}

}  // extern "C"
