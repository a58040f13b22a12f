// xtn_tcrdist_filter_noalloc: the TCRdist post-filter with every piece of
// scratch memory in one fixed, file-scope device array, for callers that
// cannot allocate device memory: a process that must stay inside a fixed
// device-memory budget, or a library loaded into a host application whose
// own allocator owns the device memory, so that a cudaMalloc of ours could
// fail or take memory the host application counted on.  The same kernels as
// xtn_tcrdist_filter run; only the place their scratch lives differs.  The
// call reads the row count back, so it waits for its stream.
#include <mutex>

#include "xtn_common.cuh"
#include "xtn_kernels.h"

namespace xtn {
namespace {

constexpr int64_t NA_MAX_SEQS = XTN_NOALLOC_MAX_SEQS;
constexpr int64_t NA_MAX_ROWS = XTN_NOALLOC_MAX_ROWS;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// Layout of the scratch array (byte offsets, each section 256-byte aligned).
constexpr size_t OFF_KEYS = 0;                                                // Key128[]
constexpr size_t OFF_LENS = align256(OFF_KEYS + 16 * (size_t)NA_MAX_SEQS);   // uint8_t[]
constexpr size_t OFF_EQ = align256(OFF_LENS + (size_t)NA_MAX_SEQS);          // uint32_t[]
constexpr size_t OFF_VCOUNT = align256(OFF_EQ + 4 * (size_t)NA_MAX_SEQS);    // uint32_t[]
constexpr size_t OFF_STATUS = align256(OFF_VCOUNT + 4 * (size_t)NA_MAX_SEQS);
constexpr size_t STATUS_BYTES = align256(verify_status_bytes_for(NA_MAX_ROWS));
constexpr size_t OFF_COUNTERS = OFF_STATUS + STATUS_BYTES;                    // err, total
constexpr size_t NA_BYTES = OFF_COUNTERS + 256;

}  // namespace
}  // namespace xtn

// Host code may only use this name through cudaGetSymbolAddress: on the host
// it is a stand-in, not a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[xtn::NA_BYTES];

namespace xtn {
namespace {

std::mutex g_na_mu;
void* g_na_addr[256] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does it).
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return XTN_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(g_na_mu);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return XTN_ERR_CUDA;
    }
    g_na_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_na_addr[dev]);
  return XTN_OK;
}

// Device memory of the current device (or managed memory, which any device
// may reach): a buffer of another GPU would be read through this device's
// launch, so it is refused like a host buffer.
bool on_device(const void* p) {
  cudaPointerAttributes a;
  int dev = -1;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int map_err(uint32_t e) {
  if (e & DERR_TIMEOUT) return XTN_ERR_DEVICE_TIMEOUT;
  if (e & DERR_BAD_RESIDUE) return XTN_ERR_BAD_RESIDUE;
  if (e & DERR_TOO_LONG) return XTN_ERR_SEQ_TOO_LONG;
  if (e & DERR_RANGE) return XTN_ERR_INVALID_ARG;
  return XTN_OK;
}

}  // namespace
}  // namespace xtn

extern "C" int xtn_tcrdist_filter_noalloc(const uint8_t* seqs, const int64_t* offsets, int64_t n,
                                          const xtn_triple* in, int64_t n_in, int max_score,
                                          xtn_triple* out, int64_t* n_out, xtn_stream_t stream) {
  using namespace xtn;
  if (!n_out) return XTN_ERR_INVALID_ARG;
  *n_out = 0;
  if (n < 0 || n_in < 0 || !offsets) return XTN_ERR_INVALID_ARG;
  if (n > NA_MAX_SEQS || n_in > NA_MAX_ROWS) return XTN_ERR_TOO_LARGE;
  if (n_in == 0) return XTN_OK;
  if (n == 0 || !in || !out) return XTN_ERR_INVALID_ARG;
  // every buffer must already be on the device: a host buffer would need a
  // device copy, i.e. an allocation
  if (!on_device(offsets) || !on_device(in) || !on_device(out) || !on_device(seqs))
    return XTN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  Key128* keys = reinterpret_cast<Key128*>(base + OFF_KEYS);
  uint8_t* lens = base + OFF_LENS;
  uint32_t* eq = reinterpret_cast<uint32_t*>(base + OFF_EQ);
  uint32_t* vcount = reinterpret_cast<uint32_t*>(base + OFF_VCOUNT);
  uint64_t* status = reinterpret_cast<uint64_t*>(base + OFF_STATUS);
  uint32_t* err = reinterpret_cast<uint32_t*>(base + OFF_COUNTERS);
  uint64_t* total = reinterpret_cast<uint64_t*>(base + OFF_COUNTERS + 16);
  // the array keeps the previous call's contents: clear what must start at 0
  if (cudaMemsetAsync(base + OFF_COUNTERS, 0, 256, s) != cudaSuccess) {
    cudaGetLastError();
    return XTN_ERR_CUDA;
  }
  launch_encode(seqs, offsets, n, 0, keys, lens, eq, vcount, err, s);
  launch_tcrdist_filter(in, n_in, keys, lens, n, max_score, out, status, err, total, s);
  if (cudaGetLastError() != cudaSuccess) return XTN_ERR_CUDA;
  uint64_t h_total = 0;
  uint32_t h_err = 0;
  if (cudaMemcpyAsync(&h_total, total, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return XTN_ERR_CUDA;
  }
  if (h_err) return map_err(h_err);
  *n_out = (int64_t)h_total;
  return XTN_OK;
}
