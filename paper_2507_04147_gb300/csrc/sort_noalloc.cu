// sort_noalloc.cu -- a3fr_sort_pairs_noalloc: the stable radix sort of a3fr_sort_pairs
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a real-time render thread whose frame budget cannot
// absorb the device-wide synchronisation that cudaMalloc/cudaFree may cause, or host code
// running inside an engine that owns every byte of device memory through its own
// allocator.  For them this entry point takes its scratch (the ping-pong key/value
// buffers, the digit histograms, the partition counters and the look-back words) from one
// file-scope device array of fixed size instead of from the caller or from an allocator.
//
// The array is a static __device__ symbol, so every GPU that loads the library holds it
// until the process exits.  In host code its name is only a stand-in, not a device
// address, so the address is looked up with cudaGetSymbolAddress once per device, with
// that device current, the first time the entry point is called on it.
#include <mutex>

#include "../../include/a3fr.h"
#include "common.cuh"

namespace {

constexpr size_t kMaxPairs = A3FR_NOALLOC_MAX_PAIRS;
constexpr size_t kAltBytes = kMaxPairs * (sizeof(uint64_t) + sizeof(uint32_t));
constexpr size_t kStateBytes = 256;            // device count + status word
constexpr size_t kWorkspaceBytes = 1u << 20;   // histograms, counters, look-back words
constexpr size_t kScratchBytes = kAltBytes + kStateBytes + kWorkspaceBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

__global__ void set_count_kernel(uint32_t *state, uint32_t n) {
  state[0] = n;   // device-resident pair count
  state[4] = 0u;  // status word
}

// Device address of the scratch array on the current device (set up on first use).
cudaError_t scratch_on_current_device(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int a3fr_sort_pairs_noalloc(uint64_t *keys, uint32_t *vals, size_t n, int key_bits,
                                       void *stream) {
  if (n == 0) return A3FR_OK;
  if (!keys || !vals || key_bits < 1 || key_bits > 64) return A3FR_ERR_INVALID_ARG;
  if (n > kMaxPairs) return A3FR_ERR_CAPACITY;
  if (a3fr::sort_workspace_bytes(n) > kWorkspaceBytes) return A3FR_ERR_CAPACITY;
  unsigned char *base = nullptr;
  if (scratch_on_current_device(&base) != cudaSuccess) return A3FR_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint64_t *keys_alt = reinterpret_cast<uint64_t *>(base);
  uint32_t *vals_alt = reinterpret_cast<uint32_t *>(base + kMaxPairs * sizeof(uint64_t));
  uint32_t *state = reinterpret_cast<uint32_t *>(base + kAltBytes);
  void *workspace = base + kAltBytes + kStateBytes;
  set_count_kernel<<<1, 1, 0, st>>>(state, static_cast<uint32_t>(n));
  if (cudaGetLastError() != cudaSuccess) return A3FR_ERR_CUDA;
  bool in_alt = false;
  if (a3fr::launch_sort(keys, vals, keys_alt, vals_alt, state, n, key_bits, workspace,
                        state + 4, &in_alt, st) != cudaSuccess)
    return A3FR_ERR_CUDA;
  if (in_alt) {
    if (cudaMemcpyAsync(keys, keys_alt, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(vals, vals_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
      return A3FR_ERR_CUDA;
  }
  // the status word the look-back sets when a bounded wait gives up (the result is then
  // not sorted), read once the sort has finished; a host stack variable, so still nothing
  // is allocated
  uint32_t host_status = 0;
  if (cudaMemcpyAsync(&host_status, state + 4, sizeof host_status, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return A3FR_ERR_CUDA;
  return (host_status & a3fr::kStatusTimeout) ? A3FR_ERR_TIMEOUT : A3FR_OK;
}
