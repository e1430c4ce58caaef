// binning.cu -- tile binning of the projected Gaussians (Sec. 2.3: "determining which
// ellipses intersect with a given pixel tile"): offsets of each Gaussian's instances,
// emission of the 64-bit (tile << 32 | depth bits) keys, and the per-tile ranges of the
// sorted keys ("subsets of Gaussian points on each tile", Sec. 3.5).
//
// Offsets use reduce-then-scan: preprocess already reduced the touched-tile counts of each
// 128-Gaussian block, scan_blocks turns the block totals into block offsets in one CTA,
// and emit_keys re-scans its block in registers/shared memory.  No step waits on another
// block, so nothing here can stall.
#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// counts[0] = instances kept (<= capacity), counts[1..2] = per-eye totals,
// counts[3] = unclamped total (low 32 bits).  block_offsets are 64-bit.
__global__ void __launch_bounds__(kScanThreads)
scan_blocks_kernel(const uint32_t *__restrict__ block_sums, int n_blocks,
                   unsigned long long *__restrict__ block_offsets, uint32_t *__restrict__ counts,
                   uint32_t capacity, uint32_t *__restrict__ status) {
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_carry;
  __shared__ uint64_t s_eye[2];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) { s_carry = 0; s_eye[0] = 0; s_eye[1] = 0; }
  uint64_t e0 = 0, e1 = 0;
  __syncthreads();
  for (int base = 0; base < n_blocks; base += kScanThreads) {
    const int b = base + t;
    uint64_t v = 0;
    if (b < n_blocks) {
      const uint32_t a0 = block_sums[2 * b], a1 = block_sums[2 * b + 1];
      e0 += a0;
      e1 += a1;
      v = (uint64_t)a0 + a1;
    }
    const uint64_t incl = warp_incl_scan(v, lane);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint64_t w = s_warp[lane];
      s_warp[lane] = warp_incl_scan(w, lane) - w;   // exclusive over warps
    }
    __syncthreads();
    const uint64_t excl = s_carry + s_warp[warp] + incl - v;
    if (b < n_blocks) block_offsets[b] = excl;
    __syncthreads();
    if (t == kScanThreads - 1) s_carry = excl + v;
    __syncthreads();
  }
  // per-eye totals
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e0 += __shfl_xor_sync(0xffffffffu, e0, o);
    e1 += __shfl_xor_sync(0xffffffffu, e1, o);
  }
  if (lane == 0) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_eye[0]), (unsigned long long)e0);
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_eye[1]), (unsigned long long)e1);
  }
  __syncthreads();
  if (t == 0) {
    const uint64_t total = s_carry;
    counts[0] = (uint32_t)(total < capacity ? total : capacity);
    counts[1] = (uint32_t)s_eye[0];
    counts[2] = (uint32_t)s_eye[1];
    counts[3] = (uint32_t)total;
    if (total > capacity) atomicOr(status, kStatusCapacity);
  }
}

__global__ void __launch_bounds__(kPreThreads)
emit_keys_kernel(int n, int n_eyes, int tiles_x, int n_tiles, const float *__restrict__ rec,
                 const ushort4 *__restrict__ rect, const uint32_t *__restrict__ touched,
                 const unsigned long long *__restrict__ block_offsets, uint32_t capacity,
                 uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  __shared__ uint32_t s_warp[kPreThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int i = blockIdx.x * kPreThreads + t;
  const uint32_t mine = i < n ? touched[i] : 0u;
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  if (i >= n || mine == 0) return;
  uint64_t off = block_offsets[blockIdx.x] + before + incl - mine;
  for (int e = 0; e < n_eyes; ++e) {
    const ushort4 rc = rect[(size_t)e * n + i];
    if (rc.x >= rc.z) continue;
    const uint32_t depth_bits = __float_as_uint(rec[((size_t)e * n + i) * kRec + 9]);
    for (int ty = rc.y; ty < rc.w; ++ty) {
      for (int tx = rc.x; tx < rc.z; ++tx) {
        if (off < capacity) {
          const uint64_t tile = (uint64_t)e * n_tiles + (uint64_t)ty * tiles_x + tx;
          keys[off] = (tile << 32) | depth_bits;
          vals[off] = (uint32_t)i;
        }
        ++off;
      }
    }
  }
}

__global__ void tile_ranges_kernel(const uint64_t *__restrict__ keys,
                                   const uint32_t *__restrict__ d_count, uint2 *__restrict__ ranges,
                                   uint32_t n_ranges) {
  const uint32_t count = *d_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += gridDim.x * blockDim.x) {
    const uint32_t tile = (uint32_t)(keys[i] >> 32);
    if (tile >= n_ranges) continue;   // only after a failed sort (status already set)
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != tile) ranges[tile].x = i;
    if (i == count - 1 || (uint32_t)(keys[i + 1] >> 32) != tile) ranges[tile].y = i + 1;
  }
}

}  // namespace

cudaError_t launch_scan_blocks(const uint32_t *block_sums, int n_blocks,
                               unsigned long long *block_offsets, uint32_t *counts,
                               uint32_t capacity, uint32_t *status, cudaStream_t s) {
  scan_blocks_kernel<<<1, kScanThreads, 0, s>>>(block_sums, n_blocks, block_offsets, counts,
                                                capacity, status);
  return cudaGetLastError();
}

cudaError_t launch_emit_keys(int n, int n_eyes, int tiles_x, int n_tiles, const float *rec,
                             const ushort4 *rect, const uint32_t *touched,
                             const unsigned long long *block_offsets, uint32_t capacity,
                             uint64_t *keys, uint32_t *vals, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (n + kPreThreads - 1) / kPreThreads;
  emit_keys_kernel<<<blocks, kPreThreads, 0, s>>>(n, n_eyes, tiles_x, n_tiles, rec, rect,
                                                  touched, block_offsets, capacity, keys, vals);
  return cudaGetLastError();
}

cudaError_t launch_tile_ranges(const uint64_t *keys, const uint32_t *d_count, size_t capacity,
                               uint2 *ranges, int n_ranges, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_ranges, s);
  if (e != cudaSuccess) return e;
  if (capacity == 0) return cudaSuccess;
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (capacity + 255) / 256;
  const int blocks = (int)(want < (size_t)sms * 8 ? want : (size_t)sms * 8);
  tile_ranges_kernel<<<blocks, 256, 0, s>>>(keys, d_count, ranges, (uint32_t)n_ranges);
  return cudaGetLastError();
}

}  // namespace a3fr
