// binning.cu -- tile binning of the projected Gaussians (Sec. 2.3: "determining which
// ellipses intersect with a given pixel tile") and the per-tile ranges of the sorted
// instances ("subsets of Gaussian points on each tile", Sec. 3.5).
//
// The Gaussians of all eyes have already been sorted by depth (sort.cu).  emit walks them
// in that order and writes one (tile index, Gaussian index) instance per overlapped tile,
// so a STABLE sort of the instances by tile index alone gives every tile's Gaussians front
// to back with ties in index order -- exactly the order of the (tile << 32 | depth bits)
// keys sorted stably.
//
// emit (one kernel):
//   * instance offsets by a single-pass scan with decoupled look-back over dynamically
//     numbered blocks (64-bit flag|value words; bounded waits that set a status bit);
//   * warp-cooperative expansion: the 32 entries of a warp own a contiguous run of the
//     output, which the 32 lanes fill together (coalesced stores, no imbalance from large
//     Gaussians);
//   * the digit histograms of the tile sort are accumulated on the fly (shared-memory
//     counters aggregated per warp with __match_any_sync), so that sort needs no
//     histogram pass.
#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kEmitThreads = 256;
constexpr int kEmitWarps = kEmitThreads / 32;
constexpr unsigned long long kEFlagAgg = 1ull << 62;
constexpr unsigned long long kEFlagPrefix = 2ull << 62;
constexpr unsigned long long kEValMask = (1ull << 62) - 1ull;
constexpr uint32_t kSpinLimit = 1u << 20;

__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(EmitParams p, const uint32_t *__restrict__ entries, const uint32_t *__restrict__ touched,
            const ushort4 *__restrict__ rect, uint32_t *__restrict__ tile_keys,
            uint32_t *__restrict__ vals, unsigned long long *__restrict__ lookback,
            uint32_t *__restrict__ block_counter, uint32_t *__restrict__ counts,
            uint32_t *__restrict__ status, uint32_t *__restrict__ tile_hist) {
  __shared__ uint32_t s_blk;
  __shared__ uint32_t s_warp_total[kEmitWarps];
  __shared__ unsigned long long s_prefix;
  __shared__ uint32_t s_hist[kMaxSortPasses][256];
  __shared__ uint32_t s_excl[kEmitThreads];   // exclusive offset within the warp
  __shared__ uint32_t s_tile0[kEmitThreads];  // first tile index of the rectangle
  __shared__ uint32_t s_width[kEmitThreads];  // rectangle width in tiles
  __shared__ uint32_t s_gid[kEmitThreads];    // Gaussian index

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_blk = atomicAdd(block_counter, 1u);
  for (int i = t; i < p.tile_plan.passes * 256; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t blk = s_blk;
  const uint32_t j = blk * kEmitThreads + t;

  uint32_t cnt = 0, eye = 0;
  if (j < (uint32_t)p.n_entries) {
    const uint32_t v = entries[j];          // e * n + i
    cnt = touched[v];
    eye = v >= (uint32_t)p.n ? 1u : 0u;
    const uint32_t gi = v - eye * (uint32_t)p.n;
    if (cnt) {
      const ushort4 rc = rect[v];
      s_tile0[t] = eye * (uint32_t)p.n_tiles + (uint32_t)rc.y * (uint32_t)p.tiles_x + rc.x;
      s_width[t] = (uint32_t)(rc.z - rc.x);
      s_gid[t] = gi;
    }
  }
  // warp and block scans of the instance counts
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  s_excl[t] = incl - cnt;
  if (lane == 31) s_warp_total[warp] = incl;
  // per-eye totals
  uint32_t e0 = eye ? 0u : cnt, e1 = eye ? cnt : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e0 += __shfl_xor_sync(0xffffffffu, e0, o);
    e1 += __shfl_xor_sync(0xffffffffu, e1, o);
  }
  if (lane == 0) {
    if (e0) atomicAdd(&counts[1], e0);
    if (e1) atomicAdd(&counts[2], e1);
  }
  __syncthreads();

  // block prefix by decoupled look-back (thread 0)
  if (t == 0) {
    uint32_t block_total = 0;
    for (int w = 0; w < kEmitWarps; ++w) block_total += s_warp_total[w];
    unsigned long long *mine = lookback + blk;
    st_relaxed64(mine, (blk == 0 ? kEFlagPrefix : kEFlagAgg) | block_total);
    unsigned long long prefix = 0;
    if (blk > 0) {
      int q = (int)blk - 1;
      uint32_t spins = 0;
      while (true) {
        const unsigned long long w = ld_relaxed64(lookback + q);
        const unsigned long long flag = w & ~kEValMask;
        if (flag == 0ull) {
          if (++spins > kSpinLimit) {
            atomicOr(status, kStatusTimeout);
            break;
          }
          continue;
        }
        prefix += w & kEValMask;
        if (flag == kEFlagPrefix || q == 0) break;
        --q;
      }
      st_relaxed64(mine, kEFlagPrefix | ((prefix + block_total) & kEValMask));
    }
    s_prefix = prefix;
    if (blk == gridDim.x - 1) {
      const unsigned long long total = prefix + block_total;
      counts[0] = (uint32_t)(total < p.capacity ? total : p.capacity);
      counts[3] = (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull);
      if (total > p.capacity) atomicOr(status, kStatusCapacity);
    }
  }
  __syncthreads();

  // warp-cooperative expansion of the warp's contiguous run of instances
  uint32_t warp_before = 0;
  for (int w = 0; w < warp; ++w) warp_before += s_warp_total[w];
  const unsigned long long wbase = s_prefix + warp_before;
  const uint32_t W = s_warp_total[warp];
  const int wb = warp * 32;
  for (uint32_t q0 = 0; q0 < W; q0 += 32) {
    const uint32_t q = q0 + lane;
    const unsigned long long off = wbase + q;
    const bool valid = q < W && off < p.capacity;
    const unsigned m = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      int k = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (s_excl[wb + k + step] <= q) k += step;
      const uint32_t r = q - s_excl[wb + k];
      const uint32_t w = s_width[wb + k];
      const uint32_t dy = r / w, dx = r - dy * w;
      const uint32_t tile = s_tile0[wb + k] + dy * (uint32_t)p.tiles_x + dx;
      tile_keys[off] = tile;
      vals[off] = s_gid[wb + k];
      for (int ps = 0; ps < p.tile_plan.passes; ++ps) {
        const uint32_t d = (tile >> p.tile_plan.shift[ps]) & p.tile_plan.mask;
        const unsigned peers = __match_any_sync(m, d);
        if (lane == 31 - __clz(peers)) atomicAdd(&s_hist[ps][d], (uint32_t)__popc(peers));
      }
    }
  }
  __syncthreads();
  for (int i = t; i < p.tile_plan.passes * 256; i += kEmitThreads) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(tile_hist + i, v);
  }
}

__global__ void tile_ranges_kernel(const uint32_t *__restrict__ tile_keys,
                                   const uint32_t *__restrict__ d_count, uint2 *__restrict__ ranges,
                                   uint32_t n_ranges) {
  const uint32_t count = *d_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += gridDim.x * blockDim.x) {
    const uint32_t tile = tile_keys[i];
    if (tile >= n_ranges) continue;   // only after a failed sort (status already set)
    if (i == 0 || tile_keys[i - 1] != tile) ranges[tile].x = i;
    if (i == count - 1 || tile_keys[i + 1] != tile) ranges[tile].y = i + 1;
  }
}

__global__ void materialize_keys_kernel(const uint32_t *__restrict__ tile_keys,
                                        const uint32_t *__restrict__ vals,
                                        const float *__restrict__ rec, int n, int n_tiles,
                                        uint32_t count, uint64_t *__restrict__ keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += gridDim.x * blockDim.x) {
    const uint32_t tile = tile_keys[i];
    const uint32_t eye = tile / (uint32_t)n_tiles;
    const uint32_t g = min(vals[i], (uint32_t)(n - 1));
    const float depth = rec[((size_t)eye * n + g) * kRec + 9];
    keys[i] = ((uint64_t)tile << 32) | __float_as_uint(depth);
  }
}

int grid_for(size_t work, int per_block) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (work + per_block - 1) / per_block;
  const size_t cap = (size_t)sms * 8;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

size_t emit_lookback_bytes(int n_entries) {
  return sizeof(unsigned long long) * (size_t)((n_entries + kEmitThreads - 1) / kEmitThreads + 1);
}

cudaError_t launch_emit(const EmitParams &p, const uint32_t *entries, const uint32_t *touched,
                        const ushort4 *rect, uint32_t *tile_keys, uint32_t *vals,
                        unsigned long long *lookback, uint32_t *block_counter, uint32_t *counts,
                        uint32_t *status, uint32_t *tile_hist, cudaStream_t s) {
  if (p.n_entries <= 0) return cudaSuccess;
  const int blocks = (p.n_entries + kEmitThreads - 1) / kEmitThreads;
  emit_kernel<<<blocks, kEmitThreads, 0, s>>>(p, entries, touched, rect, tile_keys, vals,
                                              lookback, block_counter, counts, status,
                                              tile_hist);
  return cudaGetLastError();
}

cudaError_t launch_tile_ranges(const uint32_t *tile_keys, const uint32_t *d_count,
                               size_t capacity, uint2 *ranges, int n_ranges, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_ranges, s);
  if (e != cudaSuccess) return e;
  if (capacity == 0) return cudaSuccess;
  tile_ranges_kernel<<<grid_for(capacity, 256), 256, 0, s>>>(tile_keys, d_count, ranges,
                                                              (uint32_t)n_ranges);
  return cudaGetLastError();
}

cudaError_t launch_materialize_keys(const uint32_t *tile_keys, const uint32_t *vals,
                                    const float *rec, int n, int n_tiles, uint32_t count,
                                    uint64_t *keys, cudaStream_t s) {
  if (count == 0 || n <= 0) return cudaSuccess;
  materialize_keys_kernel<<<grid_for(count, 256), 256, 0, s>>>(tile_keys, vals, rec, n, n_tiles,
                                                               count, keys);
  return cudaGetLastError();
}

}  // namespace a3fr
