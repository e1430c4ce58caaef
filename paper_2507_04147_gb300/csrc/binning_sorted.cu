// binning_sorted.cu -- the sort-based tile binning, for renders with many tiles (Sec. 2.3
// "determining which ellipses intersect with a given pixel tile"; Sec. 3.5 tile subsets).
//
// binning.cu places every instance directly, but its per-warp cursor table holds one word
// per tile; beyond a few thousand tiles too few warps fit on an SM.  This path keeps no
// per-tile state in shared memory: emit walks the depth-ordered entries and writes one
// (tile index, Gaussian index) instance per overlapped tile, so a STABLE sort of the
// instances by tile index alone (onesweep, sort.cu) gives every tile's Gaussians front to
// back with ties in index order -- the same lists as binning.cu.
//
// tile_count + tile_scan give every tile's instance count without enumerating instances:
// each tile rectangle adds +1/-1/-1/+1 at its corners in a 2-D difference grid (per CTA in
// shared memory, partial grids summed without atomics), whose 2-D prefix sum is the count.
// The exclusive scan of the counts over tiles is exactly where the stable sort by tile puts
// each tile's run, i.e. the tile ranges; the digit histograms of that sort follow from the
// same prefix sums.
//
// emit: the instance offset of every depth-ordered entry (a chained scan over blocks of 1024
// entries) and the entry holding the first slot of each partition of the tile sort.  The
// instances themselves are not written: the first pass of the tile sort generates them from
// these offsets (sort.cu), so a Gaussian covering hundreds of tiles costs one slot per thread
// like any other.
#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kEmitThreads = 256;
constexpr int kEmitWarps = kEmitThreads / 32;
constexpr int kEmitPer = 4;                                // entries per thread
constexpr int kEmitEntries = kEmitThreads * kEmitPer;      // entries per block
// Instance offsets of the depth-ordered entries, one block of kEmitEntries entries per CTA:
// the CTAs take consecutive blocks from a ticket counter and chain their instance sums by
// decoupled look-back, then every entry stores its global offset off[j], every entry holding
// the first slot of a partition of kGenPart slots (the generated sort pass's unit) stores its
// index in pstart[k], and the last block stores the total after the look-back words.
__global__ void __launch_bounds__(kEmitThreads)
emit_scan_kernel(EmitParams p, Entries ents, const uint32_t *__restrict__ touched,
                 unsigned long long *__restrict__ lookback, uint32_t *__restrict__ off,
                 uint32_t *__restrict__ pstart, int n_parts, uint32_t *__restrict__ ticket,
                 uint32_t *__restrict__ status) {
  pdl_begin();
  const uint32_t *__restrict__ entries = ents.get();
  __shared__ uint32_t s_wsum[kEmitWarps];
  __shared__ uint32_t s_b;
  __shared__ unsigned long long s_before;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_b = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t b = s_b;
  const uint32_t j0 = b * kEmitEntries + t * kEmitPer;
  uint32_t c[kEmitPer], mine = 0;
  if (j0 + kEmitPer <= (uint32_t)p.n_entries && (reinterpret_cast<uintptr_t>(entries) & 15u) == 0u) {
    const uint4 v = *reinterpret_cast<const uint4 *>(entries + j0);
    c[0] = touched[v.x];
    c[1] = touched[v.y];
    c[2] = touched[v.z];
    c[3] = touched[v.w];
  } else {
#pragma unroll
    for (int k = 0; k < kEmitPer; ++k) c[k] = j0 + k < (uint32_t)p.n_entries ? touched[entries[j0 + k]] : 0u;
  }
#pragma unroll
  for (int k = 0; k < kEmitPer; ++k) mine += c[k];
  // block-exclusive offsets of this thread's entries (a block holds < 2^32 instances)
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  uint32_t excl = incl - mine, agg = 0;
  for (int w = 0; w < kEmitWarps; ++w) {
    excl += w < warp ? s_wsum[w] : 0u;
    agg += s_wsum[w];
  }
  if (warp == 0) {
    unsigned long long before = 0;
    if (b == 0) {
      if (lane == 0) st_relaxed64(lookback, kPrefixFlag | agg);
    } else {
      if (lane == 0) st_relaxed64(lookback + b, kAggFlag | agg);
      before = block_lookback(lookback, (int)b, status);
      if (lane == 0) st_relaxed64(lookback + b, kPrefixFlag | ((before + agg) & kVal62));
    }
    if (lane == 0) {
      s_before = before;
      if (b == gridDim.x - 1) lookback[gridDim.x] = before + agg;   // the total
    }
  }
  __syncthreads();
  unsigned long long g = s_before + excl;
  uint32_t o4[kEmitPer];
#pragma unroll
  for (int k = 0; k < kEmitPer; ++k) {
    o4[k] = (uint32_t)(g < 0xffffffffull ? g : 0xffffffffull);
    // the partitions whose first slot lies in this entry's run [g, g + c)
    for (unsigned long long q = (g + kGenPart - 1) / kGenPart; q < (unsigned long long)n_parts && q * kGenPart < g + c[k]; ++q)
      pstart[q] = j0 + k;
    g += c[k];
  }
  if (j0 + kEmitPer <= (uint32_t)p.n_entries && (reinterpret_cast<uintptr_t>(off) & 15u) == 0u) {
    *reinterpret_cast<uint4 *>(off + j0) = make_uint4(o4[0], o4[1], o4[2], o4[3]);
  } else {
#pragma unroll
    for (int k = 0; k < kEmitPer; ++k)
      if (j0 + k < (uint32_t)p.n_entries) off[j0 + k] = o4[k];
  }
}

constexpr int kCountThreads = 512;

// Per CTA: the difference grid of a contiguous slice of the (eye, Gaussian) rectangles in
// shared memory, written to partials[blockIdx.x][cells].
__global__ void __launch_bounds__(kCountThreads)
tile_count_kernel(TileScanParams p, const ushort4 *__restrict__ rect,
                  uint32_t *__restrict__ partials) {
  pdl_begin();
  extern __shared__ uint32_t s_grid[];
  const int gw = p.tiles_x + 1, gh = p.tiles_y + 1;
  const int cells = p.n_eyes * gw * gh;
  for (int i = threadIdx.x; i < cells; i += kCountThreads) s_grid[i] = 0;
  __syncthreads();
  const int entries = p.n_eyes * p.n;
  const int per = (entries + gridDim.x - 1) / gridDim.x;
  const int e0 = blockIdx.x * per, e1 = min(entries, e0 + per);
  for (int v = e0 + threadIdx.x; v < e1; v += kCountThreads) {
    const ushort4 rc = rect[v];
    if (rc.x >= rc.z) continue;
    const int eye = v >= p.n ? 1 : 0;
    uint32_t *g = s_grid + eye * gw * gh;
    atomicAdd(g + rc.y * gw + rc.x, 1u);
    atomicAdd(g + rc.y * gw + rc.z, 0xffffffffu);
    atomicAdd(g + rc.w * gw + rc.x, 0xffffffffu);
    atomicAdd(g + rc.w * gw + rc.z, 1u);
  }
  __syncthreads();
  uint32_t *out = partials + (size_t)blockIdx.x * cells;
  for (int i = threadIdx.x; i < cells; i += kCountThreads) out[i] = s_grid[i];
}

// Sum of the per-CTA difference grids: blockIdx.y takes a group of kReduceParts partial
// grids, each thread one cell; the group sums are added into the zeroed grid (integer adds,
// so the result does not depend on their order).
constexpr int kReduceParts = 19;

__global__ void __launch_bounds__(256)
tile_reduce_kernel(const uint32_t *__restrict__ partials, int parts, int cells,
                   uint32_t *__restrict__ grid) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cells) return;
  const int b0 = blockIdx.y * kReduceParts, b1 = min(parts, b0 + kReduceParts);
  uint32_t acc = 0;
#pragma unroll 4
  for (int b = b0; b < b1; ++b) acc += partials[(size_t)b * cells + i];
  if (acc) atomicAdd(grid + i, acc);
}

// Inclusive scan of one value per lane across the warp.
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// One CTA: 2-D prefix sums of the summed difference grids in shared memory (a warp per row,
// then a warp per column, 32 cells per step), then the exclusive scan of the counts over
// tiles (eye-major, row-major) -> ranges: each thread owns a contiguous run of tiles, so
// one block-wide scan of the run totals suffices.  The digit histograms of the tile sort
// are accumulated from the same counts (one shared atomic per run of equal digits), and
// the per-eye totals are read from the scanned ranges.
__global__ void __launch_bounds__(1024)
tile_scan_kernel(TileScanParams p, const uint32_t *__restrict__ diff, uint2 *__restrict__ ranges,
                 uint32_t *__restrict__ tile_hist, uint32_t *__restrict__ counts,
                 uint32_t *__restrict__ status) {
  pdl_begin();
  extern __shared__ uint32_t s_grid[];
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_hist[kMaxSortPasses][256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, n_warps = blockDim.x >> 5;
  const int gw = p.tiles_x + 1, gh = p.tiles_y + 1;
  const int cells = p.n_eyes * gw * gh;
  for (int i = t; i < kMaxSortPasses * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  // bulk copy, four independent loads in flight per thread
  for (int i0 = t; i0 < cells; i0 += 4 * blockDim.x) {
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k * blockDim.x;
      v[k] = i < cells ? diff[i] : 0u;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k * blockDim.x;
      if (i < cells) s_grid[i] = v[k];
    }
  }
  __syncthreads();
  // rows
  for (int r = warp; r < p.n_eyes * gh; r += n_warps) {
    uint32_t *row = s_grid + r * gw;
    uint32_t carry = 0;
    for (int x0 = 0; x0 < gw; x0 += 32) {
      const int x = x0 + lane;
      uint32_t v = x < gw ? row[x] : 0u;
      v = warp_incl_scan(v, lane) + carry;
      if (x < gw) row[x] = v;
      carry = __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  // columns
  for (int c = warp; c < p.n_eyes * gw; c += n_warps) {
    const int e = c / gw, x = c - e * gw;
    uint32_t *col = s_grid + e * gw * gh + x;
    uint32_t carry = 0;
    for (int y0 = 0; y0 < gh; y0 += 32) {
      const int y = y0 + lane;
      uint32_t v = y < gh ? col[y * gw] : 0u;
      v = warp_incl_scan(v, lane) + carry;
      if (y < gh) col[y * gw] = v;
      carry = __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  // this thread's run of tiles [r0, r1) and its total
  const int n_ranges = p.n_eyes * p.n_tiles;
  const int per = (n_ranges + (int)blockDim.x - 1) / (int)blockDim.x;
  const int r0 = min(n_ranges, t * per), r1 = min(n_ranges, r0 + per);
  unsigned long long sum = 0;
  if (r0 < r1) {
    int eye = r0 / p.n_tiles, tile = r0 - eye * p.n_tiles;
    int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
    for (int r = r0; r < r1; ++r) {
      sum += s_grid[eye * gw * gh + ty * gw + tx];
      if (++tx == p.tiles_x) {
        tx = 0;
        if (++ty == p.tiles_y) { ty = 0; ++eye; }
      }
    }
  }
  // block-wide exclusive scan of the run totals
  const unsigned long long incl = warp_incl_scan(sum, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long w = lane < n_warps ? s_warp[lane] : 0ull;
    s_warp[lane] = warp_incl_scan(w, lane) - w;
  }
  __syncthreads();
  unsigned long long excl = s_warp[warp] + incl - sum;
  if (r0 < r1) {
    int eye = r0 / p.n_tiles, tile = r0 - eye * p.n_tiles;
    int ty = tile / p.tiles_x, tx = tile - ty * p.tiles_x;
    uint32_t run_d[kMaxSortPasses], run_v[kMaxSortPasses];
#pragma unroll
    for (int ps = 0; ps < kMaxSortPasses; ++ps) {
      run_d[ps] = 0xffffffffu;
      run_v[ps] = 0;
    }
    const unsigned long long lim = 0xffffffffull;
    for (int r = r0; r < r1; ++r) {
      const uint32_t cnt = s_grid[eye * gw * gh + ty * gw + tx];
      // unclamped: the composite clamps every range to the instances the sort kept
      ranges[r] = make_uint2((uint32_t)(excl < lim ? excl : lim),
                             (uint32_t)(excl + cnt < lim ? excl + cnt : lim));
      excl += cnt;
#pragma unroll
      for (int ps = 0; ps < kMaxSortPasses; ++ps) {
        if (ps < p.tile_plan.passes) {
          const uint32_t d = ((uint32_t)r >> p.tile_plan.shift[ps]) & p.tile_plan.mask;
          if (d != run_d[ps]) {
            if (run_v[ps]) atomicAdd(&s_hist[ps][run_d[ps]], run_v[ps]);
            run_d[ps] = d;
            run_v[ps] = 0;
          }
          run_v[ps] += cnt;
        }
      }
      if (++tx == p.tiles_x) {
        tx = 0;
        if (++ty == p.tiles_y) { ty = 0; ++eye; }
      }
    }
#pragma unroll
    for (int ps = 0; ps < kMaxSortPasses; ++ps)
      if (ps < p.tile_plan.passes && run_v[ps]) atomicAdd(&s_hist[ps][run_d[ps]], run_v[ps]);
  }
  __syncthreads();
  for (int i = t; i < p.tile_plan.passes * 256; i += blockDim.x) tile_hist[i] = (&s_hist[0][0])[i];
  if (t == blockDim.x - 1) {
    // the last thread's running offset is the total (threads past the tiles carry it too)
    const unsigned long long total = excl;
    const uint32_t eye0 = p.n_eyes > 1 ? ranges[p.n_tiles].x : (uint32_t)total;
    counts[0] = (uint32_t)(total < p.capacity ? total : p.capacity);
    counts[1] = eye0;
    counts[2] = (uint32_t)total - eye0;
    counts[3] = (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull);
    if (total > p.capacity) atomicOr(status, kStatusCapacity);
  }
}

}  // namespace

size_t emit_lookback_bytes(int n_entries) {
  return sizeof(unsigned long long) * (size_t)((n_entries + kEmitEntries - 1) / kEmitEntries + 1);
}

cudaError_t launch_emit_offsets(const EmitParams &p, Entries entries, const uint32_t *touched,
                                unsigned long long *lookback, uint32_t *off, uint32_t *pstart, int n_parts,
                                uint32_t *ticket, uint32_t *status, cudaStream_t s) {
  if (p.n_entries <= 0) return cudaSuccess;
  const int blocks = (p.n_entries + kEmitEntries - 1) / kEmitEntries;
  {
    const cudaError_t e_ = launch_pdl(emit_scan_kernel, blocks, kEmitThreads, 0, s, p, entries, touched,
                                      lookback, off, pstart, n_parts, ticket, status);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

size_t tile_grid_cells(int n_eyes, int tiles_x, int tiles_y) {
  return (size_t)n_eyes * (tiles_x + 1) * (tiles_y + 1);
}

size_t tile_scan_smem_bytes(int n_eyes, int tiles_x, int tiles_y) {
  return sizeof(uint32_t) * tile_grid_cells(n_eyes, tiles_x, tiles_y);
}

int tile_count_blocks() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

cudaError_t launch_tile_count(const TileScanParams &p, const ushort4 *rect, uint32_t *partials,
                              uint32_t *grid, cudaStream_t s) {
  const size_t cells = tile_grid_cells(p.n_eyes, p.tiles_x, p.tiles_y);
  const size_t smem = sizeof(uint32_t) * cells;
  cudaError_t e = cudaFuncSetAttribute(tile_count_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int parts = tile_count_blocks();
  {
    const cudaError_t e_ = launch_pdl(tile_count_kernel, parts, kCountThreads, smem, s, p, rect, partials);
    if (e_ != cudaSuccess) return e_;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(grid, 0, sizeof(uint32_t) * cells, s);
  if (e != cudaSuccess) return e;
  const dim3 rb((unsigned)((cells + 255) / 256), (unsigned)((parts + kReduceParts - 1) / kReduceParts));
  {
    const cudaError_t e_ = launch_pdl(tile_reduce_kernel, rb, 256, 0, s, partials, parts, (int)cells, grid);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_tile_scan(const TileScanParams &p, const uint32_t *grid, uint2 *ranges,
                             uint32_t *tile_hist, uint32_t *counts, uint32_t *status,
                             cudaStream_t s) {
  const size_t smem = tile_scan_smem_bytes(p.n_eyes, p.tiles_x, p.tiles_y);
  cudaError_t e = cudaFuncSetAttribute(tile_scan_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  {
    const cudaError_t e_ = launch_pdl(tile_scan_kernel, 1, 1024, smem, s, p, grid, ranges, tile_hist, counts,
                                      status);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

}  // namespace a3fr
