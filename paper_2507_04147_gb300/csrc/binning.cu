// binning.cu -- tile binning of the projected Gaussians (Sec. 2.3: "determining which
// ellipses intersect with a given pixel tile") and the per-tile ranges of the sorted
// instances ("subsets of Gaussian points on each tile", Sec. 3.5).
//
// The Gaussians of all eyes have already been sorted by depth (sort.cu).  A tile's list is
// the depth-ordered entries whose tile rectangle covers the tile, in that order -- exactly
// the order of the (tile << 32 | depth bits) keys sorted stably.  Binning writes every
// (tile, Gaussian) instance straight to its final slot; there is no sort by tile:
//
//  bin_plan     The entries are cut into C chunks of consecutive entries holding about
//               equal numbers of instances (a look-back prefix of the entries' counts).
//  bin_count    Per chunk
//               (one CTA), shared-memory atomics over the tile rectangles give the
//               chunk's instance count of every tile, h[c][r].
//  bin_offsets  With T[r] = sum over chunks of h[c][r], tile r's run starts at R[r] = sum
//               of T over the tiles before it (these are the tile ranges), and chunk c's
//               instances of tile r at R[r] + sum over the earlier chunks of h[c'][r]; the
//               start overwrites h.  One CTA per 32 tiles; the CTAs chain their sums by a
//               decoupled look-back (bounded waits, like the sort's).
//  bin_emit     One warp per (chunk, band of tile rows) walks the chunk's instances in its
//               band in entry order, 32 at a time (lane = instance).  A lane's slot is the tile's cursor plus the number
//               of lower lanes with the same tile; the highest of them advances the cursor.
//               Every tile's instances land in entry (= depth) order, the same on every run.
//
// Instances whose slot is at or past the capacity are dropped (the render raises the
// capacity status and the composite clamps ranges to the instances kept).
#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kCountThreads = 256;
constexpr int kPlanThreads = 256;
constexpr int kPlanPer = 8;                  // entries per thread of bin_plan
constexpr int kPlanEntries = kPlanThreads * kPlanPer;
constexpr int kOffsetThreads = 1024;
constexpr int kMaxChunks = kBinMaxChunks;
constexpr int kSegUnroll = 16;              // bin_offsets loads in flight per thread
constexpr int kMap = 256;                   // instances a bin_emit warp expands per window
constexpr int kBandTiles = 3200;            // tiles per bin_emit band (12.8 KB of cursors)
constexpr int kMapPad = kMap + kMap / 32;   // one pad word per 32 (fewer bank conflicts)
constexpr long long kMaxChunkCells = 24ll << 20;   // bound on C * tiles (u32 cells of h)

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

// Per chunk: the instance count of every tile by shared-memory atomics over the chunk's
// tile rectangles (each thread walks the rectangles of its entries), written as h[c][r].
__global__ void __launch_bounds__(kCountThreads)
bin_count_kernel(BinParams p, Entries ents, const ushort4 *__restrict__ rect,
                 const uint32_t *__restrict__ bounds, uint32_t *__restrict__ h) {
  pdl_begin();
  const uint32_t *__restrict__ entries = ents.get();
  extern __shared__ uint32_t s_hist[];
  const int t = threadIdx.x;
  const int n_ranges = p.n_eyes * p.n_tiles;
  for (int i = t; i < n_ranges; i += kCountThreads) s_hist[i] = 0u;
  __syncthreads();
  const int j0 = (int)bounds[blockIdx.x], j1 = (int)bounds[blockIdx.x + 1];
  for (int j = j0 + t; j < j1; j += kCountThreads) {
    const uint32_t v = entries[j];
    const ushort4 rc = rect[v];
    if (rc.x >= rc.z) continue;
    const int row0 = (v >= (uint32_t)p.n ? p.tiles_y : 0) + (int)rc.y;
    const int rows = (int)rc.w - (int)rc.y;
    for (int y = 0; y < rows; ++y) {
      uint32_t *hr = s_hist + (row0 + y) * p.tiles_x;
      for (int x = rc.x; x < (int)rc.z; ++x) atomicAdd(hr + x, 1u);
    }
  }
  __syncthreads();
  uint32_t *out = h + (size_t)blockIdx.x * p.row;
  for (int r = t; r < n_ranges; r += kCountThreads) out[r] = s_hist[r];
}

// Chunk plan: bounds[c] = the first entry j whose preceding instances P_j (prefix of the
// entries' tile counts in depth order) reach c T / C, T the render's instance total, so
// every chunk holds about T / C instances (near Gaussians, first in depth order, cover
// many tiles: equal entry counts would load the first chunks with twice the mean).  An
// entry j writes bounds[c] = j + 1 for the c with floor(P_j C / T) < c <= floor(P_{j+1} C / T).
// The blocks chain their sums by the same look-back as bin_offsets.
__global__ void __launch_bounds__(kPlanThreads)
bin_plan_kernel(BinParams p, Entries ents, const uint32_t *__restrict__ touched,
                const unsigned long long *__restrict__ inst_total,
                unsigned long long *__restrict__ lookback, uint32_t *__restrict__ bounds,
                uint32_t *__restrict__ status) {
  pdl_begin();
  const uint32_t *__restrict__ entries = ents.get();
  __shared__ unsigned long long s_warp[kPlanThreads / 32];
  __shared__ unsigned long long s_before;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned long long T = *inst_total;
  const unsigned long long C = (unsigned long long)p.n_chunks;
  if (blockIdx.x == 0 && t == 0) {
    bounds[0] = 0u;
    bounds[p.n_chunks] = (uint32_t)p.n_entries;
  }
  if (T == 0ull) {
    // no instances: any split will do
    for (int c = 1 + blockIdx.x * kPlanThreads + t; c < p.n_chunks; c += gridDim.x * kPlanThreads)
      bounds[c] = (uint32_t)((unsigned long long)p.n_entries * (unsigned long long)c / C);
    return;
  }
  const int jb = blockIdx.x * kPlanEntries + t * kPlanPer;
  uint32_t cnt[kPlanPer];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < kPlanPer; ++k) {
    const int j = jb + k;
    cnt[k] = j < p.n_entries ? touched[entries[j]] : 0u;
    sum += cnt[k];
  }
  const unsigned long long incl = warp_incl_scan<unsigned long long>(sum, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  unsigned long long wbefore = 0, agg = 0;
  for (int w = 0; w < kPlanThreads / 32; ++w) {
    if (w < warp) wbefore += s_warp[w];
    agg += s_warp[w];
  }
  if (warp == 0) {
    unsigned long long before = 0;
    if (blockIdx.x == 0) {
      if (lane == 0) st_relaxed64(lookback, kPrefixFlag | (agg & kVal62));
    } else {
      if (lane == 0) st_relaxed64(lookback + blockIdx.x, kAggFlag | (agg & kVal62));
      before = block_lookback(lookback, blockIdx.x, status);
      if (lane == 0) st_relaxed64(lookback + blockIdx.x, kPrefixFlag | ((before + agg) & kVal62));
    }
    if (lane == 0) s_before = before;
  }
  __syncthreads();
  unsigned long long P = s_before + wbefore + incl - sum;
  unsigned long long c_lo = P * C / T;
#pragma unroll
  for (int k = 0; k < kPlanPer; ++k) {
    const unsigned long long P1 = P + cnt[k];
    const unsigned long long c_hi = P1 * C / T;
    for (unsigned long long c = c_lo + 1; c <= c_hi && c < C; ++c) bounds[c] = (uint32_t)(jb + k + 1);
    P = P1;
    c_lo = c_hi;
  }
}

// Block b owns tiles [32 b, 32 b + 32) (lane = tile) and warp w the chunk segment
// [C w / 32, C (w + 1) / 32), staged in shared memory (s_seg[k][thread]).  Starts are stored clamped to 2^31 - 1,
// so the cursors of bin_emit cannot wrap; bin_emit drops every slot at or past the
// capacity.  counts[1] (the first eye's instances) comes from the block holding the first
// tile of the second eye, counts[0] and [3] from the last block.
__global__ void __launch_bounds__(kOffsetThreads)
bin_offsets_kernel(BinParams p, uint32_t *__restrict__ h, unsigned long long *__restrict__ lookback,
                   uint2 *__restrict__ ranges, uint32_t *__restrict__ counts,
                   uint32_t *__restrict__ status) {
  pdl_begin();
  extern __shared__ uint32_t s_seg[];
  __shared__ uint32_t s_part[32][33];
  __shared__ unsigned long long s_before;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n_ranges = p.n_eyes * p.n_tiles;
  const int r = blockIdx.x * 32 + lane;
  const int c0 = (int)((long long)p.n_chunks * warp / 32);
  const int c1 = (int)((long long)p.n_chunks * (warp + 1) / 32);
  const int n_seg = r < n_ranges ? c1 - c0 : 0;
  uint32_t *col = h + (size_t)c0 * p.row + (r < n_ranges ? r : 0);
  uint32_t part = 0;
  for (int k0 = 0; k0 < n_seg; k0 += kSegUnroll) {
    uint32_t v[kSegUnroll];
#pragma unroll
    for (int u = 0; u < kSegUnroll; ++u)
      v[u] = k0 + u < n_seg ? col[(size_t)(k0 + u) * p.row] : 0u;
#pragma unroll
    for (int u = 0; u < kSegUnroll; ++u) {
      if (k0 + u < n_seg) s_seg[(k0 + u) * kOffsetThreads + t] = v[u];
      part += v[u];
    }
  }
  s_part[warp][lane] = part;
  __syncthreads();
  unsigned long long tot = 0, earlier = 0;
  for (int w = 0; w < 32; ++w) {
    const uint32_t v = s_part[w][lane];
    tot += v;
    if (w < warp) earlier += v;
  }
  unsigned long long agg = tot;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) agg += __shfl_xor_sync(0xffffffffu, agg, o);
  if (warp == 0) {
    unsigned long long before = 0;
    if (blockIdx.x == 0) {
      if (lane == 0) st_relaxed64(lookback, kPrefixFlag | (agg & kVal62));
    } else {
      if (lane == 0) st_relaxed64(lookback + blockIdx.x, kAggFlag | (agg & kVal62));
      before = block_lookback(lookback, blockIdx.x, status);
      if (lane == 0) st_relaxed64(lookback + blockIdx.x, kPrefixFlag | ((before + agg) & kVal62));
    }
    if (lane == 0) s_before = before;
  }
  __syncthreads();
  const unsigned long long before = s_before;
  const unsigned long long start = before + warp_incl_scan<unsigned long long>(tot, lane) - tot;
  unsigned long long run = start + earlier;
  const unsigned long long lim = 0xffffffffull, clamp = 0x7fffffffull;
  for (int k = 0; k < n_seg; ++k) {
    *col = (uint32_t)(run < clamp ? run : clamp);
    run += s_seg[k * kOffsetThreads + t];
    col += p.row;
  }
  if (warp == 0 && r < n_ranges) {
    // unclamped: the composite clamps every range to the instances kept
    ranges[r] = make_uint2((uint32_t)(start < lim ? start : lim),
                           (uint32_t)(start + tot < lim ? start + tot : lim));
    if (p.n_eyes > 1 && r == p.n_tiles) counts[1] = (uint32_t)(start < lim ? start : lim);
  }
  if (warp == 0 && lane == 0 && blockIdx.x == gridDim.x - 1) {
    const unsigned long long total = before + agg;
    counts[0] = (uint32_t)(total < p.capacity ? total : p.capacity);
    if (p.n_eyes < 2) counts[1] = (uint32_t)(total < lim ? total : lim);
    counts[3] = (uint32_t)(total < lim ? total : lim);
    if (total > p.capacity) atomicOr(status, kStatusCapacity);
  }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// One warp (CTA) per (chunk, band): blockIdx.x = chunk * n_bands + band, the band being the
// tile rows [R0, R1) (row index eye * tiles_y + y), i.e. the contiguous tiles [R0 tiles_x,
// R1 tiles_x).  The warp walks the chunk's entries 32 at a time (lane = entry), scans their
// instance counts inside the band and expands those instances into its map (band tile,
// Gaussian) in windows of kMap, then takes the map 32 instances at a time (lane = instance:
// full warps whatever the rectangle sizes).  A lane's rank among the step's instances of its
// tile is the number of lower lanes with the same tile (__match_any_sync); the highest of
// them advances the tile's cursor.  Shared memory: the band's cursors (from the chunk's row
// of h, copied in by cp.async) and the map.  Entry values are loaded two rounds ahead,
// rectangles one round ahead.
__global__ void __launch_bounds__(32)
bin_emit_kernel(BinParams p, Entries ents, const ushort4 *__restrict__ rect,
                const uint32_t *__restrict__ bounds, const uint32_t *__restrict__ h,
                uint32_t *__restrict__ vals) {
  pdl_begin();
  const uint32_t *__restrict__ entries = ents.get();
  extern __shared__ __align__(16) uint32_t s_dyn[];
  __shared__ uint32_t s_map_tile[kMapPad];
  __shared__ uint32_t s_map_gid[kMapPad];
  const int lane = threadIdx.x;
  const int chunk = blockIdx.x / p.n_bands, band = blockIdx.x - chunk * p.n_bands;
  const int R0 = band * p.band_rows, R1 = min(p.n_eyes * p.tiles_y, R0 + p.band_rows);
  // the band's tiles [R0 tiles_x, R1 tiles_x) of the chunk's row of h, copied from the
  // 16-byte boundary at or below its start; s_cur[t] is the cursor of band tile t
  const int t0 = R0 * p.tiles_x, a0 = t0 & ~3, a1 = min(p.row, (R1 * p.tiles_x + 3) & ~3);
  uint32_t *s_cur = s_dyn + (t0 - a0);
  {
    const uint32_t *hb = h + (size_t)chunk * p.row;
    for (int i = a0 + lane * 4; i < a1; i += 128) cp_async16(s_dyn + (i - a0), hb + i);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const unsigned below = (1u << lane) - 1u;
  const int j0 = (int)bounds[chunk], j1 = (int)bounds[chunk + 1];
  const ushort4 none = make_ushort4(0, 0, 0, 0);
  uint32_t v_cur = j0 + lane < j1 ? entries[j0 + lane] : 0u;
  uint32_t v_next = j0 + 32 + lane < j1 ? entries[j0 + 32 + lane] : 0u;
  ushort4 r_cur = j0 + lane < j1 ? rect[v_cur] : none;
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();
  for (int b = j0; b < j1; b += 32) {
    const uint32_t v = v_cur;
    const ushort4 rc = r_cur;
    {
      const int jn = b + 32 + lane, jnn = jn + 32;
      r_cur = jn < j1 ? rect[v_next] : none;
      v_cur = v_next;
      v_next = jnn < j1 ? entries[jnn] : 0u;
    }
    const uint32_t w = rc.z > rc.x ? (uint32_t)(rc.z - rc.x) : 0u;
    const int eye = v >= (uint32_t)p.n ? 1 : 0;
    const uint32_t gid = v - (uint32_t)eye * (uint32_t)p.n;
    // the rectangle's rows inside the band
    const int row0 = max(R0, eye * p.tiles_y + (int)rc.y);
    const int row1 = min(R1, eye * p.tiles_y + (int)rc.w);
    const uint32_t cnt = (b + lane < j1 && row1 > row0) ? w * (uint32_t)(row1 - row0) : 0u;
    const uint32_t incl = warp_incl_scan(cnt, lane);
    const uint32_t first = incl - cnt;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t base = 0; base < total; base += kMap) {
      const uint32_t wend = min(total, base + kMap);
      // this lane's instances in [base, wend) into the map
      const uint32_t lo = max(first, base), hi = min(incl, wend);
      if (lo < hi) {
        const uint32_t off = lo - first;
        const uint32_t dy = off ? div_small(off, w) : 0u;
        int x = (int)rc.x + (int)(off - dy * w);
        int tile = (row0 - R0 + (int)dy) * p.tiles_x + x;   // band tile index
        for (uint32_t j = lo; j < hi; ++j) {
          const uint32_t mj = j - base;
          s_map_tile[mj + (mj >> 5)] = (uint32_t)tile;
          s_map_gid[mj + (mj >> 5)] = gid;
          ++tile;
          if (++x == (int)rc.z) {
            x = rc.x;
            tile += p.tiles_x - (int)w;
          }
        }
      }
      __syncwarp();
      for (uint32_t q0 = base; q0 < wend; q0 += 32) {
        const uint32_t mj = q0 - base + lane;
        const bool valid = q0 + lane < wend;
        const uint32_t tile = valid ? s_map_tile[mj + (mj >> 5)] : (0x80000000u | lane);
        const unsigned m = __match_any_sync(0xffffffffu, tile);
        uint32_t cur = 0u;
        if (valid) {
          cur = s_cur[tile];
          const uint32_t pos = cur + (uint32_t)__popc(m & below);
          if (pos < p.capacity) vals[pos] = s_map_gid[mj + (mj >> 5)];
        }
        __syncwarp();
        if (valid && (m >> lane) == 1u) s_cur[tile] = cur + (uint32_t)__popc(m);
        __syncwarp();
      }
    }
  }
}

// keys[i] = (tile << 32) | depth bits of the Gaussian vals[i]: the tile is the last range
// starting at or before i (ranges are contiguous, so that range holds i).
__global__ void materialize_keys_kernel(const uint2 *__restrict__ ranges, int n_ranges,
                                        const uint32_t *__restrict__ vals,
                                        const float *__restrict__ rec, int n, int n_tiles,
                                        uint32_t count, uint64_t *__restrict__ keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += gridDim.x * blockDim.x) {
    int lo = 0, hi = n_ranges;   // ranges[lo].x <= i < ranges[hi].x (hi = n_ranges: none)
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (ranges[mid].x <= i) lo = mid;
      else hi = mid;
    }
    const uint32_t eye = (uint32_t)lo / (uint32_t)n_tiles;
    const uint32_t g = min(vals[i], (uint32_t)(n - 1));
    const float depth = rec[((size_t)eye * n + g) * kRec + 9];
    keys[i] = ((uint64_t)lo << 32) | __float_as_uint(depth);
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

BinParams bin_params(int n_eyes, int n, int tiles_x, int tiles_y, uint32_t capacity) {
  BinParams p{};
  p.n_eyes = n_eyes;
  p.n = n;
  p.n_entries = n_eyes * n;
  p.tiles_x = tiles_x;
  p.tiles_y = tiles_y;
  p.n_tiles = tiles_x * tiles_y;
  p.capacity = capacity;
  const long long n_ranges = (long long)n_eyes * p.n_tiles;
  p.row = (int)((n_ranges + 3) / 4 * 4);
  // bin_emit: one warp per (chunk, band of tile rows); a band holds at most kBandTiles tiles
  // (whole rows, at least one), so a warp's cursor table stays small however many tiles the
  // render has and many warps fit on an SM
  const int rows = n_eyes * tiles_y;
  p.band_rows = kBandTiles / (tiles_x > 0 ? tiles_x : 1);
  if (p.band_rows < 1) p.band_rows = 1;
  if (p.band_rows > rows) p.band_rows = rows > 0 ? rows : 1;
  p.n_bands = rows > 0 ? (rows + p.band_rows - 1) / p.band_rows : 1;
  // chunks: enough (chunk, band) warps to fill the device (as many as fit at once), at
  // least 256 entries each, at most kMaxChunks and kMaxChunkCells cells of h
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long per_warp = (long long)sizeof(uint32_t) * ((long long)p.band_rows * tiles_x + 8) +
                             2 * sizeof(uint32_t) * kMapPad + 1024;
  long long warps_per_sm = (228ll * 1024) / per_warp;
  if (warps_per_sm > 32) warps_per_sm = 32;
  if (warps_per_sm < 1) warps_per_sm = 1;
  long long max_chunks = kMaxChunkCells / (p.row > 0 ? p.row : 1);
  if (max_chunks > kMaxChunks) max_chunks = kMaxChunks;
  const long long fill = (warps_per_sm * sms + p.n_bands - 1) / p.n_bands;
  if (max_chunks > fill) max_chunks = fill;
  if (max_chunks < 1) max_chunks = 1;
  long long chunks = ((long long)p.n_entries + 255) / 256;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  long long L = ((long long)p.n_entries + chunks - 1) / chunks;
  L = (L + 31) / 32 * 32;
  if (L < 32) L = 32;
  p.chunk = (int)L;
  p.n_chunks = (int)(((long long)p.n_entries + L - 1) / L);
  if (p.n_chunks < 1) p.n_chunks = 1;
  return p;
}

size_t bin_chunk_cells(const BinParams &p) { return (size_t)p.n_chunks * (size_t)p.row; }

size_t bin_emit_smem_bytes(const BinParams &p) {
  // one band's cursors and up to 3 words either side of its 16-byte-aligned copy
  return sizeof(uint32_t) * ((size_t)p.band_rows * p.tiles_x + 8);
}

size_t bin_smem_bytes(int n_eyes, int tiles_x, int tiles_y) {
  const size_t a = bin_count_smem_bytes(n_eyes, tiles_x, tiles_y);
  const size_t b = bin_emit_smem_bytes(bin_params(n_eyes, 1, tiles_x, tiles_y, 0)) +
                   2 * sizeof(uint32_t) * kMapPad;
  return a > b ? a : b;
}

size_t bin_count_smem_bytes(int n_eyes, int tiles_x, int tiles_y) {
  return sizeof(uint32_t) * (size_t)n_eyes * tiles_x * tiles_y;
}

size_t bin_plan_lookback_bytes(int n_entries) {
  return sizeof(unsigned long long) * (size_t)((n_entries + kPlanEntries - 1) / kPlanEntries + 1);
}

cudaError_t launch_bin_plan(const BinParams &p, Entries entries, const uint32_t *touched,
                            const unsigned long long *inst_total, unsigned long long *lookback,
                            uint32_t *bounds, uint32_t *status, cudaStream_t s) {
  const int blocks = p.n_entries > 0 ? (p.n_entries + kPlanEntries - 1) / kPlanEntries : 1;
  {
    const cudaError_t e_ = launch_pdl(bin_plan_kernel, blocks, kPlanThreads, 0, s, p, entries, touched,
                                      inst_total, lookback, bounds, status);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_bin_count(const BinParams &p, Entries entries, const ushort4 *rect,
                             const uint32_t *bounds, uint32_t *h, cudaStream_t s) {
  const size_t smem = bin_count_smem_bytes(p.n_eyes, p.tiles_x, p.tiles_y);
  cudaError_t e = cudaFuncSetAttribute(bin_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  {
    const cudaError_t e_ = launch_pdl(bin_count_kernel, p.n_chunks, kCountThreads, smem, s, p, entries, rect,
                                      bounds, h);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

size_t bin_lookback_bytes(int n_eyes, int n_tiles) {
  return sizeof(unsigned long long) * (size_t)((n_eyes * n_tiles + 31) / 32 + 1);
}

cudaError_t launch_bin_offsets(const BinParams &p, uint32_t *h, unsigned long long *lookback,
                               uint2 *ranges, uint32_t *counts, uint32_t *status, cudaStream_t s) {
  const int n_ranges = p.n_eyes * p.n_tiles;
  const int blocks = (n_ranges + 31) / 32;
  const size_t smem = sizeof(uint32_t) * kOffsetThreads * (size_t)((p.n_chunks + 31) / 32);
  cudaError_t e = cudaFuncSetAttribute(bin_offsets_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  {
    const cudaError_t e_ = launch_pdl(bin_offsets_kernel,
                                      blocks > 0 ? blocks : 1, kOffsetThreads, smem, s, p, h, lookback, ranges, counts, status);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_bin_emit(const BinParams &p, Entries entries, const ushort4 *rect,
                            const uint32_t *bounds, const uint32_t *h, uint32_t *vals,
                            cudaStream_t s) {
  if (p.n_entries <= 0 || p.capacity == 0) return cudaSuccess;
  const size_t smem = bin_emit_smem_bytes(p);
  cudaError_t e = cudaFuncSetAttribute(bin_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  {
    const cudaError_t e_ = launch_pdl(bin_emit_kernel, p.n_chunks * p.n_bands, 32, smem, s, p, entries, rect,
                                      bounds, h, vals);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_materialize_keys(const uint2 *ranges, int n_ranges, const uint32_t *vals,
                                    const float *rec, int n, int n_tiles, uint32_t count,
                                    uint64_t *keys, cudaStream_t s) {
  if (count == 0 || n <= 0 || n_ranges <= 0) return cudaSuccess;
  materialize_keys_kernel<<<grid_for(count, 256), 256, 0, s>>>(ranges, n_ranges, vals, rec, n, n_tiles,
                                                               count, keys);
  return cudaGetLastError();
}

}  // namespace a3fr
