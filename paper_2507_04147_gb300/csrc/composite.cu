// composite.cu -- foveated front-to-back compositing of every tile of every eye (Sec. 2.3
// "Rasterization"; Sec. 3.4 AMR; Sec. 3.5 implementation details).
//
// Work is split the way the paper splits a tile: one group per 2x2-block label (TL 1,
// BR 2, TR 3, BL 4), and a level-k tile runs only the groups of labels 1..k.  Here a group
// is two warps: a 16x16 tile has 64 pixels per label, one per lane.
//
// fovea_plan computes every tile's level from the gaze in the device mailbox (Eq. 1: the
// distance from the gaze to the tile's nearest pixel centre against r_k = f tan(theta_k))
// and buckets the tiles by level.  composite then packs 8-warp CTAs so that no warp idles:
//   level 4: one tile per CTA, the CTA stages each batch of Gaussians together;
//   level 3: one tile per CTA, the last two warps only help staging;
//   level 2: two tiles per CTA, each half stages its own tile (named barrier);
//   level 1: four tiles per CTA, each warp pair stages its own tile (named barrier).
// A full-resolution render skips the plan: every tile is a level-4 CTA.
//
// Per batch, the staging threads gather the tile's next Gaussians (indices from the
// sorted values) into shared memory; each warp then blends them front to back with the
// 1/255 skip, the 0.99 clamp and the 1e-4 transmittance stop; the staging group stops when
// all its pixels are done.  The exp of the falloff uses the MUFU ex2 unit with log2(e)
// folded into the conic.  The blend is branch-free (predicated updates), so a warp whose
// lanes disagree on the accept test does not run both sides.  Label-1 warps also write the
// inherited pixels of their blocks.
#include <algorithm>

#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kTile = 16;
constexpr int kThreads = 256;          // 8 warps
// Level of tile `tile` of eye `eye` (exactly rounded; the same decision as the definition).
__device__ __forceinline__ int tile_level(const CompositeParams &p, int eye, int tile,
                                          const float *gaze) {
  const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
  const float gx = gaze[2 * eye], gy = gaze[2 * eye + 1];
  const float x0 = (float)(tx * p.tile), y0 = (float)(ty * p.tile);
  const float x1 = (float)(min((tx + 1) * p.tile, p.width) - 1);
  const float y1 = (float)(min((ty + 1) * p.tile, p.height) - 1);
  const float dx = fmaxf(fmaxf(fs(x0, gx), fs(gx, x1)), 0.0f);
  const float dy = fmaxf(fmaxf(fs(y0, gy), fs(gy, y1)), 0.0f);
  const float d2 = fa(fm(dx, dx), fm(dy, dy));
  int layer = p.n_layers - 1;
  for (int k = p.n_layers - 2; k >= 0; --k)
    if (d2 <= p.r2[eye][k]) layer = k;
  return p.level[layer];
}

// Count-based tile levels (Sec. 3.6, 4.6): per eye, the instance count tau of the k-th
// heaviest tile, k = floor(count_frac * tiles), by an exact radix select (four 8-bit digits,
// most significant first) over the tiles' range lengths in one CTA; tau = UINT32_MAX when
// k < 1 (no tile is heavy).
__global__ void __launch_bounds__(1024)
tile_threshold_kernel(const CompositeParams *__restrict__ pp, const uint2 *__restrict__ ranges,
                      uint32_t *__restrict__ thresholds) {
  pdl_begin();
  const CompositeParams &p = *pp;
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_prefix, s_k;
  const int t = threadIdx.x;
  for (int e = 0; e < p.n_eyes; ++e) {
    const uint32_t k0 = (uint32_t)floorf(p.count_frac * (float)p.n_tiles);
    if (k0 < 1u) {
      if (t == 0) thresholds[e] = 0xffffffffu;
      continue;
    }
    if (t == 0) {
      s_prefix = 0u;
      s_k = min(k0, (uint32_t)p.n_tiles);
    }
    __syncthreads();
    for (int shift = 24; shift >= 0; shift -= 8) {
      for (int i = t; i < 256; i += blockDim.x) s_hist[i] = 0u;
      __syncthreads();
      const uint32_t prefix = s_prefix;
      for (int i = t; i < p.n_tiles; i += blockDim.x) {
        const uint2 r = ranges[e * p.n_tiles + i];
        const uint32_t c = r.y - r.x;
        const bool match = shift == 24 || (c >> (shift + 8)) == prefix;
        if (match) atomicAdd(&s_hist[(c >> shift) & 255u], 1u);
      }
      __syncthreads();
      if (t == 0) {
        uint32_t k = s_k;
        int d = 255;
        for (; d > 0; --d) {
          if (s_hist[d] >= k) break;
          k -= s_hist[d];
        }
        s_k = k;
        s_prefix = (prefix << 8) | (uint32_t)d;
      }
      __syncthreads();
    }
    if (t == 0) thresholds[e] = s_prefix;
    __syncthreads();
  }
}

// Label interval (lo, hi] a composite renders in tile gt (eye-major global tile index), and
// the tile's bookkeeping (cur, levels).  Three uses:
//   * a normal foveated render: lo = 0, hi = the tile's level from the gaze mailbox (Eq. 1),
//     lowered for heavy tiles by the count-based rule when count_frac > 0;
//   * a uniform render (uniform > 0): lo = 0, hi = uniform for every tile (the first round of
//     a frame, and the full-resolution render with uniform = 4);
//   * a later round (round != nullptr): hi = the level from the round's gaze and radii, lo =
//     the level already rendered (cur); tiles with hi <= lo render nothing; cur becomes hi.
__device__ __forceinline__ void tile_interval(const CompositeParams &p, int gt, const float *gaze,
                                              const RoundPlan *round, int uniform, uint8_t *cur,
                                              uint8_t *levels, const uint2 *ranges,
                                              const uint32_t *thresholds, int *lo_out, int *hi_out) {
  const int eye = gt / p.n_tiles;
  const int tile = gt - eye * p.n_tiles;
  int lo = 0, hi;
  if (uniform > 0) {
    hi = uniform;
  } else if (round != nullptr) {
    hi = 0;
    if (round->active) {
      CompositeParams q = p;
      for (int k = 0; k < 3; ++k) q.r2[eye][k] = round->r2[eye][k];
      hi = tile_level(q, eye, tile, &round->gaze[0][0]);
    }
    lo = cur[gt];
  } else {
    hi = tile_level(p, eye, tile, gaze);
    if (p.count_frac > 0.0f && (hi == 2 || hi == 3)) {
      // a heavy tile (count >= the k-th largest count of its eye) drops one level
      const uint2 r = ranges[gt];
      const uint32_t c = r.y - r.x;
      if (c > 0u && c >= thresholds[eye]) hi -= 1;
    }
  }
  if (cur != nullptr && hi > lo) cur[gt] = (uint8_t)hi;
  levels[gt] = (uint8_t)(hi > lo ? hi : lo);
  *lo_out = lo;
  *hi_out = hi;
}

// Work plan of one 16-pixel-tile composite launch: entries (tile << 2 | lo) bucketed by
// hi - lo in plan[(hi - lo - 1) * n_ranges + slot], the bucket sizes in plan_counts[0..3].
__global__ void __launch_bounds__(256)
plan_kernel(const CompositeParams *__restrict__ pp, const float *__restrict__ gaze_ring,
            const RoundPlan *__restrict__ round, int uniform, uint8_t *__restrict__ cur,
            uint8_t *__restrict__ levels, uint32_t *__restrict__ plan,
            uint32_t *__restrict__ plan_counts, const uint2 *__restrict__ ranges,
            const uint32_t *__restrict__ thresholds) {
  pdl_begin();
  const CompositeParams &p = *pp;
  const float *gaze = gaze_ring + 4 * p.gaze_slot;
  const int n_ranges = p.n_eyes * p.n_tiles;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int lo = 0, count = 0;
  if (gt < n_ranges) {
    int hi;
    tile_interval(p, gt, gaze, round, uniform, cur, levels, ranges, thresholds, &lo, &hi);
    count = hi > lo ? hi - lo : 0;
  }
  for (int c = 1; c <= 4; ++c) {
    const unsigned m = __ballot_sync(0xffffffffu, count == c);
    if (!m) continue;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(plan_counts + (c - 1), (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (count == c)
      plan[(size_t)(c - 1) * n_ranges + base + __popc(m & ((1u << lane) - 1u))] =
          ((uint32_t)gt << 2) | (uint32_t)lo;
  }
}

// Work plan of one 32-pixel-tile composite launch (composite_px_kernel).  A tile rendering
// the P = hi - lo labels (lo, hi] is two work items, its top and bottom halves; a tile with
// no instances is one item that only writes background.  Items go into kItemClasses classes by the tile's
// instance count (class 0: none; class c: 4^(c-1) <= count < 4^c; the last class unbounded)
// and the composite takes the heaviest class first, so the longest items start first and
// the short ones fill in behind them.  items[c * 4 * n_ranges + slot] = gt << 6 |
// (P - 1) << 4 | region << 2 | lo, class sizes in class_counts[0..kItemClasses).
constexpr int kItemClasses = 8;

__global__ void __launch_bounds__(256)
plan32_kernel(const CompositeParams *__restrict__ pp, const float *__restrict__ gaze_ring,
              const RoundPlan *__restrict__ round, int uniform, uint8_t *__restrict__ cur,
              uint8_t *__restrict__ levels, uint32_t *__restrict__ items,
              uint32_t *__restrict__ class_counts, const uint2 *__restrict__ ranges,
              const uint32_t *__restrict__ thresholds) {
  pdl_begin();
  const CompositeParams &p = *pp;
  const float *gaze = gaze_ring + 4 * p.gaze_slot;
  const int n_ranges = p.n_eyes * p.n_tiles;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  if (gt >= n_ranges) return;
  int lo, hi;
  tile_interval(p, gt, gaze, round, uniform, cur, levels, ranges, thresholds, &lo, &hi);
  if (hi <= lo) return;
  const int P = hi - lo;
  const uint2 r = ranges[gt];
  const uint32_t count = r.y > r.x ? r.y - r.x : 0u;
  const int n_items = count == 0u ? 1 : 2;
  const int cls = count == 0u ? 0 : min(kItemClasses - 1, 1 + (31 - __clz(count)) / 2);
  const uint32_t slot = atomicAdd(class_counts + cls, (uint32_t)n_items);
  uint32_t *dst = items + (size_t)cls * 4 * n_ranges + slot;
  for (int k = 0; k < n_items; ++k)
    dst[k] = ((uint32_t)gt << 6) | ((uint32_t)(P - 1) << 4) | ((uint32_t)k << 2) | (uint32_t)lo;
}

// Conservative box of the pixels where a Gaussian can reach alpha >= 1/255: the ellipse
// d^T conic d <= 2 ln(255 opacity) has half-extents k sqrt(cov_xx), k sqrt(cov_yy) with cov
// the inverse of the conic; one pixel of margin absorbs rounding.  Empty (never hit) when
// opacity < 1/255.  (x0, x1, y0, y1).
__device__ __forceinline__ float4 support_box(float u, float v, float ca, float cb, float cc, float op) {
  const float k2 = 2.0f * __logf(255.0f * op);
  if (!(k2 > 0.0f)) return make_float4(1e30f, -1e30f, 1e30f, -1e30f);
  const float det = ca * cc - cb * cb;
  const float ex = sqrtf(k2 * cc / det) + 1.0f, ey = sqrtf(k2 * ca / det) + 1.0f;
  if (!(ex < 1e6f) || !(ey < 1e6f)) return make_float4(-1e30f, 1e30f, -1e30f, 1e30f);
  return make_float4(u - ex, u + ex, v - ey, v + ey);
}

// A support box rounded outward to whole pixels in 16 bits (clamped to +-kBoxFar, which no
// pixel reaches): a superset of the float box, so the integer test rejects no more.
constexpr short kBoxFar = 30000;
__device__ __forceinline__ short4 int_box(float4 b) {
  auto lo = [](float v) { return (short)fminf(fmaxf(floorf(v), -(float)kBoxFar), (float)kBoxFar); };
  auto hi = [](float v) { return (short)fminf(fmaxf(ceilf(v), -(float)kBoxFar), (float)kBoxFar); };
  return make_short4(lo(b.x), hi(b.y), lo(b.z), hi(b.w));
}

// Whether a Gaussian can reach alpha >= 1/255 at some point of the rectangle [x0, x1] x
// [y0, y1] (pixel coordinates relative to its centre): the log2 falloff f = A x^2 + B x y +
// C y^2 (A, C < 0: concave) is largest at the centre if the rectangle holds it, else on an
// edge, where the best point along the edge is the clamped stationary point.  thr is the
// falloff alpha = 1/255 needs, lowered by a margin (0.01 in log2) far above the rounding
// of f, of the stationary points and of the kernel's own alpha, so a Gaussian it rejects
// has alpha < 1/255 at every pixel of the rectangle: rejecting it changes no output bit.
__device__ __forceinline__ bool falloff_reaches(float A, float B, float C, float thr, float x0, float x1,
                                                float y0, float y1) {
  if (!(A < 0.0f) || !(C < 0.0f) || !(4.0f * A * C > 1.0001f * B * B)) return true;   // not concave
  if (x0 <= 0.0f && x1 >= 0.0f && y0 <= 0.0f && y1 >= 0.0f) return thr <= 0.0f;
  const float ky = __fdividef(-B, 2.0f * C), kx = __fdividef(-B, 2.0f * A);
  auto f = [&](float x, float y) { return (A * x + B * y) * x + C * y * y; };
  const float ya = fminf(fmaxf(ky * x0, y0), y1), yb = fminf(fmaxf(ky * x1, y0), y1);
  const float xa = fminf(fmaxf(kx * y0, x0), x1), xb = fminf(fmaxf(kx * y1, x0), x1);
  const float best = fmaxf(fmaxf(f(x0, ya), f(x1, yb)), fmaxf(f(xa, y0), f(xb, y1)));
  return best >= thr;
}

// Barrier of a staging group of `size` threads (64, 128 or 256) with barrier id `bar`
// (1..4).  The ids are literals so the kernel reserves 5 hardware barriers, not 16 (the
// per-SM barrier budget would otherwise cap residency at 4 CTAs).
__device__ __forceinline__ void group_sync(int size, int bar) {
  switch (bar) {
    case 1: asm volatile("bar.sync 1, %0;" ::"r"(size) : "memory"); break;
    case 2: asm volatile("bar.sync 2, %0;" ::"r"(size) : "memory"); break;
    case 3: asm volatile("bar.sync 3, %0;" ::"r"(size) : "memory"); break;
    default: asm volatile("bar.sync 4, %0;" ::"r"(size) : "memory"); break;
  }
}

template <bool kAux, bool kFull, int kMult>
__global__ void __launch_bounds__(kThreads, 6)
composite_kernel(const CompositeParams *__restrict__ pp, const float *__restrict__ rec, int n,
                 const uint2 *__restrict__ ranges, const uint32_t *__restrict__ kept,
                 const uint32_t *__restrict__ vals, const uint32_t *__restrict__ plan,
                 const uint32_t *__restrict__ plan_counts, int incremental,
                 uint8_t *__restrict__ levels, float *__restrict__ t_final,
                 uint32_t *__restrict__ n_contrib, float *__restrict__ depth,
                 unsigned long long *__restrict__ counters) {
  pdl_begin();
  const CompositeParams &p = *pp;   // per-render parameters in device memory
  float *out = p.out;
  __shared__ float4 s_geo[kThreads * kMult];   // u, v, -0.5 log2e a, -log2e b
  __shared__ float2 s_cz[kThreads * kMult];    // -0.5 log2e c, camera-space depth
  __shared__ float4 s_rgb[kThreads * kMult];   // r, g, b, opacity
  __shared__ int s_done[kThreads / 32];
  __shared__ float s_out[4][kTile][kTile * 3];   // the tiles of the CTA, assembled for stores

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_ranges = p.n_eyes * p.n_tiles;

  // ---- which tile, which labels (lo, level], which staging group; a label group is
  // two warps, and group = the label index (0 = top-left) this warp pair renders
  int gtile = -1, group = warp >> 1, level = 4, lo = 0, gsize = kThreads, gbar = 1, gfirst = 0;
  if (kFull) {
    gtile = blockIdx.x;
    if (threadIdx.x == 0) levels[gtile] = 4;
  } else {
    const int c = blockIdx.x;
    const int n4 = plan_counts[3], n3 = plan_counts[2], n2 = plan_counts[1], n1 = plan_counts[0];
    const int c3 = n4 + n3, c2 = c3 + (n2 + 1) / 2, c1 = c2 + (n1 + 3) / 4;
    uint32_t entry = 0xffffffffu;
    int count = 4;
    if (c < n4) {
      entry = plan[3 * (size_t)n_ranges + c];
    } else if (c < c3) {
      entry = plan[2 * (size_t)n_ranges + (c - n4)];
      count = 3;
    } else if (c < c2) {
      const int half = warp >> 2;
      const int slot = 2 * (c - c3) + half;
      count = 2;
      group = (warp >> 1) & 1;
      gsize = 128;
      gbar = 1 + half;
      gfirst = half * 128;
      if (slot < n2) entry = plan[(size_t)n_ranges + slot];
    } else if (c < c1) {
      const int quarter = warp >> 1;
      const int slot = 4 * (c - c2) + quarter;
      count = 1;
      group = 0;
      gsize = 64;
      gbar = 1 + quarter;
      gfirst = quarter * 64;
      if (slot < n1) entry = plan[slot];
    } else {
      return;
    }
    if (entry == 0xffffffffu) return;   // a partly filled pair or quad: these warps have no tile
    gtile = (int)(entry >> 2);
    lo = (int)(entry & 3u);
    level = lo + count;
    group += lo;
  }
  const int eye = gtile / p.n_tiles;
  const int tile = gtile - eye * p.n_tiles;
  const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;

  // ---- this lane's pixel: label `group` of block (bx, by) of the tile's 8x8 blocks
  const int ox = (group == 1 || group == 2) ? 1 : 0;   // BR, TR
  const int oy = (group == 1 || group == 3) ? 1 : 0;   // BR, BL
  const int bx = lane & 7, by = (warp & 1) * 4 + (lane >> 3);
  const int px = tx * kTile + 2 * bx + ox, py = ty * kTile + 2 * by + oy;
  const bool inside = group >= lo && group < level && px < p.width && py < p.height;
  const float fpx = (float)px, fpy = (float)py;

  uint2 range = ranges[gtile];
  const uint32_t n_kept = *kept;   // fewer than the instances only after a capacity overflow
  range.x = min(range.x, n_kept);
  range.y = min(range.y, n_kept);
  const float *rec_eye = rec + (size_t)eye * n * kRec;

  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
  float Z = 0.0f;                      // expected depth (auxiliary output)
  uint32_t last = 0;                   // 1-based position of the last contributor
  uint32_t stop = 0;                   // Gaussians evaluated when the pixel stopped
  uint32_t blended = 0;                // Gaussians blended into the pixel (auxiliary mode)
  bool done = !inside;
  uint32_t staged = 0;
  if (kFull) {   // compile-time layout: one level-4 tile, the whole CTA stages together
    group = warp >> 1;
    level = 4;
    lo = 0;
    gsize = kThreads;
    gbar = 1;
    gfirst = 0;
  }
  const int gt = threadIdx.x - gfirst;   // thread index inside the staging group
  const int sbase = gfirst * kMult;      // the group's staging slots
  const uint32_t bsz = (uint32_t)(gsize * kMult);   // Gaussians per batch

  for (uint32_t start = range.x; start < range.y; start += bsz) {
    // stop when every pixel of the staging group is done
    const bool wdone = __all_sync(0xffffffffu, done);
    if (lane == 0) s_done[warp] = wdone;
    group_sync(gsize, gbar);
    bool all = true;
    for (int w = gfirst >> 5; w < (gfirst + gsize) >> 5; ++w) all = all && s_done[w];
    if (all) break;
    const uint32_t cnt = min(bsz, range.y - start);
    staged += cnt;
#pragma unroll
    for (int j = 0; j < kMult; ++j) {
      const uint32_t slot = (uint32_t)(gt + j * gsize);
      if (slot < cnt) {
        const uint32_t gidx = min(vals[start + slot], (uint32_t)(n - 1));   // in range unless a sort failed
        const float4 *r4 = reinterpret_cast<const float4 *>(rec_eye + (size_t)gidx * kRec);
        const float4 a = __ldg(r4), b = __ldg(r4 + 1), c = __ldg(r4 + 2);
        s_geo[sbase + slot] = make_float4(a.x, a.y, __fmul_rn(-0.5f * kLog2e, a.z), __fmul_rn(-kLog2e, a.w));
        s_cz[sbase + slot] = make_float2(__fmul_rn(-0.5f * kLog2e, b.x), c.y);
        s_rgb[sbase + slot] = make_float4(b.z, b.w, c.x, b.y);
      } else if (slot < ((cnt + 3u) & ~3u)) {
        // padding up to a multiple of 4: zero opacity never passes the 1/255 test
        s_geo[sbase + slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        s_cz[sbase + slot] = make_float2(0.0f, 0.0f);
        s_rgb[sbase + slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
    }
    group_sync(gsize, gbar);
    if (!__all_sync(0xffffffffu, done)) {
      // Branch-free blending: every lane evaluates every Gaussian of the batch and the
      // update is predicated (a lane that is done, or outside the Gaussian's support or
      // below 1/255, keeps its state), so the warp never splits on the accept test.
      const uint32_t cnt4 = (cnt + 3u) & ~3u;
      const uint32_t pos0 = start - range.x + 1;
      for (uint32_t k = 0; k < cnt4; k += 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int e = sbase + (int)k + j;
          const float4 geo = s_geo[e];
          const float2 cz = s_cz[e];
          const float cc = cz.x;
          const float4 rgb = s_rgb[e];
          const float dx = __fsub_rn(geo.x, fpx), dy = __fsub_rn(geo.y, fpy);
          // power * log2(e) = -0.5 log2e (a dx^2 + c dy^2) - log2e b dx dy
          const float pw = falloff_log2(geo.z, geo.w, cc, dx, dy);
          const float alpha = blend_alpha(rgb.w, pw);
          const float tt = __fmul_rn(T, __fsub_rn(1.0f, alpha));
          const bool ok = !done && pw <= 0.0f && alpha >= 1.0f / 255.0f;
          const bool fin = ok && tt < 0.0001f;    // this Gaussian would end the pixel: stop
          const bool upd = ok && !fin;
          const uint32_t pos = pos0 + k + (uint32_t)j;
          const float w = upd ? alpha * T : 0.0f;
          C0 += rgb.x * w;
          C1 += rgb.y * w;
          C2 += rgb.z * w;
          if (kAux) {
            Z += cz.y * w;
            blended += upd ? 1u : 0u;
          }
          T = upd ? tt : T;
          last = upd ? pos : last;
          stop = fin ? pos : stop;
          done = done || fin;
        }
        if (__all_sync(0xffffffffu, done)) break;
      }
    }
    group_sync(gsize, gbar);   // the next batch overwrites the staged Gaussians
  }
  if (inside && !done) stop = range.y - range.x;

  // ---- outputs.  A tile rendered from label 0 is assembled in shared memory (its pixel,
  // and for label 1 the inherited pixels of its block) and stored row by row; a later
  // round (lo > 0) stores only the pixels it rendered, keeping the others.
  if (!kFull && incremental) {
    if (inside) {
      float *o = out + (((size_t)eye * p.height + py) * p.width + px) * 3;
      o[0] = C0;
      o[1] = C1;
      o[2] = C2;
      if (kAux) {
        const size_t pix = ((size_t)eye * p.height + py) * p.width + px;
        t_final[pix] = T;
        n_contrib[pix] = last;
        depth[pix] = Z;
      }
    }
  } else {
    const int slot = gfirst >> 6 >> (gsize == 256 ? 2 : (gsize == 128 ? 1 : 0));   // tile slot
    const int lx = 2 * bx + ox, ly = 2 * by + oy;
    if (inside) {
      float *o = &s_out[slot][ly][3 * lx];
      o[0] = C0;
      o[1] = C1;
      o[2] = C2;
      if (kAux) {
        const size_t pix = ((size_t)eye * p.height + py) * p.width + px;
        t_final[pix] = T;
        n_contrib[pix] = last;
        depth[pix] = Z;
      }
      if (group == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          // inherited pixels of the block: BR (label 2), TR (label 3), BL (label 4)
          const int dx = k < 2 ? 1 : 0, dy = k == 1 ? 0 : 1;
          if (level < k + 2 && px + dx < p.width && py + dy < p.height) {
            float *f = &s_out[slot][ly + dy][3 * (lx + dx)];
            f[0] = C0;
            f[1] = C1;
            f[2] = C2;
            if (kAux) {
              const size_t pix = ((size_t)eye * p.height + py + dy) * p.width + px + dx;
              t_final[pix] = T;
              n_contrib[pix] = last;
        depth[pix] = Z;
            }
          }
        }
      }
    }
    group_sync(gsize, gbar);
    const int w_tile = min(kTile, p.width - tx * kTile);
    const int h_tile = min(kTile, p.height - ty * kTile);
    const size_t row = (size_t)p.width * 3;
    float *dst = out + ((size_t)eye * p.height + ty * kTile) * row + (size_t)tx * kTile * 3;
    for (int f = gt; f < kTile * kTile * 3; f += gsize) {
      const int r = f / (3 * kTile), c = f - r * (3 * kTile);
      if (r < h_tile && c < 3 * w_tile) dst[(size_t)r * row + c] = s_out[slot][r][c];
    }
  }

  // ---- statistics: evaluations of this warp, records staged by this staging group, and
  // (auxiliary mode) blends
  unsigned long long ev = stop, bl = blended;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if (kAux) bl += __shfl_xor_sync(0xffffffffu, bl, o);
  }
  if (lane == 0) {
    if (kAux && ev) atomicAdd(counters, ev);
    if (gt == 0 && staged) atomicAdd(counters + 1, (unsigned long long)staged);
    if (kAux && bl) atomicAdd(counters + 2, bl);
  }
}


// 32 x 32 tiles (the paper's tiling, Sec. 3.5): a tile is 16 x 16 blocks of 2 x 2 pixels and
// a tile of labels (lo, hi] renders those P = hi - lo labels of every block and no others (the
// paper's groups above the level exit; here their pixels are never assigned).  Work items are
// half tiles (16 x 8 blocks): one persistent launch renders every item of the plan
// (plan32_kernel) -- both eyes, every layer -- taking items heaviest class first from an
// atomic counter, so the longest lists start first and the short ones fill in behind them,
// and a heavy tile is rendered by two CTAs at once.  A 128-thread CTA renders one item: each
// lane the P pixels of one block, so a staged Gaussian is set up once for the lane's P
// pixels; each warp covers 8 x 4 blocks (a 16 x 8 pixel area).  Per batch the CTA stages the
// tile's next Gaussians in shared memory with the box where each can reach alpha = 1/255;
// every warp builds its hit list (box test, then the exact falloff over its patch: a
// Gaussian left out has alpha < 1/255 at every pixel of the patch, so no output bit changes)
// and blends only those, front to back, with the 1/255 skip, the 0.99 clamp and the 1e-4
// stop.  The per-pixel arithmetic is the same as everywhere else, so images do not depend on
// how tiles are cut into items.  A tile rendered from label 0 also writes its inherited
// pixels (the labels above hi take the top-left value).
constexpr int kHalfThreads = 128;
constexpr int kBatch = 256;   // Gaussians staged per batch (times the staging multiple)

__device__ __forceinline__ int label_dx(int L) { return (L == 1 || L == 2) ? 1 : 0; }
__device__ __forceinline__ int label_dy(int L) { return (L == 1 || L == 3) ? 1 : 0; }

// Two fp32 values in one 64-bit register pair, and the packed fp32 arithmetic of sm_100 and
// later (add / mul / fma .rn.f32x2: each half rounded exactly as the scalar instruction), so
// two pixels of a lane take one instruction where the arithmetic is the same for both.
using f32x2 = unsigned long long;
__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// 1.0f where a >= b, else 0.0f (one instruction instead of a compare and a select)
__device__ __forceinline__ float ge_factor(float a, float b) {
  float r;
  asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

template <int kMult>
struct HalfSmem {
  float4 geo[kBatch * kMult];
  float2 cz[kBatch * kMult];
  float4 rgb[kBatch * kMult];
  short4 box[kBatch * kMult];        // support box, outward-rounded pixels
  float thr[kBatch * kMult];         // log2 falloff needed for alpha = 1/255
  uint16_t hits[kHalfThreads / 32][kBatch * kMult];   // per warp: batch slots that reach its patch
  int done[kHalfThreads / 32];
  uint32_t prefix[kItemClasses + 1];  // item index ranges, heaviest class first
  uint32_t item;
};

// One item: labels lo .. lo + P - 1 of the blocks of half `half` of tile gtile (kLo0: lo is
// 0, so the lane's pixel offsets are known at compile time).  Without the auxiliary outputs
// a finished pixel is marked by T = 0 (a live pixel keeps T >= 1e-4): skipped Gaussians then
// blend with alpha 0, which leaves T and the colour bit for bit as they were, and every
// later Gaussian of a finished pixel stops with weight 0.  With them the loop also keeps the
// final transmittance, the last contributor and the evaluation and blend counts.
template <int P, bool kAux, int kMult, bool kLo0>
__device__ __forceinline__ void render_half(HalfSmem<kMult> &sm, const CompositeParams &p, const float *rec,
                                            int n, uint2 range, int gtile, int half, int lo,
                                            bool inherit, const uint32_t *vals, float *t_final,
                                            uint32_t *n_contrib, float *depth,
                                            unsigned long long &ev, unsigned long long &bl,
                                            unsigned long long &staged) {
  constexpr int T32 = 32;
  constexpr int NB = kBatch * kMult;
  float *out = p.out;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int hi = lo + P;
  const int eye = gtile / p.n_tiles;
  const int tile = gtile - eye * p.n_tiles;
  const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
  const int bx = (lane & 7) + 8 * (warp & 1), by = 8 * half + 4 * (warp >> 1) + (lane >> 3);
  const int px0 = tx * T32 + 2 * bx, py0 = ty * T32 + 2 * by;   // the block's top-left pixel
  float fpx[P], fpy[P];
  bool inside[P];
  int any_ox = 0, all_ox = 1, any_oy = 0, all_oy = 1;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int L = kLo0 ? k : lo + k;
    const int ox = label_dx(L), oy = label_dy(L);
    any_ox |= ox;
    all_ox &= ox;
    any_oy |= oy;
    all_oy &= oy;
    inside[k] = px0 + ox < p.width && py0 + oy < p.height;
    fpx[k] = (float)(px0 + ox);
    fpy[k] = (float)(py0 + oy);
  }
  // the warp's patch: the span of its pixels (one label: every other pixel of 16 x 8)
  const int wxb = tx * T32 + 16 * (warp & 1), wyb = ty * T32 + 16 * half + 8 * (warp >> 1);
  const float wx0 = (float)(wxb + all_ox), wx1 = (float)(wxb + 14 + any_ox);
  const float wy0 = (float)(wyb + all_oy), wy1 = (float)(wyb + 6 + any_oy);
  const float *rec_eye = rec + (size_t)eye * n * kRec;

  float T[P], C0[P], C1[P], C2[P], Z[P];
  uint32_t last[P], stop[P];
  bool done[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    T[k] = kAux || inside[k] ? 1.0f : 0.0f;
    C0[k] = C1[k] = C2[k] = Z[k] = 0.0f;
    last[k] = stop[k] = 0u;
    done[k] = !inside[k];
  }
  auto all_done = [&]() {
    bool a = true;
#pragma unroll
    for (int k = 0; k < P; ++k) a = a && (kAux ? done[k] : T[k] == 0.0f);
    return a;
  };
  for (uint32_t start = range.x; start < range.y; start += NB) {
    const bool wdone = __all_sync(0xffffffffu, all_done());
    if (lane == 0) sm.done[warp] = wdone;
    __syncthreads();
    bool all = true;
#pragma unroll
    for (int w = 0; w < kHalfThreads / 32; ++w) all = all && sm.done[w];
    if (all) break;
    const uint32_t cnt = min((uint32_t)NB, range.y - start);
    if (t == 0) staged += cnt;
#pragma unroll
    for (int j = 0; j < NB / kHalfThreads; ++j) {
      const uint32_t slot = (uint32_t)(t + j * kHalfThreads);
      if (slot < cnt) {
        const uint32_t gidx = min(vals[start + slot], (uint32_t)(n - 1));   // in range unless a sort failed
        const float4 *r4 = reinterpret_cast<const float4 *>(rec_eye + (size_t)gidx * kRec);
        const float4 a = __ldg(r4), b = __ldg(r4 + 1), c = __ldg(r4 + 2);
        sm.geo[slot] = make_float4(a.x, a.y, __fmul_rn(-0.5f * kLog2e, a.z), __fmul_rn(-kLog2e, a.w));
        sm.cz[slot] = make_float2(__fmul_rn(-0.5f * kLog2e, b.x), c.y);
        sm.rgb[slot] = make_float4(b.z, b.w, c.x, b.y);
        sm.box[slot] = int_box(support_box(a.x, a.y, a.z, a.w, b.x, b.y));
        sm.thr[slot] = -__log2f(255.0f * b.y) - 0.01f;
      }
    }
    __syncthreads();
    if (!__all_sync(0xffffffffu, all_done())) {
      // the warp's hit list: 32 Gaussians tested per step (support box, then the falloff
      // over the patch), slots kept in list order
      int n_hit = 0;
      for (uint32_t base = 0; base < cnt; base += 32) {
        const uint32_t k = base + (uint32_t)lane;
        bool hit = false;
        if (k < cnt) {
          const short4 box = sm.box[k];
          hit = !((float)box.y < wx0 || (float)box.x > wx1 || (float)box.w < wy0 || (float)box.z > wy1);
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) sm.hits[warp][n_hit + __popc(m & ((1u << lane) - 1u))] = (uint16_t)k;
        n_hit += __popc(m);
      }
      __syncwarp();
      {
        int n_keep = 0;
        for (int base = 0; base < n_hit; base += 32) {
          const int i = base + lane;
          int k = 0;
          bool keep = false;
          if (i < n_hit) {
            k = sm.hits[warp][i];
            const float4 geo = sm.geo[k];
            keep = falloff_reaches(geo.z, geo.w, sm.cz[k].x, sm.thr[k], wx0 - geo.x, wx1 - geo.x,
                                   wy0 - geo.y, wy1 - geo.y);
          }
          __syncwarp();
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          if (keep) sm.hits[warp][n_keep + __popc(m & ((1u << lane) - 1u))] = (uint16_t)k;
          n_keep += __popc(m);
        }
        n_hit = n_keep;
      }
      __syncwarp();
      const uint32_t pos0 = start - range.x + 1;
      for (int i = 0; i < n_hit; i += 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (i + j >= n_hit) break;
          const int e = sm.hits[warp][i + j];
          const float4 geo = sm.geo[e];
          const float2 cz = sm.cz[e];
          const float4 rgb = sm.rgb[e];
          const uint32_t pos = pos0 + (uint32_t)e;
          if constexpr (!kAux && P >= 2) {
            // pixel pairs (0, 1) and (2, 3): the same operations as the scalar loop below, two
            // pixels per instruction wherever both take the same one
            const f32x2 gx = f2_pack(geo.x, geo.x), gy = f2_pack(geo.y, geo.y);
            const f32x2 ca = f2_pack(geo.z, geo.z), cb = f2_pack(geo.w, geo.w), cc = f2_pack(cz.x, cz.x);
            const f32x2 op = f2_pack(rgb.w, rgb.w);
            const f32x2 cr = f2_pack(rgb.x, rgb.x), cg = f2_pack(rgb.y, rgb.y), cbl = f2_pack(rgb.z, rgb.z);
            const f32x2 one = f2_pack(1.0f, 1.0f), mone = f2_pack(-1.0f, -1.0f);
#pragma unroll
            for (int k = 0; k + 1 < P; k += 2) {
              const f32x2 dx = f2_add(gx, f2_pack(-fpx[k], -fpx[k + 1]));
              const f32x2 dy = f2_add(gy, f2_pack(-fpy[k], -fpy[k + 1]));
              // falloff_log2: (A dx + B dy) dx + (C dy) dy, rounded step by step
              const f32x2 pw2 = f2_fma(f2_fma(ca, dx, f2_mul(cb, dy)), dx, f2_mul(f2_mul(cc, dy), dy));
              float pw0, pw1;
              f2_unpack(pw2, pw0, pw1);
              float oe0, oe1;
              f2_unpack(f2_mul(op, f2_pack(ex2_approx(pw0), ex2_approx(pw1))), oe0, oe1);
              const float al0 = fminf(0.99f, oe0), al1 = fminf(0.99f, oe1);
              const float a0 = (pw0 <= 0.0f && al0 >= 1.0f / 255.0f) ? al0 : 0.0f;
              const float a1 = (pw1 <= 0.0f && al1 >= 1.0f / 255.0f) ? al1 : 0.0f;
              const f32x2 a2 = f2_pack(a0, a1), t2 = f2_pack(T[k], T[k + 1]);
              const f32x2 tt2 = f2_mul(t2, f2_fma(a2, mone, one));   // T (1 - a)
              float tt0, tt1;
              f2_unpack(tt2, tt0, tt1);
              // 1 while the pixel goes on, 0 once this Gaussian would end it (or it ended):
              // multiplying by it equals the scalar path's selects bit for bit (T, a T >= 0)
              const f32x2 keep = f2_pack(ge_factor(tt0, 0.0001f), ge_factor(tt1, 0.0001f));
              const f32x2 w2 = f2_mul(f2_mul(a2, t2), keep);
              f2_unpack(f2_fma(cr, w2, f2_pack(C0[k], C0[k + 1])), C0[k], C0[k + 1]);
              f2_unpack(f2_fma(cg, w2, f2_pack(C1[k], C1[k + 1])), C1[k], C1[k + 1]);
              f2_unpack(f2_fma(cbl, w2, f2_pack(C2[k], C2[k + 1])), C2[k], C2[k + 1]);
              f2_unpack(f2_mul(tt2, keep), T[k], T[k + 1]);
            }
          }
          if constexpr (kAux && P >= 2) {
            // the same pairs with the auxiliary outputs: the arithmetic packed, the bookkeeping
            // (done, last contributor, stop position, blend count) per pixel
            const f32x2 gx = f2_pack(geo.x, geo.x), gy = f2_pack(geo.y, geo.y);
            const f32x2 ca = f2_pack(geo.z, geo.z), cb = f2_pack(geo.w, geo.w), cc = f2_pack(cz.x, cz.x);
            const f32x2 op = f2_pack(rgb.w, rgb.w);
            const f32x2 cr = f2_pack(rgb.x, rgb.x), cg = f2_pack(rgb.y, rgb.y), cbl = f2_pack(rgb.z, rgb.z);
            const f32x2 cdz = f2_pack(cz.y, cz.y);
            const f32x2 one = f2_pack(1.0f, 1.0f), mone = f2_pack(-1.0f, -1.0f);
#pragma unroll
            for (int k = 0; k + 1 < P; k += 2) {
              const f32x2 dx = f2_add(gx, f2_pack(-fpx[k], -fpx[k + 1]));
              const f32x2 dy = f2_add(gy, f2_pack(-fpy[k], -fpy[k + 1]));
              const f32x2 pw2 = f2_fma(f2_fma(ca, dx, f2_mul(cb, dy)), dx, f2_mul(f2_mul(cc, dy), dy));
              float pw0, pw1;
              f2_unpack(pw2, pw0, pw1);
              float oe0, oe1;
              f2_unpack(f2_mul(op, f2_pack(ex2_approx(pw0), ex2_approx(pw1))), oe0, oe1);
              const float al0 = fminf(0.99f, oe0), al1 = fminf(0.99f, oe1);
              const f32x2 al2 = f2_pack(al0, al1), t2 = f2_pack(T[k], T[k + 1]);
              float tt0, tt1, at0, at1;
              f2_unpack(f2_mul(t2, f2_fma(al2, mone, one)), tt0, tt1);   // T (1 - alpha)
              f2_unpack(f2_mul(al2, t2), at0, at1);
              const bool ok0 = !done[k] && pw0 <= 0.0f && al0 >= 1.0f / 255.0f;
              const bool ok1 = !done[k + 1] && pw1 <= 0.0f && al1 >= 1.0f / 255.0f;
              const bool fin0 = ok0 && tt0 < 0.0001f, fin1 = ok1 && tt1 < 0.0001f;
              const bool upd0 = ok0 && !fin0, upd1 = ok1 && !fin1;
              const f32x2 w2 = f2_pack(upd0 ? at0 : 0.0f, upd1 ? at1 : 0.0f);
              f2_unpack(f2_fma(cr, w2, f2_pack(C0[k], C0[k + 1])), C0[k], C0[k + 1]);
              f2_unpack(f2_fma(cg, w2, f2_pack(C1[k], C1[k + 1])), C1[k], C1[k + 1]);
              f2_unpack(f2_fma(cbl, w2, f2_pack(C2[k], C2[k + 1])), C2[k], C2[k + 1]);
              f2_unpack(f2_fma(cdz, w2, f2_pack(Z[k], Z[k + 1])), Z[k], Z[k + 1]);
              bl += (upd0 ? 1u : 0u) + (upd1 ? 1u : 0u);
              T[k] = upd0 ? tt0 : T[k];
              T[k + 1] = upd1 ? tt1 : T[k + 1];
              last[k] = upd0 ? pos : last[k];
              last[k + 1] = upd1 ? pos : last[k + 1];
              stop[k] = fin0 ? pos : stop[k];
              stop[k + 1] = fin1 ? pos : stop[k + 1];
              done[k] = done[k] || fin0;
              done[k + 1] = done[k + 1] || fin1;
            }
          }
#pragma unroll
          for (int k = 0; k < P; ++k) {
            if constexpr (P >= 2) {
              if (k + 1 < P || P % 2 == 0) continue;   // done in pairs above (all but an odd last)
            }
            const float dx = __fsub_rn(geo.x, fpx[k]), dy = __fsub_rn(geo.y, fpy[k]);
            const float pw = falloff_log2(geo.z, geo.w, cz.x, dx, dy);
            const float alpha = blend_alpha(rgb.w, pw);
            if constexpr (kAux) {
              const float tt = __fmul_rn(T[k], __fsub_rn(1.0f, alpha));
              const bool ok = !done[k] && pw <= 0.0f && alpha >= 1.0f / 255.0f;
              const bool fin = ok && tt < 0.0001f;
              const bool upd = ok && !fin;
              const float w = upd ? __fmul_rn(alpha, T[k]) : 0.0f;
              C0[k] = __fmaf_rn(rgb.x, w, C0[k]);
              C1[k] = __fmaf_rn(rgb.y, w, C1[k]);
              C2[k] = __fmaf_rn(rgb.z, w, C2[k]);
              Z[k] = __fmaf_rn(cz.y, w, Z[k]);
              bl += upd ? 1u : 0u;
              T[k] = upd ? tt : T[k];
              last[k] = upd ? pos : last[k];
              stop[k] = fin ? pos : stop[k];
              done[k] = done[k] || fin;
            } else {
              const float a = (pw <= 0.0f && alpha >= 1.0f / 255.0f) ? alpha : 0.0f;
              const float tt = __fmul_rn(T[k], __fsub_rn(1.0f, a));
              const bool fin = tt < 0.0001f;   // this Gaussian would end the pixel, or it ended
              const float w = fin ? 0.0f : __fmul_rn(a, T[k]);
              C0[k] = __fmaf_rn(rgb.x, w, C0[k]);
              C1[k] = __fmaf_rn(rgb.y, w, C1[k]);
              C2[k] = __fmaf_rn(rgb.z, w, C2[k]);
              T[k] = fin ? 0.0f : tt;
            }
          }
        }
        if (__all_sync(0xffffffffu, all_done())) break;
      }
    }
    __syncthreads();   // the next batch overwrites the staged Gaussians
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    if (!inside[k]) continue;
    if (kAux) {
      if (!done[k]) stop[k] = range.y - range.x;
      ev += stop[k];
    }
    const size_t pix = ((size_t)eye * p.height + (size_t)fpy[k]) * p.width + (size_t)fpx[k];
    out[3 * pix] = C0[k];
    out[3 * pix + 1] = C1[k];
    out[3 * pix + 2] = C2[k];
    if (kAux) {
      t_final[pix] = T[k];
      n_contrib[pix] = last[k];
      depth[pix] = Z[k];
    }
  }
  if (inherit && inside[0]) {
    // the inherited pixels of the block: the labels above the level take the top-left value
    for (int L = hi; L < 4; ++L) {
      const int x = px0 + label_dx(L), y = py0 + label_dy(L);
      if (x >= p.width || y >= p.height) continue;
      const size_t q = ((size_t)eye * p.height + y) * p.width + x;
      out[3 * q] = C0[0];
      out[3 * q + 1] = C1[0];
      out[3 * q + 2] = C2[0];
      if (kAux) {
        t_final[q] = T[0];
        n_contrib[q] = last[0];
        depth[q] = Z[0];
      }
    }
  }
}

template <bool kAux, int kMult>
__global__ void __launch_bounds__(kHalfThreads, kAux ? 6 : 7)
composite_px_kernel(const CompositeParams *__restrict__ pp, const float *__restrict__ rec, int n,
                    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ kept,
                    const uint32_t *__restrict__ vals, const uint32_t *__restrict__ items,
                    const uint32_t *__restrict__ class_counts, uint32_t *__restrict__ work,
                    int incremental, float *__restrict__ t_final,
                    uint32_t *__restrict__ n_contrib, float *__restrict__ depth,
                    unsigned long long *__restrict__ counters) {
  pdl_begin();
  __shared__ HalfSmem<kMult> sm;
  const CompositeParams &p = *pp;
  float *out = p.out;
  const int t = threadIdx.x, lane = t & 31;
  const int n_ranges = p.n_eyes * p.n_tiles;
  const size_t cap = 4 * (size_t)n_ranges;
  if (t == 0) {
    sm.prefix[0] = 0u;
    for (int i = 0; i < kItemClasses; ++i)
      sm.prefix[i + 1] = sm.prefix[i] + class_counts[kItemClasses - 1 - i];
  }
  __syncthreads();
  const uint32_t total = sm.prefix[kItemClasses];
  const uint32_t n_kept = *kept;   // fewer than the instances only after a capacity overflow
  unsigned long long ev = 0, bl = 0, staged = 0;

  for (;;) {
    if (t == 0) sm.item = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t w = sm.item;
    if (w >= total) break;
    int ci = 0;
    while (w >= sm.prefix[ci + 1]) ++ci;
    const uint32_t item = items[(size_t)(kItemClasses - 1 - ci) * cap + (w - sm.prefix[ci])];
    const int gtile = (int)(item >> 6);
    const int P = (int)((item >> 4) & 3u) + 1;
    const int half = (int)((item >> 2) & 3u);
    const int lo = (int)(item & 3u), hi = lo + P;
    uint2 range = ranges[gtile];
    range.x = min(range.x, n_kept);
    range.y = min(range.y, n_kept);
    const bool inherit = !incremental && lo == 0 && hi < 4;
    if (range.y <= range.x) {
      // no Gaussian reaches the tile: background (0) for every pixel the tile's items would
      // write (this is the tile's only item)
      const int eye = gtile / p.n_tiles;
      const int tile = gtile - eye * p.n_tiles;
      const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
      for (int b = t; b < 256; b += kHalfThreads) {
        const int px0 = tx * 32 + 2 * (b & 15), py0 = ty * 32 + 2 * (b >> 4);
        for (int L = lo; L < 4; ++L) {
          if (L >= hi && !inherit) break;
          const int x = px0 + label_dx(L), y = py0 + label_dy(L);
          if (x >= p.width || y >= p.height) continue;
          const size_t pix = ((size_t)eye * p.height + y) * p.width + x;
          out[3 * pix] = 0.0f;
          out[3 * pix + 1] = 0.0f;
          out[3 * pix + 2] = 0.0f;
          if (kAux) {
            t_final[pix] = 1.0f;
            n_contrib[pix] = 0u;
            depth[pix] = 0.0f;
          }
        }
      }
    } else {
#define A3FR_HALF(PP, LO0) \
  render_half<PP, kAux, kMult, LO0>(sm, p, rec, n, range, gtile, half, lo, inherit, vals, t_final, \
                                    n_contrib, depth, ev, bl, staged)
      if (lo == 0) {
        switch (P) {
          case 1: A3FR_HALF(1, true); break;
          case 2: A3FR_HALF(2, true); break;
          case 3: A3FR_HALF(3, true); break;
          default: A3FR_HALF(4, true); break;
        }
      } else {   // later rounds: labels above the ones already rendered (lo + P <= 4)
        switch (P) {
          case 1: A3FR_HALF(1, false); break;
          case 2: A3FR_HALF(2, false); break;
          default: A3FR_HALF(3, false); break;
        }
      }
#undef A3FR_HALF
    }
    __syncthreads();   // every thread has read sm.item and is done with the staging arrays
  }
  // statistics: records staged (thread 0 counts its CTA's); with the auxiliary outputs also
  // the evaluations and the blends
  if (kAux) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ev += __shfl_xor_sync(0xffffffffu, ev, o);
      bl += __shfl_xor_sync(0xffffffffu, bl, o);
    }
    if (lane == 0) {
      if (ev) atomicAdd(counters, ev);
      if (bl) atomicAdd(counters + 2, bl);
    }
  }
  if (t == 0 && staged) atomicAdd(counters + 1, staged);
}

}  // namespace

// The plan buffer: the 16-pixel path's buckets [4 * n_ranges] and counts [4] at its start,
// the 32-pixel path's items [kItemClasses * 4 * n_ranges], then its class counts
// [kItemClasses] and work counter.
size_t plan_bytes(int n_ranges) {
  return sizeof(uint32_t) * ((size_t)kItemClasses * 4 * (size_t)n_ranges + kItemClasses + 8);
}

cudaError_t launch_composite(const CompositeParams &p, const CompositeParams *p_dev,
                             const float *rec, int n, const uint2 *ranges, const uint32_t *kept,
                             const uint32_t *vals, const float *gaze, const RoundPlan *round,
                             int uniform, uint8_t *cur, uint32_t *plan, uint8_t *levels,
                             float *t_final, uint32_t *n_contrib, float *depth,
                             unsigned long long *counters, int batch_mult, uint32_t *thresholds,
                             cudaStream_t s, int *kernels) {
  const int n_ranges = p.n_eyes * p.n_tiles;
  if (kernels) *kernels = 0;
  if (n_ranges <= 0) return cudaSuccess;
  const int inc = round != nullptr ? 1 : 0;
  const bool aux = t_final != nullptr;
  const int mult = batch_mult == 2 ? 2 : 1;
  const bool by_count = !p.full && p.count_frac > 0.0f && round == nullptr && uniform == 0;
  // shared memory preferred so that registers, not the carveout, set residency
  auto prefer_smem = [](auto kern, int variant) {
    static bool carve[64][16] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && variant >= 0 && variant < 16 &&
        !carve[dev][variant]) {
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
      carve[dev][variant] = true;
    }
  };
  if (by_count) {
    {
      const cudaError_t e_ = launch_pdl(tile_threshold_kernel, 1, 1024, 0, s, p_dev, ranges, thresholds);
      if (e_ != cudaSuccess) return e_;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (kernels) ++*kernels;
  }
  if (p.tile == 32) {
    // plan (every tile, also for the full render: uniform level 4) + one persistent composite
    uint32_t *items = plan;
    uint32_t *class_counts = plan + (size_t)kItemClasses * 4 * n_ranges;
    uint32_t *work = class_counts + kItemClasses;
    cudaError_t e = cudaMemsetAsync(class_counts, 0, sizeof(uint32_t) * (kItemClasses + 1), s);
    if (e != cudaSuccess) return e;
    {
      const cudaError_t e_ = launch_pdl(plan32_kernel, (n_ranges + 255) / 256, 256, 0, s, p_dev, gaze, round,
                                        p.full ? 4 : uniform, cur, levels, items, class_counts, ranges,
                                        thresholds);
      if (e_ != cudaSuccess) return e_;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto go = [&](auto kern, int variant) -> cudaError_t {
      prefer_smem(kern, variant);
      static int per_sm[64][16] = {};
      int dev = 0;
      cudaGetDevice(&dev);
      int occ = (dev >= 0 && dev < 64) ? per_sm[dev][variant] : 0;
      int sms = 0;
      if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kHalfThreads, 0) != cudaSuccess || occ < 1)
          occ = 1;
        if (dev >= 0 && dev < 64) per_sm[dev][variant] = occ;
      }
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
      const long max_items = 2L * n_ranges;
      const int grid = (int)std::min<long>((long)sms * occ, max_items);
      {
        const cudaError_t e_ = launch_pdl(kern, grid, kHalfThreads, 0, s, p_dev, rec, n, ranges, kept, vals,
                                          items, class_counts, work, inc, t_final, n_contrib, depth,
                                          counters);
        if (e_ != cudaSuccess) return e_;
      }
      return cudaGetLastError();
    };
    e = aux ? (mult == 2 ? go(composite_px_kernel<true, 2>, 0) : go(composite_px_kernel<true, 1>, 1))
            : (mult == 2 ? go(composite_px_kernel<false, 2>, 2) : go(composite_px_kernel<false, 1>, 3));
    if (kernels) *kernels += 2;
    return e;
  }
  uint32_t *pc = plan + 4 * (size_t)n_ranges;
  if (!p.full) {
    cudaError_t e = cudaMemsetAsync(pc, 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    {
      const cudaError_t e_ = launch_pdl(plan_kernel, (n_ranges + 255) / 256, 256, 0, s, p_dev, gaze, round,
                                        uniform, cur, levels, plan, pc, ranges, thresholds);
      if (e_ != cudaSuccess) return e_;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (kernels) ++*kernels;
  }
  auto launch = [&](auto kern, int variant) -> cudaError_t {
    prefer_smem(kern, 4 + variant);
    {
      const cudaError_t e_ = launch_pdl(kern, n_ranges, kThreads, 0, s, p_dev, rec, n, ranges, kept, vals,
                                        plan, pc, p.full ? 0 : inc, levels, t_final, n_contrib, depth,
                                        counters);
      if (e_ != cudaSuccess) return e_;
    }
    if (kernels) ++*kernels;
    return cudaGetLastError();
  };
  if (aux) {
    if (p.full) return mult == 2 ? launch(composite_kernel<true, true, 2>, 0) : launch(composite_kernel<true, true, 1>, 1);
    return mult == 2 ? launch(composite_kernel<true, false, 2>, 2) : launch(composite_kernel<true, false, 1>, 3);
  }
  if (p.full) return mult == 2 ? launch(composite_kernel<false, true, 2>, 4) : launch(composite_kernel<false, true, 1>, 5);
  return mult == 2 ? launch(composite_kernel<false, false, 2>, 6) : launch(composite_kernel<false, false, 1>, 7);
}

}  // namespace a3fr
