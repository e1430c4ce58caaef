// composite.cu -- foveated front-to-back compositing of every tile of every eye in one
// launch (Sec. 2.3 "Rasterization"; Sec. 3.4 AMR; Sec. 3.5 implementation details).
//
// One CTA renders one 16x16 tile.  Its level (Eq. 1: distance from the gaze in the
// device mailbox to the tile's nearest pixel centre against r_k = f tan(theta_k)) is
// computed by the CTA itself, so the level map costs no launch.  The 256 threads form the
// paper's four groups of 64, one per 2x2-block label (TL 1, BR 2, TR 3, BL 4): group g
// renders label g+1 of each of the tile's 8x8 blocks, and a level-k tile runs groups
// 0..k-1 while the other warps only help stage Gaussians (they never touch the FP32 or
// MUFU pipes).  Pixels are compacted by label, so every warp that works holds 32 live
// pixels.
//
// Each round, all 256 threads gather the records of the next 256 Gaussians of the tile's
// depth-sorted list (indices from the sorted values) into shared memory; the live
// threads then blend them front to back with the 1/255 skip, the 0.99 clamp and the 1e-4
// transmittance stop.  A CTA-wide vote ends the tile as soon as every pixel is done.  The
// exp of the Gaussian falloff uses the MUFU ex2 unit with log2(e) folded into the conic,
// and the 1/255 test is made on the exponent first (log2 threshold per Gaussian), so
// pixels outside a Gaussian's support never reach the exp.
// Results are assembled in shared memory (label-1 threads also write the inherited
// pixels of their block) and stored row by row.
#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kTile = 16;
constexpr int kThreads = 256;
constexpr int kBatch = 256;
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <bool kAux>
__global__ void __launch_bounds__(kThreads)
composite_kernel(CompositeParams p, const float *__restrict__ rec, int n,
                 const uint2 *__restrict__ ranges, const uint32_t *__restrict__ kept,
                 const uint32_t *__restrict__ vals,
                 const float *__restrict__ gaze, float *__restrict__ out,
                 uint8_t *__restrict__ levels, float *__restrict__ t_final,
                 uint32_t *__restrict__ n_contrib, unsigned long long *__restrict__ counters) {
  __shared__ float4 s_geo[kBatch];    // u, v, -0.5 log2e a, -log2e b
  __shared__ float4 s_co[kBatch];     // -0.5 log2e c, log2 threshold, unused, unused
  __shared__ float4 s_rgb[kBatch];    // r, g, b, opacity
  __shared__ float s_out[kTile][kTile][3];
  __shared__ unsigned long long s_eval;

  const int gtile = blockIdx.x;
  const int eye = gtile / p.n_tiles;
  const int tile = gtile - eye * p.n_tiles;
  const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
  const int t = threadIdx.x;

  // tile level from the gaze (exactly rounded, same decision as the definition)
  int level = 4;
  if (!p.full) {
    const float gx = gaze[2 * eye], gy = gaze[2 * eye + 1];
    const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
    const float x1 = (float)(min((tx + 1) * kTile, p.width) - 1);
    const float y1 = (float)(min((ty + 1) * kTile, p.height) - 1);
    const float dx = fmaxf(fmaxf(fs(x0, gx), fs(gx, x1)), 0.0f);
    const float dy = fmaxf(fmaxf(fs(y0, gy), fs(gy, y1)), 0.0f);
    const float d2 = fa(fm(dx, dx), fm(dy, dy));
    int layer = p.n_layers - 1;
    for (int k = p.n_layers - 2; k >= 0; --k)
      if (d2 <= p.r2[eye][k]) layer = k;
    level = p.level[layer];
  }
  if (t == 0) {
    levels[gtile] = (uint8_t)level;
    s_eval = 0ull;
  }

  // compacted pixel of this thread: group g = label g+1, block (bx, by) of the 8x8
  const int g = t >> 6, j = t & 63;
  const int bx = j & 7, by = j >> 3;
  const int ox = (g == 1 || g == 2) ? 1 : 0;     // BR, TR
  const int oy = (g == 1 || g == 3) ? 1 : 0;     // BR, BL
  const int lx = 2 * bx + ox, ly = 2 * by + oy;
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool inside = px < p.width && py < p.height;
  const bool live = (g < level) && inside;
  const float fpx = (float)px, fpy = (float)py;

  uint2 range = ranges[gtile];
  const uint32_t n_kept = *kept;   // fewer than the instances only after a capacity overflow
  range.x = min(range.x, n_kept);
  range.y = min(range.y, n_kept);
  const float *rec_eye = rec + (size_t)eye * n * kRec;
  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
  uint32_t contrib = 0, evals = 0;
  bool done = !live;
  uint32_t staged = 0;

  for (uint32_t start = range.x; start < range.y; start += kBatch) {
    if (__syncthreads_count(done) == kThreads) break;
    staged += min((uint32_t)kBatch, range.y - start);
    const uint32_t idx = start + t;
    if (idx < range.y) {
      const uint32_t gidx = min(vals[idx], (uint32_t)(n - 1));   // in range unless a sort failed
      const float4 *r4 = reinterpret_cast<const float4 *>(rec_eye + (size_t)gidx * kRec);
      const float4 a = __ldg(r4), b = __ldg(r4 + 1), c = __ldg(r4 + 2);
      // alpha >= 1/255  <=>  power * log2e >= log2(1 / (255 opacity)) = thr
      const float op = b.y;
      const float thr = -lg2_approx(255.0f * op);
      s_geo[t] = make_float4(a.x, a.y, -0.5f * kLog2e * a.z, -kLog2e * a.w);
      s_co[t] = make_float4(-0.5f * kLog2e * b.x, thr, 0.0f, 0.0f);
      s_rgb[t] = make_float4(b.z, b.w, c.x, op);
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kBatch, range.y - start);
    if (!done) {
      for (int k = 0; k < cnt; ++k) {
        const float4 geo = s_geo[k];
        const float4 co = s_co[k];
        ++evals;
        const float dx = geo.x - fpx, dy = geo.y - fpy;
        // power * log2(e) = -0.5 log2e (a dx^2 + c dy^2) - log2e b dx dy
        const float pw = geo.z * dx * dx + co.x * dy * dy + geo.w * dx * dy;
        if (pw > 0.0f || pw < co.y) continue;
        const float4 rgb = s_rgb[k];
        const float alpha = fminf(0.99f, rgb.w * ex2_approx(pw));
        if (alpha < 1.0f / 255.0f) continue;
        const float test_t = T * (1.0f - alpha);
        if (test_t < 0.0001f) {
          done = true;
          break;
        }
        const float w = alpha * T;
        C0 += rgb.x * w;
        C1 += rgb.y * w;
        C2 += rgb.z * w;
        T = test_t;
        contrib = evals;
      }
    }
  }

  // statistics: evaluations and staged records of the tile
  unsigned long long ev = evals;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
  if ((t & 31) == 0 && ev) atomicAdd(&s_eval, ev);

  // assemble the tile: live pixels, then label-1 threads fill the inherited ones
  if (live) {
    s_out[ly][lx][0] = C0;
    s_out[ly][lx][1] = C1;
    s_out[ly][lx][2] = C2;
    if (g == 0) {
      if (level < 2) { s_out[ly + 1][lx + 1][0] = C0; s_out[ly + 1][lx + 1][1] = C1; s_out[ly + 1][lx + 1][2] = C2; }
      if (level < 3) { s_out[ly][lx + 1][0] = C0; s_out[ly][lx + 1][1] = C1; s_out[ly][lx + 1][2] = C2; }
      if (level < 4) { s_out[ly + 1][lx][0] = C0; s_out[ly + 1][lx][1] = C1; s_out[ly + 1][lx][2] = C2; }
    }
  }
  if (kAux && inside) {
    // aux buffers describe the shaded pixel; inherited pixels repeat their top-left
    const size_t pix = ((size_t)eye * p.height + py) * p.width + px;
    if (live) {
      t_final[pix] = T;
      n_contrib[pix] = contrib;
    }
  }
  __syncthreads();
  if (kAux && g == 0 && inside) {
    // inherited pixels of this block take the top-left pixel's aux values
    const int sx[3] = {1, 1, 0}, sy[3] = {1, 0, 1}, need[3] = {2, 3, 4};
    for (int q = 0; q < 3; ++q) {
      const int qx = px + sx[q], qy = py + sy[q];
      if (level < need[q] && qx < p.width && qy < p.height) {
        const size_t pix = ((size_t)eye * p.height + qy) * p.width + qx;
        t_final[pix] = T;
        n_contrib[pix] = contrib;
      }
    }
  }
  const int w_tile = min(kTile, p.width - tx * kTile);
  const int h_tile = min(kTile, p.height - ty * kTile);
  const int row_floats = 3 * w_tile;
  for (int f = t; f < kTile * 3 * kTile; f += kThreads) {
    const int r = f / (3 * kTile), c = f - r * (3 * kTile);
    if (r < h_tile && c < row_floats) {
      const size_t o = (((size_t)eye * p.height + ty * kTile + r) * p.width + tx * kTile) * 3 + c;
      out[o] = (&s_out[r][0][0])[c];
    }
  }
  if (t == 0) {
    atomicAdd(counters, s_eval);
    atomicAdd(counters + 1, (unsigned long long)staged);
  }
}

}  // namespace

cudaError_t launch_composite(const CompositeParams &p, const float *rec, int n,
                             const uint2 *ranges, const uint32_t *kept, const uint32_t *vals,
                             const float *gaze,
                             float *out, uint8_t *levels, float *t_final, uint32_t *n_contrib,
                             unsigned long long *counters, cudaStream_t s) {
  const int blocks = p.n_eyes * p.n_tiles;
  if (blocks <= 0) return cudaSuccess;
  if (t_final != nullptr)
    composite_kernel<true><<<blocks, kThreads, 0, s>>>(p, rec, n, ranges, kept, vals, gaze, out,
                                                       levels, t_final, n_contrib, counters);
  else
    composite_kernel<false><<<blocks, kThreads, 0, s>>>(p, rec, n, ranges, kept, vals, gaze, out,
                                                        levels, t_final, n_contrib, counters);
  return cudaGetLastError();
}

}  // namespace a3fr
