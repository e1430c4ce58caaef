// backward.cu -- gradients of the 3DGS forward pass (Sec. 2.3: projection, rasterization)
// with respect to the scene parameters, for a loss whose gradient with respect to the
// rendered image is given (L = sum(dl_drgb * image)).
//
// composite_backward: one CTA per 16 x 16 quadrant of an (eye, tile), one pixel per thread.  A pixel walks its
// tile's Gaussians back to front from its last contributor (n_contrib), recovering the
// transmittance before each contributor from the stored final one (T_before = T_after /
// (1 - alpha)) instead of storing it per Gaussian.  The colour accumulated behind a
// contributor enters the alpha gradient only through its dot product with dL/dC, so one
// scalar D carries it:  dL/dalpha_i = T_i (c_i . g - D_i),  D_{i-1} = alpha_i c_i . g +
// (1 - alpha_i) D_i.  Alpha is recomputed exactly as the forward computed it (shared
// helpers, explicitly rounded), so every skip / accept decision is the forward's.  The
// per-Gaussian partials (2-D mean, conic, opacity, colour) are summed over the warp and
// added to a per-(eye, Gaussian) buffer with one atomic per warp and value.  A foveated
// render's inherited pixels pass their gradient to the top-left pixel of their block.
//
// preprocess_backward: one thread per Gaussian, summing the eyes: conic -> 2-D covariance
// -> (3-D covariance, Jacobian) -> camera-space position -> mean; 3-D covariance ->
// scales (through exp) and rotation -> quaternion (through the normalisation); opacity
// through the sigmoid; colour -> SH coefficients and, through the view direction, mean.
#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kTile = 16;
constexpr int kThreads = 256;
constexpr int kG2 = 9;   // per (eye, Gaussian): du dv dconic_a dconic_b dconic_c dopacity dr dg db
constexpr int kPreBwdThreads = 128;

__global__ void __launch_bounds__(kThreads)
composite_backward_kernel(BackwardParams p, const float *__restrict__ rec, const uint2 *__restrict__ ranges,
                          const uint32_t *__restrict__ kept, const uint32_t *__restrict__ vals,
                          const uint8_t *__restrict__ levels, const float *__restrict__ t_final,
                          const uint32_t *__restrict__ n_contrib, const float *__restrict__ dl_drgb,
                          float *__restrict__ g2d) {
  __shared__ float4 s_geo[kThreads];   // u, v, A, B (base-2 falloff coefficients)
  __shared__ float4 s_cn[kThreads];    // C, conic a, conic b, conic c
  __shared__ float4 s_rgb[kThreads];   // r, g, b, opacity
  __shared__ uint32_t s_gid[kThreads];
  __shared__ uint32_t s_max[kThreads / 32];

  // one CTA per 16 x 16 quadrant of a tile (a 16-pixel tile is one quadrant, a 32-pixel tile
  // four, each walking the tile's whole list for its own pixels)
  const int qn = p.tile / kTile;
  const int gtile = blockIdx.x / (qn * qn);
  const int quad = blockIdx.x - gtile * qn * qn;
  const int eye = gtile / p.n_tiles;
  const int tile = gtile - eye * p.n_tiles;
  const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int px = tx * p.tile + (quad % qn) * kTile + (t & 15);
  const int py = ty * p.tile + (quad / qn) * kTile + (t >> 4);
  const bool inside = px < p.width && py < p.height;
  // labels of the 2x2 block: top-left 0, bottom-right 1, top-right 2, bottom-left 3
  const int bx = px & 1, by = py & 1;
  const int lab = bx == by ? (bx ? 1 : 0) : (bx ? 2 : 3);
  const int level = levels ? levels[gtile] : 4;
  const bool rendered = inside && lab < level;

  float T = 1.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
  uint32_t last = 0;
  if (rendered) {
    const size_t pix = ((size_t)eye * p.height + py) * p.width + px;
    T = t_final[pix];
    last = n_contrib[pix];
    g0 = dl_drgb[3 * pix];
    g1 = dl_drgb[3 * pix + 1];
    g2 = dl_drgb[3 * pix + 2];
    if (lab == 0 && level < 4) {
      // inherited pixels of the block copy this one: BR (label 2), TR (label 3), BL (label 4)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int dx = k < 2 ? 1 : 0, dy = k == 1 ? 0 : 1;
        if (level < k + 2 && px + dx < p.width && py + dy < p.height) {
          const size_t q = pix + (size_t)dy * p.width + dx;
          g0 += dl_drgb[3 * q];
          g1 += dl_drgb[3 * q + 1];
          g2 += dl_drgb[3 * q + 2];
        }
      }
    }
  }
  uint2 range = ranges[gtile];
  const uint32_t n_kept = *kept;
  range.x = min(range.x, n_kept);
  range.y = min(range.y, n_kept);
  last = min(last, range.y - range.x);

  // the block's deepest last contributor bounds the walk
  uint32_t m = last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s_max[warp] = m;
  __syncthreads();
  uint32_t max_last = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) max_last = max(max_last, s_max[w]);

  const float fpx = (float)px, fpy = (float)py;
  const float *rec_eye = rec + (size_t)eye * p.n * kRec;
  float *g_eye = g2d + (size_t)eye * p.n * kG2;
  float D = 0.0f;   // (colour accumulated behind, normalised by T) . dL/dC

  for (int hi = (int)max_last; hi >= 1; hi -= kThreads) {
    const int lo = max(1, hi - kThreads + 1);
    const int cnt = hi - lo + 1;
    __syncthreads();   // the previous batch is no longer read
    if (t < cnt) {
      const uint32_t pos = (uint32_t)(hi - t);   // 1-based position in the tile's list
      const uint32_t gidx = min(vals[range.x + pos - 1], (uint32_t)(p.n - 1));
      const float4 *r4 = reinterpret_cast<const float4 *>(rec_eye + (size_t)gidx * kRec);
      const float4 a = __ldg(r4), b = __ldg(r4 + 1), c = __ldg(r4 + 2);
      s_geo[t] = make_float4(a.x, a.y, __fmul_rn(-0.5f * kLog2e, a.z), __fmul_rn(-kLog2e, a.w));
      s_cn[t] = make_float4(__fmul_rn(-0.5f * kLog2e, b.x), a.z, a.w, b.x);
      s_rgb[t] = make_float4(b.z, b.w, c.x, b.y);
      s_gid[t] = gidx;
    }
    __syncthreads();
    for (int k = 0; k < cnt; ++k) {
      const uint32_t pos = (uint32_t)(hi - k);
      const float4 geo = s_geo[k];
      const float4 cn = s_cn[k];
      const float4 rgb = s_rgb[k];
      float vu = 0.f, vv = 0.f, va = 0.f, vb = 0.f, vc = 0.f, vo = 0.f, vr = 0.f, vg = 0.f, vbl = 0.f;
      bool ok = false;
      if (pos <= last) {
        const float dx = __fsub_rn(geo.x, fpx), dy = __fsub_rn(geo.y, fpy);
        const float pw = falloff_log2(geo.z, geo.w, cn.x, dx, dy);
        const float G = ex2_approx(pw);
        const float araw = __fmul_rn(rgb.w, G);
        const float alpha = fminf(0.99f, araw);
        ok = pw <= 0.0f && alpha >= 1.0f / 255.0f;
        if (ok) {
          const float om = __fsub_rn(1.0f, alpha);
          T = T / om;                              // transmittance in front of this Gaussian
          const float w = alpha * T;
          vr = w * g0;
          vg = w * g1;
          vbl = w * g2;
          const float cdot = rgb.x * g0 + rgb.y * g1 + rgb.z * g2;
          const float dalpha = T * (cdot - D);
          D = alpha * cdot + om * D;
          if (araw <= 0.99f) {                     // the 0.99 clamp passes no gradient
            const float dpow = dalpha * araw;      // d alpha / d power = opacity * exp(power)
            vo = dalpha * G;
            // power = -0.5 (a dx^2 + c dy^2) - b dx dy with dx = u - x, dy = v - y
            vu = -dpow * (cn.y * dx + cn.z * dy);
            vv = -dpow * (cn.w * dy + cn.z * dx);
            va = -0.5f * dpow * dx * dx;
            vb = -dpow * dx * dy;
            vc = -0.5f * dpow * dy * dy;
          }
        }
      }
      if (__ballot_sync(0xffffffffu, ok)) {
        // warp sums of the nine partials by recursive halving: at each of the first three
        // steps a lane keeps half of its values and sends the other half to its partner, so
        // the first eight cost 4 + 2 + 1 + 1 + 1 shuffles instead of 8 x 5; value j ends in
        // the lanes whose bits 4, 3, 2 spell j, and eight lanes add them to memory at once
        float h[8] = {vu, vv, va, vb, vc, vo, vr, vg};
        {
          const bool up = (lane & 16) != 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float keep = up ? h[j + 4] : h[j], send = up ? h[j] : h[j + 4];
            h[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
          }
        }
        {
          const bool up = (lane & 8) != 0;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const float keep = up ? h[j + 2] : h[j], send = up ? h[j] : h[j + 2];
            h[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
          }
        }
        {
          const bool up = (lane & 4) != 0;
          const float keep = up ? h[1] : h[0], send = up ? h[0] : h[1];
          h[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        h[0] += __shfl_xor_sync(0xffffffffu, h[0], 2);
        h[0] += __shfl_xor_sync(0xffffffffu, h[0], 1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vbl += __shfl_xor_sync(0xffffffffu, vbl, o);
        float *d = g_eye + (size_t)s_gid[k] * kG2;
        if ((lane & 3) == 0) {
          const int j = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
          atomicAdd(d + j, h[0]);
        }
        if (lane == 1) atomicAdd(d + 8, vbl);
      }
    }
  }
}

// Real SH basis (3DGS order and signs) at the unit direction (x, y, z) and its gradient
// contracted with per-coefficient weights wk: returns sum_k wk * dY_k/d(x, y, z).
template <int K>
__device__ __forceinline__ void sh_basis_eval(const ShConsts &c, float x, float y, float z, float *Y) {
  Y[0] = c.c0;
  if constexpr (K > 1) {
    Y[1] = -c.c1 * y;
    Y[2] = c.c1 * z;
    Y[3] = -c.c1 * x;
  }
  if constexpr (K > 4) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = c.c2a * x * y;
    Y[5] = -c.c2a * y * z;
    Y[6] = c.c2b * (2.0f * zz - xx - yy);
    Y[7] = -c.c2a * x * z;
    Y[8] = c.c2c * (xx - yy);
    if constexpr (K > 9) {
      Y[9] = -c.c3a * y * (3.0f * xx - yy);
      Y[10] = c.c3b * x * y * z;
      Y[11] = -c.c3c * y * (4.0f * zz - xx - yy);
      Y[12] = c.c3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
      Y[13] = -c.c3c * x * (4.0f * zz - xx - yy);
      Y[14] = c.c3e * z * (xx - yy);
      Y[15] = -c.c3a * x * (xx - 3.0f * yy);
    }
  }
}

template <int K>
__device__ __forceinline__ void sh_basis_vjp(const ShConsts &c, float x, float y, float z,
                                             const float *wk, float &gx, float &gy, float &gz) {
  gx = gy = gz = 0.0f;
  if constexpr (K > 1) {
    gy += -c.c1 * wk[1];
    gz += c.c1 * wk[2];
    gx += -c.c1 * wk[3];
  }
  if constexpr (K > 4) {
    // Y4 = c2a x y, Y5 = -c2a y z, Y6 = c2b (2zz - xx - yy), Y7 = -c2a x z, Y8 = c2c (xx - yy)
    gx += c.c2a * y * wk[4];
    gy += c.c2a * x * wk[4];
    gy += -c.c2a * z * wk[5];
    gz += -c.c2a * y * wk[5];
    gx += -2.0f * c.c2b * x * wk[6];
    gy += -2.0f * c.c2b * y * wk[6];
    gz += 4.0f * c.c2b * z * wk[6];
    gx += -c.c2a * z * wk[7];
    gz += -c.c2a * x * wk[7];
    gx += 2.0f * c.c2c * x * wk[8];
    gy += -2.0f * c.c2c * y * wk[8];
    if constexpr (K > 9) {
      const float xx = x * x, yy = y * y, zz = z * z;
      // Y9 = -c3a y (3xx - yy)
      gx += -6.0f * c.c3a * x * y * wk[9];
      gy += -3.0f * c.c3a * (xx - yy) * wk[9];
      // Y10 = c3b x y z
      gx += c.c3b * y * z * wk[10];
      gy += c.c3b * x * z * wk[10];
      gz += c.c3b * x * y * wk[10];
      // Y11 = -c3c y (4zz - xx - yy)
      gx += 2.0f * c.c3c * x * y * wk[11];
      gy += -c.c3c * (4.0f * zz - xx - 3.0f * yy) * wk[11];
      gz += -8.0f * c.c3c * y * z * wk[11];
      // Y12 = c3d z (2zz - 3xx - 3yy)
      gx += -6.0f * c.c3d * x * z * wk[12];
      gy += -6.0f * c.c3d * y * z * wk[12];
      gz += c.c3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * wk[12];
      // Y13 = -c3c x (4zz - xx - yy)
      gx += -c.c3c * (4.0f * zz - 3.0f * xx - yy) * wk[13];
      gy += 2.0f * c.c3c * x * y * wk[13];
      gz += -8.0f * c.c3c * x * z * wk[13];
      // Y14 = c3e z (xx - yy)
      gx += 2.0f * c.c3e * x * z * wk[14];
      gy += -2.0f * c.c3e * y * z * wk[14];
      gz += c.c3e * (xx - yy) * wk[14];
      // Y15 = -c3a x (xx - 3yy)
      gx += -3.0f * c.c3a * (xx - yy) * wk[15];
      gy += 6.0f * c.c3a * x * y * wk[15];
    }
  }
}

// Shared-memory row stride (floats) of a block's SH coefficients and their gradients: the
// 3K coefficients rounded up to an odd count, so the threads of a warp, reading the same
// coefficient of consecutive rows, hit distinct banks.
template <int K> constexpr int sh_stride() { return (3 * K) % 2 ? 3 * K : 3 * K + 1; }
template <int K> constexpr size_t backward_smem_bytes() {
  return 2 * sizeof(float) * (size_t)kPreBwdThreads * sh_stride<K>();
}

// One thread per Gaussian.  The block's SH coefficients are copied into shared memory with
// coalesced loads and their gradients accumulated there, then written back coalesced (read
// and accumulated per thread in global memory, the 48-float rows made every access a
// separate sector).
template <int K>
__global__ void __launch_bounds__(kPreBwdThreads)
preprocess_backward_kernel(const PreParams *__restrict__ pp, int n, const float *__restrict__ means,
                           const float *__restrict__ log_scales, const float *__restrict__ quats,
                           const float *__restrict__ opacity_logits, const float *__restrict__ sh,
                           const float *__restrict__ rec, const float *__restrict__ g2d,
                           float *__restrict__ d_means, float *__restrict__ d_log_scales,
                           float *__restrict__ d_quats, float *__restrict__ d_logits,
                           float *__restrict__ d_sh) {
  constexpr int SS = sh_stride<K>();
  constexpr int ROW = 3 * K;
  __shared__ PreParams s_p;
  extern __shared__ float s_sh_dyn[];
  float *s_coef = s_sh_dyn;                          // [kPreBwdThreads][SS]
  float *s_dsh = s_sh_dyn + kPreBwdThreads * SS;     // [kPreBwdThreads][SS]
  static_assert(sizeof(PreParams) % 4 == 0 && sizeof(PreParams) / 4 <= kPreBwdThreads, "PreParams copy");
  if (threadIdx.x < sizeof(PreParams) / 4)
    reinterpret_cast<uint32_t *>(&s_p)[threadIdx.x] = reinterpret_cast<const uint32_t *>(pp)[threadIdx.x];
  const int i0 = blockIdx.x * kPreBwdThreads;
  const int rows = min(kPreBwdThreads, n - i0);
  {
    const float *src = sh + (size_t)ROW * i0;
    for (int f = threadIdx.x; f < rows * ROW; f += kPreBwdThreads) {
      const int r = f / ROW, c = f - r * ROW;
      s_coef[r * SS + c] = src[f];
      s_dsh[r * SS + c] = 0.0f;
    }
  }
  __syncthreads();
  const PreParams &p = s_p;
  const int i = i0 + threadIdx.x;
  if (i < n) {

  const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
  float s2[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float s = expf(log_scales[3 * i + j]);
    s2[j] = s * s;
  }
  const float q0 = quats[4 * i], q1 = quats[4 * i + 1], q2 = quats[4 * i + 2], q3 = quats[4 * i + 3];
  const float qn = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  const float qw = q0 / qn, qx = q1 / qn, qy = q2 / qn, qz = q3 / qn;
  float R[3][3];
  R[0][0] = 1.0f - 2.0f * (qy * qy + qz * qz);
  R[0][1] = 2.0f * (qx * qy - qw * qz);
  R[0][2] = 2.0f * (qx * qz + qw * qy);
  R[1][0] = 2.0f * (qx * qy + qw * qz);
  R[1][1] = 1.0f - 2.0f * (qx * qx + qz * qz);
  R[1][2] = 2.0f * (qy * qz - qw * qx);
  R[2][0] = 2.0f * (qx * qz - qw * qy);
  R[2][1] = 2.0f * (qy * qz + qw * qx);
  R[2][2] = 1.0f - 2.0f * (qx * qx + qy * qy);
  float S[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      S[j][k] = R[j][0] * s2[0] * R[k][0] + R[j][1] * s2[1] * R[k][1] + R[j][2] * s2[2] * R[k][2];
  const float opacity = 1.0f / (1.0f + expf(-opacity_logits[i]));
  const float *coef = s_coef + threadIdx.x * SS;

  float dmu[3] = {0.f, 0.f, 0.f};
  float dS[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  float dlogit = 0.0f;
  float *dsh = s_dsh + threadIdx.x * SS;

  for (int e = 0; e < p.n_eyes; ++e) {
    if (rec[((size_t)e * n + i) * kRec + 11] == 0.0f) continue;   // culled for this eye
    const float *g = g2d + ((size_t)e * n + i) * kG2;
    const float gu = g[0], gv = g[1], gca = g[2], gcb = g[3], gcc = g[4], gop = g[5];
    const float gr[3] = {g[6], g[7], g[8]};
    const CamParams &c = p.cam[e];
    const float *W = c.R;
    const float tx = W[0] * mx + W[1] * my + W[2] * mz + c.t[0];
    const float ty = W[3] * mx + W[4] * my + W[5] * mz + c.t[1];
    const float tz = W[6] * mx + W[7] * my + W[8] * mz + c.t[2];
    const float txz = tx / tz, tyz = ty / tz;
    const bool clx = txz < -c.limx || txz > c.limx;
    const bool cly = tyz < -c.limy || tyz > c.limy;
    const float xc = fminf(c.limx, fmaxf(-c.limx, txz)) * tz;
    const float yc = fminf(c.limy, fmaxf(-c.limy, tyz)) * tz;
    const float tz2 = tz * tz;
    const float J00 = c.fx / tz, J02 = -c.fx * xc / tz2;
    const float J11 = c.fy / tz, J12 = -c.fy * yc / tz2;
    float T[2][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T[0][j] = J00 * W[j] + J02 * W[6 + j];
      T[1][j] = J11 * W[3 + j] + J12 * W[6 + j];
    }
    float U[2][3];   // T Sigma
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int l = 0; l < 3; ++l) U[r][l] = T[r][0] * S[0][l] + T[r][1] * S[1][l] + T[r][2] * S[2][l];
    const float a = U[0][0] * T[0][0] + U[0][1] * T[0][1] + U[0][2] * T[0][2] + 0.3f;
    const float b = U[0][0] * T[1][0] + U[0][1] * T[1][1] + U[0][2] * T[1][2];
    const float cc = U[1][0] * T[1][0] + U[1][1] * T[1][1] + U[1][2] * T[1][2] + 0.3f;
    const float det = a * cc - b * b;
    const float id2 = 1.0f / (det * det);
    // conic (cc, -b, a) / det -> covariance entries
    const float ga = (-cc * cc * gca + b * cc * gcb - b * b * gcc) * id2;
    const float gb = (2.0f * b * cc * gca - (a * cc + b * b) * gcb + 2.0f * a * b * gcc) * id2;
    const float gc = (-b * b * gca + a * b * gcb - a * a * gcc) * id2;
    // cov = T Sigma T^T with G2 = [[ga, gb/2], [gb/2, gc]]: dSigma += T^T G2 T, dT = 2 G2 T Sigma
    const float G2[2][2] = {{ga, 0.5f * gb}, {0.5f * gb, gc}};
    float GT[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int j = 0; j < 3; ++j) GT[r][j] = G2[r][0] * T[0][j] + G2[r][1] * T[1][j];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) dS[j][k] += T[0][j] * GT[0][k] + T[1][j] * GT[1][k];
    float dT[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dT[r][j] = 2.0f * (G2[r][0] * U[0][j] + G2[r][1] * U[1][j]);
    // T = J W
    float dJ00 = 0.f, dJ02 = 0.f, dJ11 = 0.f, dJ12 = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dJ00 += dT[0][j] * W[j];
      dJ02 += dT[0][j] * W[6 + j];
      dJ11 += dT[1][j] * W[3 + j];
      dJ12 += dT[1][j] * W[6 + j];
    }
    float dtx = 0.f, dty = 0.f, dtz = 0.f;
    dtz += -c.fx / tz2 * dJ00 - c.fy / tz2 * dJ11;
    // J02 = -fx x' / tz^2 with x' = tx (inside the clamp) or +-limx tz (outside)
    if (!clx) {
      dtx += -c.fx / tz2 * dJ02;
      dtz += 2.0f * c.fx * tx / (tz2 * tz) * dJ02;
    } else {
      dtz += c.fx * (xc / tz) / tz2 * dJ02;
    }
    if (!cly) {
      dty += -c.fy / tz2 * dJ12;
      dtz += 2.0f * c.fy * ty / (tz2 * tz) * dJ12;
    } else {
      dtz += c.fy * (yc / tz) / tz2 * dJ12;
    }
    // u = fx tx / tz + cx, v = fy ty / tz + cy
    dtx += c.fx / tz * gu;
    dty += c.fy / tz * gv;
    dtz += -c.fx * tx / tz2 * gu - c.fy * ty / tz2 * gv;
    // t = W mu + t_c
#pragma unroll
    for (int j = 0; j < 3; ++j) dmu[j] += W[j] * dtx + W[3 + j] * dty + W[6 + j] * dtz;
    // opacity
    dlogit += gop * opacity * (1.0f - opacity);
    // colour: the unit direction from the eye centre -W^T t_c to the mean
    float C[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) C[j] = -(W[j] * c.t[0] + W[3 + j] * c.t[1] + W[6 + j] * c.t[2]);
    const float ddx = mx - C[0], ddy = my - C[1], ddz = mz - C[2];
    const float dn = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
    const float x = ddx / dn, y = ddy / dn, z = ddz / dn;
    float Y[K];
    sh_basis_eval<K>(p.shc, x, y, z, Y);
    float gch[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float acc = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) acc += Y[k] * coef[3 * k + ch];
      gch[ch] = acc > 0.0f ? gr[ch] : 0.0f;   // max(0, .) passes gradient where positive
    }
    float wk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      wk[k] = coef[3 * k] * gch[0] + coef[3 * k + 1] * gch[1] + coef[3 * k + 2] * gch[2];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) dsh[3 * k + ch] += Y[k] * gch[ch];
    }
    float gx, gy, gz;
    sh_basis_vjp<K>(p.shc, x, y, z, wk, gx, gy, gz);
    const float dot = x * gx + y * gy + z * gz;
    dmu[0] += (gx - x * dot) / dn;
    dmu[1] += (gy - y * dot) / dn;
    dmu[2] += (gz - z * dot) / dn;
  }
  // Sigma = R diag(s2) R^T (dS symmetric): ds2_k = (R^T dS R)_kk, dR = 2 dS R diag(s2)
  float dR[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dR[j][k] = 2.0f * (dS[j][0] * R[0][k] + dS[j][1] * R[1][k] + dS[j][2] * R[2][k]) * s2[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float v = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      v += R[j][k] * (dS[j][0] * R[0][k] + dS[j][1] * R[1][k] + dS[j][2] * R[2][k]);
    d_log_scales[3 * i + k] = 2.0f * s2[k] * v;   // s2 = exp(2 log s)
  }
  // R of the unit quaternion (w, x, y, z)
  const float dw = 2.0f * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] -
                           qy * dR[2][0] + qx * dR[2][1]);
  const float dx = 2.0f * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - 2.0f * qx * dR[1][1] -
                           qw * dR[1][2] + qz * dR[2][0] + qw * dR[2][1] - 2.0f * qx * dR[2][2]);
  const float dy = 2.0f * (-2.0f * qy * dR[0][0] + qx * dR[0][1] + qw * dR[0][2] + qx * dR[1][0] +
                           qz * dR[1][2] - qw * dR[2][0] + qz * dR[2][1] - 2.0f * qy * dR[2][2]);
  const float dz = 2.0f * (-2.0f * qz * dR[0][0] - qw * dR[0][1] + qx * dR[0][2] + qw * dR[1][0] -
                           2.0f * qz * dR[1][1] + qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
  // through q / |q|
  const float qd = qw * dw + qx * dx + qy * dy + qz * dz;
  d_quats[4 * i] = (dw - qw * qd) / qn;
  d_quats[4 * i + 1] = (dx - qx * qd) / qn;
  d_quats[4 * i + 2] = (dy - qy * qd) / qn;
  d_quats[4 * i + 3] = (dz - qz * qd) / qn;
  d_means[3 * i] = dmu[0];
  d_means[3 * i + 1] = dmu[1];
  d_means[3 * i + 2] = dmu[2];
  d_logits[i] = dlogit;
  }
  __syncthreads();
  float *dst = d_sh + (size_t)ROW * i0;
  for (int f = threadIdx.x; f < rows * ROW; f += kPreBwdThreads) {
    const int r = f / ROW, c = f - r * ROW;
    dst[f] = s_dsh[r * SS + c];
  }
}

}  // namespace

size_t backward_g2d_floats(int n_eyes, int n) { return (size_t)n_eyes * n * kG2; }

cudaError_t launch_backward(const BackwardParams &bp, const PreParams *pre_dev, int sh_degree,
                            const float *means, const float *log_scales, const float *quats,
                            const float *opacity_logits, const float *sh, const float *rec,
                            const uint2 *ranges, const uint32_t *kept, const uint32_t *vals,
                            const uint8_t *levels, const float *t_final, const uint32_t *n_contrib,
                            const float *dl_drgb, float *g2d, float *d_means, float *d_log_scales,
                            float *d_quats, float *d_logits, float *d_sh, cudaStream_t s) {
  if (bp.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(g2d, 0, sizeof(float) * backward_g2d_floats(bp.n_eyes, bp.n), s);
  if (e != cudaSuccess) return e;
  const int quads = (bp.tile / kTile) * (bp.tile / kTile);
  composite_backward_kernel<<<bp.n_eyes * bp.n_tiles * quads, kThreads, 0, s>>>(
      bp, rec, ranges, kept, vals, levels, t_final, n_contrib, dl_drgb, g2d);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int blocks = (bp.n + kPreBwdThreads - 1) / kPreBwdThreads;
  auto go = [&](auto kern, size_t smem) -> cudaError_t {
    // per device: the attribute lives in each device's context
    cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e2 != cudaSuccess) return e2;
    kern<<<blocks, kPreBwdThreads, smem, s>>>(pre_dev, bp.n, means, log_scales, quats, opacity_logits,
                                               sh, rec, g2d, d_means, d_log_scales, d_quats, d_logits,
                                               d_sh);
    return cudaGetLastError();
  };
  switch (sh_degree) {
    case 0: return go(preprocess_backward_kernel<1>, backward_smem_bytes<1>());
    case 1: return go(preprocess_backward_kernel<4>, backward_smem_bytes<4>());
    case 2: return go(preprocess_backward_kernel<9>, backward_smem_bytes<9>());
    default: return go(preprocess_backward_kernel<16>, backward_smem_bytes<16>());
  }
}

}  // namespace a3fr
