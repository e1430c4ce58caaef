// cnn.cu -- tensor-core (tcgen05) kernels of the learned periphery: small CNNs in BF16 with
// FP32 accumulation that reconstruct full-resolution RGB from the quarter-density peripheral
// layer (the level-1 pixels of Sec. 3.4) and its depth -- a residual network of ten 3x3
// convolutions, and a compact one (a 3x3 convolution and two per-block layers) whose whole
// fill is one fused kernel.
//
// This file starts with the single-tile GEMM that validates the operand encodings (shared-
// memory descriptors, instruction descriptor, tensor-memory round trip) before the
// convolution kernels use them.
#include "../../include/a3fr.h"
#include "common.cuh"
#include <cuda_bf16.h>

#include <cmath>
#include <new>

#include "tc.cuh"

namespace a3fr {
namespace {

constexpr int kProbeSmem = 96 * 1024;
constexpr int kProbeB = 48 * 1024;   // offset of the B tile

// D[128][N] = A[128][K] B[N][K]^T for one tile.  variant 0: leading byte offset = distance
// of K-adjacent core matrices, stride byte offset = distance of M/N-adjacent ones; variant
// 1: the two swapped.  Either way every address the tensor core can form stays inside the
// zeroed 96 KB of shared memory.
__global__ void __launch_bounds__(128)
tc_tile_gemm_kernel(const uint16_t *__restrict__ A, const uint16_t *__restrict__ B,
                    float *__restrict__ D, int N, int K, int variant, uint32_t *__restrict__ status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int i = t; i < kProbeSmem / 16; i += 128) reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(&s_tmem, 256);
  __syncthreads();
  const uint32_t sbo = (uint32_t)(K / 8) * 128u;   // a row group holds K/8 core matrices
  for (int idx = t; idx < 128 * K; idx += 128) {
    const int m = idx / K, k = idx - m * K;
    const uint32_t off = (m >> 3) * sbo + (k >> 3) * 128u + (m & 7) * 16u + (k & 7) * 2u;
    *reinterpret_cast<uint16_t *>(smem + off) = A[idx];
  }
  for (int idx = t; idx < N * K; idx += 128) {
    const int nn = idx / K, k = idx - nn * K;
    const uint32_t off = (nn >> 3) * sbo + (k >> 3) * 128u + (nn & 7) * 16u + (k & 7) * 2u;
    *reinterpret_cast<uint16_t *>(smem + kProbeB + off) = B[idx];
  }
  tc::fence_proxy_async();
  if (t == 0) tc::mbar_init(&s_bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  if (t == 0) {
    const uint32_t a0 = tc::smem_u32(smem), b0 = tc::smem_u32(smem + kProbeB);
    const uint32_t idesc = tc::idesc_bf16_f32(128, N);
    for (int kk = 0; kk < K / 16; ++kk) {
      const uint32_t lbo = variant == 0 ? 128u : sbo, s2 = variant == 0 ? sbo : 128u;
      const uint64_t ad = tc::smem_desc(a0 + kk * 256u, lbo, s2);
      const uint64_t bd = tc::smem_desc(b0 + kk * 256u, lbo, s2);
      tc::mma_bf16(tmem, ad, bd, idesc, kk > 0);
    }
    tc::mma_commit(&s_bar);
  }
  const bool ok = tc::mbar_wait(&s_bar, 0);
  if (!ok && lane == 0) atomicOr(status, kStatusTimeout);
  tc::fence_after_sync();
  float v[32];
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
  if (N == 32) tc::tmem_ld32(taddr, v);
  else tc::tmem_ld16(taddr, v);
  const int row = warp * 32 + lane;
  for (int nn = 0; nn < N; ++nn) D[row * N + nn] = v[nn];
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}


// ---------------------------------------------------------------- convolution kernels
// Activations are NHWC BF16 with 16 or 32 channels (32 or 64 bytes per pixel); a 3x3 "same"
// convolution is an implicit GEMM  D[pixel][cout] = sum over (tap, cin) of X[pixel + tap][cin]
// W[cout][cin][tap].  The A operand is never expanded: the tile's input halo sits in shared
// memory as [channel group of 8][row][column][8 channels], which is exactly the K-major core-
// matrix layout (8 pixels x 16 bytes) with the column direction inside a core matrix, so the
// operand of tap (ky, kx) is the same halo seen from a start address shifted by ky rows and kx
// columns.  Weights come pre-packed as [tap][cin group][cout][8 cin].

constexpr int kConvTW = 8;    // output tile width (pixels)
constexpr int kConvTH = 16;   // output tile height: 128 pixels = the MMA's M

struct ConvDims {
  int B, H, W;
};

enum : int { kEpiBias = 1, kEpiRelu = 2, kEpiResid = 4, kEpiMask = 8, kEpiF32 = 16 };

// Halo rows x cols of 8-channel groups around the tile whose top-left output pixel is (y0, x0).
template <int CG>
__device__ __forceinline__ void load_halo(uint8_t *hs, const __nv_bfloat16 *__restrict__ X, int b,
                                          int y0, int x0, int rows, int cols, int H, int W) {
  const int total = rows * cols * CG;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int cg = i % CG, rc = i / CG;
    const int c = rc % cols, r = rc / cols;
    const int y = y0 - 1 + r, x = x0 - 1 + c;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (y >= 0 && y < H && x >= 0 && x < W)
      v = __ldg(reinterpret_cast<const uint4 *>(X + (((size_t)b * H + y) * W + x) * (CG * 8)) + cg);
    *reinterpret_cast<uint4 *>(hs + ((size_t)(cg * rows + r) * cols + c) * 16) = v;
  }
}

// The same halo with asynchronous 16-byte copies (zero-filled outside the image); the caller
// waits with cp_async_wait_all() before the data is used.
template <int CG>
__device__ __forceinline__ void load_halo_async(uint8_t *hs, const __nv_bfloat16 *__restrict__ X, int b,
                                                int y0, int x0, int rows, int cols, int H, int W) {
  const int total = rows * cols * CG;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int cg = i % CG, rc = i / CG;
    const int c = rc % cols, r = rc / cols;
    const int y = y0 - 1 + r, x = x0 - 1 + c;
    const bool in = y >= 0 && y < H && x >= 0 && x < W;
    const __nv_bfloat16 *src = in ? X + (((size_t)b * H + y) * W + x) * (CG * 8) + cg * 8 : X;
    const uint32_t dst = tc::smem_u32(hs + ((size_t)(cg * rows + r) * cols + c) * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The image side of the learned fill, for the two convolutions that touch it when the fill
// runs fused: the first reads its input straight from the render (kSrcImage), the last
// composes the skipped pixels in its epilogue (kDstCompose) -- the same values the separate
// gather and compose kernels produce, without their intermediate tensors.
struct FillIO {
  const float *depth;     // [B][H][W] expected depth of the render
  float *img;             // [B][H][W][3]: top-left pixels read, skipped pixels written
  const uint8_t *levels;  // tile levels [B][n_tiles]
  int H, W, tile, tiles_x, n_tiles;
};
enum : int { kSrcTensor = 0, kSrcImage = 1 };
enum : int { kDstTensor = 0, kDstCompose = 1 };

// The 16 input channels of block (y2, x2): r, g, b of its top-left pixel and depth / 8 in
// BF16, then zeros (the first eight as one 16-byte group; the second group is all zero).
__device__ __forceinline__ uint4 block_input(const float *__restrict__ img, const float *__restrict__ depth,
                                             int b, int H, int W, int y2, int x2) {
  const size_t src = ((size_t)b * H + 2 * y2) * W + 2 * x2;
  uint4 lo;
  __nv_bfloat162 *l2 = reinterpret_cast<__nv_bfloat162 *>(&lo);
  l2[0] = __floats2bfloat162_rn(img[3 * src], img[3 * src + 1]);
  l2[1] = __floats2bfloat162_rn(img[3 * src + 2], depth[src] * 0.125f);
  l2[2] = __floats2bfloat162_rn(0.0f, 0.0f);
  l2[3] = l2[2];
  return lo;
}

// Final image of a foveated render at block (y2, x2) from its 12 residuals res[c][2 dy + dx]:
// rendered pixels kept, the skipped sub-pixels -- top-right (label 3), bottom-left (4),
// bottom-right (2) -- set to the bilinear base of the blocks' top-left pixels (the last block
// repeated past the edge) plus the residual.  The base reads only top-left pixels, which every
// level renders and nobody writes.
__device__ __forceinline__ void compose_block(float *__restrict__ img, int b, int H, int W, int y2, int x2, int lv,
                                              const float (&res)[3][4]) {
  const int H2 = (H + 1) / 2, W2 = (W + 1) / 2;
  const int x = 2 * x2, y = 2 * y2;
  const int xr = min(x2 + 1, W2 - 1), yd = min(y2 + 1, H2 - 1);
  auto tl = [&](int yy, int xx, int c) { return img[3 * (((size_t)b * H + 2 * yy) * W + 2 * xx) + c]; };
  float a[3], right[3], down[3], diag[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a[c] = tl(y2, x2, c);
    right[c] = tl(y2, xr, c);
    down[c] = lv <= 3 ? tl(yd, x2, c) : 0.0f;
    diag[c] = lv <= 1 ? tl(yd, xr, c) : 0.0f;
  }
  auto put = [&](int dy, int dx, const float *base) {
    if (y + dy >= H || x + dx >= W) return;
    float *o = img + 3 * (((size_t)b * H + y + dy) * W + x + dx);
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = base[c] + res[c][2 * dy + dx];
  };
  float bt[3], bb[3], bd[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bt[c] = __fmul_rn(__fadd_rn(a[c], right[c]), 0.5f);                                   // top-right
    bb[c] = __fmul_rn(__fadd_rn(a[c], down[c]), 0.5f);                                    // bottom-left
    bd[c] = __fmul_rn(__fadd_rn(__fadd_rn(__fadd_rn(a[c], right[c]), down[c]), diag[c]), 0.25f);   // bottom-right
  }
  if (lv <= 2) put(0, 1, bt);   // top-right: label 3, rendered from level 3
  if (lv <= 3) put(1, 0, bb);   // bottom-left: label 4, rendered at level 4
  if (lv <= 1) put(1, 1, bd);   // bottom-right: label 2, rendered from level 2
}

template <int CIN, int COUT>
constexpr int conv_smem_bytes() {
  return 2 * (CIN / 8) * (kConvTH + 2) * (kConvTW + 2) * 16 + 9 * (CIN / 8) * COUT * 16;
}

// Persistent over 8 x 16 output tiles (128 threads: one per output pixel in the epilogue).  A
// CTA loads the layer's packed weights once, then walks tiles blockIdx.x, + gridDim.x, ...
// with a two-deep pipeline: two halo buffers in shared memory and two 32-column accumulators
// in tensor memory, so the halo of tile k+1 loads while tile k's MMAs run, and tile k's
// epilogue (tensor-memory read, bias, ReLU, residual, mask, store) runs while tile k+1's MMAs
// do.  One thread issues the 9 x (CIN/16) MMAs of a tile and commits them to the mbarrier;
// tile k completes phase k.
//
// kSrcImage (16 input channels): the halo is formed from the render (block_input) instead of
// copied from a tensor -- its loads issued before tile k's epilogue, stored to shared memory
// after it.  kDstCompose (16 output channels): the epilogue composes the block's skipped
// pixels into the image (compose_block) instead of storing the residuals.
template <int CIN, int COUT, int SRC = kSrcTensor, int DST = kDstTensor>
__global__ void __launch_bounds__(128)
conv3x3_tc_kernel(ConvDims d, const __nv_bfloat16 *__restrict__ X, const uint4 *__restrict__ Wpk,
                  const float *__restrict__ bias, const __nv_bfloat16 *__restrict__ R,
                  const __nv_bfloat16 *__restrict__ Mk, void *__restrict__ Y, int flags,
                  uint32_t *__restrict__ status, FillIO io) {
  static_assert(SRC == kSrcTensor || CIN == 16, "the image input has 16 channels");
  static_assert(DST == kDstTensor || COUT == 16, "the composed residuals have 16 channels");
  constexpr int CG = CIN / 8, HR = kConvTH + 2, HC = kConvTW + 2;
  constexpr int HALO = CG * HR * HC * 16, WBYTES = 9 * CG * COUT * 16;
  constexpr int kGPer = (HR * HC + 127) / 128;   // halo pixels per thread (image input)
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *const ws = smem + 2 * HALO;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ float s_bias[32];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t < COUT) s_bias[t] = (flags & kEpiBias) ? bias[t] : 0.0f;
  const int tiles_x = (d.W + kConvTW - 1) / kConvTW, tiles_y = (d.H + kConvTH - 1) / kConvTH;
  const int n_tiles = d.B * tiles_x * tiles_y;
  const int my_n = (int)blockIdx.x < n_tiles ? (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  auto origin = [&](int k, int &b, int &y0, int &x0) {
    const int tt = (int)blockIdx.x + k * (int)gridDim.x;
    x0 = (tt % tiles_x) * kConvTW;
    const int r = tt / tiles_x;
    y0 = (r % tiles_y) * kConvTH;
    b = r / tiles_y;
  };
  // image input: the halo pixels of a tile, loaded into registers, then stored as BF16 groups
  // (the second 8-channel group stays zero: it is cleared once here)
  uint4 gv[kGPer];
  auto gather_load = [&](int k) {
    int b, y0, x0;
    origin(k, b, y0, x0);
#pragma unroll
    for (int j = 0; j < kGPer; ++j) {
      const int q = t + 128 * j, r = q / HC, c = q - r * HC;
      const int y = y0 - 1 + r, x = x0 - 1 + c;
      gv[j] = make_uint4(0u, 0u, 0u, 0u);
      if (q < HR * HC && y >= 0 && y < d.H && x >= 0 && x < d.W)
        gv[j] = block_input(io.img, io.depth, b, io.H, io.W, y, x);
    }
  };
  auto gather_store = [&](uint8_t *hs) {
#pragma unroll
    for (int j = 0; j < kGPer; ++j) {
      const int q = t + 128 * j;
      if (q < HR * HC) *reinterpret_cast<uint4 *>(hs + (size_t)q * 16) = gv[j];
    }
  };
  if (warp == 0) tc::tmem_alloc(&s_tmem, 64);
  for (int i = t; i < WBYTES / 16; i += 128) reinterpret_cast<uint4 *>(ws)[i] = __ldg(Wpk + i);
  if constexpr (SRC == kSrcImage) {
    for (int i = t; i < 2 * HR * HC; i += 128) {   // group 1 of both halo buffers
      const int buf = i / (HR * HC), q = i - buf * (HR * HC);
      *reinterpret_cast<uint4 *>(smem + buf * HALO + (size_t)(HR * HC + q) * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (my_n > 0) {
      gather_load(0);
      gather_store(smem);
    }
  } else if (my_n > 0) {
    int b, y0, x0;
    origin(0, b, y0, x0);
    load_halo_async<CG>(smem, X, b, y0, x0, HR, HC, d.H, d.W);
  }
  cp_async_wait_all();
  tc::fence_proxy_async();
  if (t == 0) tc::mbar_init(&s_bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
  auto issue = [&](int k) {   // MMAs of tile k: halo buffer k & 1, accumulator columns 32 (k & 1)
    const uint32_t h0 = tc::smem_u32(smem + (k & 1) * HALO), w0 = tc::smem_u32(ws);
    const uint32_t dt = tmem + (uint32_t)((k & 1) * 32);
    int n = 0;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
      for (int cb = 0; cb < CIN / 16; ++cb) {
        const uint64_t a = tc::smem_desc(h0 + (2 * cb) * (HR * HC * 16) + ky * (HC * 16) + kx * 16,
                                         HR * HC * 16, HC * 16);
        const uint64_t w = tc::smem_desc(w0 + tap * (CG * COUT * 16) + (2 * cb) * (COUT * 16), COUT * 16, 128);
        tc::mma_bf16(dt, a, w, idesc, n > 0);
        ++n;
      }
    }
    tc::mma_commit(&s_bar);
  };
  if (t == 0 && my_n > 0) issue(0);
  if (my_n > 1) {   // buffer 1 is free: start tile 1's halo
    if constexpr (SRC == kSrcImage) {
      gather_load(1);
      gather_store(smem + HALO);
    } else {
      int b, y0, x0;
      origin(1, b, y0, x0);
      load_halo_async<CG>(smem + HALO, X, b, y0, x0, HR, HC, d.H, d.W);
    }
  }
  for (int k = 0; k < my_n; ++k) {
    int b, y0, x0;
    origin(k, b, y0, x0);
    const int m = warp * 32 + lane;
    const int y = y0 + m / kConvTW, x = x0 + (m % kConvTW);
    const bool inside = y < d.H && x < d.W;
    const size_t pix = inside ? ((size_t)b * d.H + y) * d.W + x : 0;
    // the epilogue's residual input, loaded now so that its latency overlaps the waits for this
    // tile's MMAs and the next halo
    uint4 rv[COUT / 8];
#pragma unroll
    for (int g = 0; g < COUT / 8; ++g)
      rv[g] = (inside && (flags & kEpiResid)) ? __ldg(reinterpret_cast<const uint4 *>(R + pix * COUT) + g)
                                              : make_uint4(0u, 0u, 0u, 0u);
    if (!tc::mbar_wait(&s_bar, (uint32_t)(k & 1)) && lane == 0) atomicOr(status, kStatusTimeout);
    cp_async_wait_all();   // halo k + 1 has landed
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();   // halo k + 1 complete everywhere; every thread saw tile k complete
    tc::fence_after_sync();
    if (t == 0 && k + 1 < my_n) issue(k + 1);
    if (k + 2 < my_n) {   // buffer k & 1 was read by tile k, which completed
      if constexpr (SRC == kSrcImage) {
        gather_load(k + 2);   // stored after this tile's epilogue
      } else {
        int b, y0, x0;
        origin(k + 2, b, y0, x0);
        load_halo_async<CG>(smem + (k & 1) * HALO, X, b, y0, x0, HR, HC, d.H, d.W);
      }
    }
    // epilogue of tile k
    float v[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((k & 1) * 32);
    if (COUT == 32) tc::tmem_ld32(taddr, v);
    else tc::tmem_ld16(taddr, v);
    if constexpr (DST == kDstCompose) {
      if (inside) {
        const int lv = io.levels[b * io.n_tiles + ((2 * y) / io.tile) * io.tiles_x + (2 * x) / io.tile];
        if (lv < 4) {   // else every pixel of the block was rendered
          // residual of colour c, sub-pixel s = 2 dy + dx: channel 4 c + s (12..15 unused)
          float res[3][4];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 4; ++q) res[c][q] = v[4 * c + q] + s_bias[4 * c + q];
          compose_block(io.img, b, io.H, io.W, y, x, lv, res);
        }
      }
    } else if (inside) {
#pragma unroll
      for (int g = 0; g < COUT / 8; ++g) {
        float o[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          o[c] = v[g * 8 + c] + s_bias[g * 8 + c];
          if (flags & kEpiRelu) o[c] = fmaxf(o[c], 0.0f);
        }
        if (flags & kEpiResid) {
          const __nv_bfloat16 *rb = reinterpret_cast<const __nv_bfloat16 *>(&rv[g]);
#pragma unroll
          for (int c = 0; c < 8; ++c) o[c] += __bfloat162float(rb[c]);
        }
        if (flags & kEpiMask) {
          const uint4 mv = __ldg(reinterpret_cast<const uint4 *>(Mk + pix * COUT) + g);
          const __nv_bfloat16 *mb = reinterpret_cast<const __nv_bfloat16 *>(&mv);
#pragma unroll
          for (int c = 0; c < 8; ++c) o[c] = __bfloat162float(mb[c]) > 0.0f ? o[c] : 0.0f;
        }
        if (flags & kEpiF32) {
          float4 *yo = reinterpret_cast<float4 *>(static_cast<float *>(Y) + pix * COUT + g * 8);
          yo[0] = make_float4(o[0], o[1], o[2], o[3]);
          yo[1] = make_float4(o[4], o[5], o[6], o[7]);
        } else {
          uint4 pk;
          __nv_bfloat162 *p2 = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
          for (int c = 0; c < 4; ++c) p2[c] = __floats2bfloat162_rn(o[2 * c], o[2 * c + 1]);
          reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(Y) + pix * COUT)[g] = pk;
        }
      }
    }
    if constexpr (SRC == kSrcImage) {
      if (k + 2 < my_n) gather_store(smem + (k & 1) * HALO);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// The compact network's whole fill in one persistent kernel, per 16 x 16 block tile made of two
// halves of 8 x 16 blocks side by side, each half one MMA of M = 128 rows (row m of half h =
// block (y0 + m / 8, x0 + 8 h + m % 8)); thread t holds row t of both halves in the epilogues:
//   layer 0: the 3x3 convolution 16 -> 32 on the tile's 18 x 18 input halo, formed from the
//            render: per half 9 MMAs, N 32, K 16;
//   layer 1: the per-block layer 32 -> 32: per half 2 MMAs (K 32);
//   layer 2: the per-block layer 32 -> 16: per half 2 MMAs, the epilogue composing the block's
//            skipped pixels.
// The halo sits in shared memory as [row][column][8 channels] (16 bytes per block): a half's A
// operand for tap (ky, kx) starts ky rows, kx + 8 h columns in, its core matrices (8 blocks of
// one row) one halo row apart (SBO).  Input channels 8..15 are zero: the MMA's second K group
// reads the first group's blocks again (leading byte offset 0) against a zero block of weights,
// so those products are exactly zero.  The epilogues of layers 0 and 1 read the accumulators
// from tensor memory, add the bias, apply the ReLU, round to BF16 and write the next layer's A
// operands to shared memory as [half][K group of 8][row][8 channels] -- K-major core matrices,
// rows 16 bytes apart (SBO 128), K groups 2,048 bytes apart (LBO) -- so no activation leaves
// the SM.  The per-block layers' weights are the centre taps of their 3x3 packs.  The halo's
// FP32 colours stay beside it, so the compose step reads its top-left pixels in shared memory.
// The three layers of a tile reuse two 32-column accumulators (one per half); the CTAs sharing
// an SM overlap one another's serial chains, and the next tile's halo and levels load into
// registers while this tile's layers run.  Tiles whose blocks are all fully rendered (level 4)
// skip the network.
constexpr int kCmpTW = 2 * kConvTW, kCmpTH = kConvTH;   // 16 x 16 blocks
constexpr int kCmpHR = kCmpTH + 2, kCmpHC = kCmpTW + 2;
constexpr int kCmpHalo = kCmpHR * kCmpHC * 16;       // input group 0 (BF16) per halo block
constexpr int kCmpRgb = kCmpHR * kCmpHC * 16;        // FP32 r, g, b (and a pad) per halo block
constexpr int kCmpW0 = 9 * 32 * 16;                  // [tap][cout][8 cin] of input group 0
constexpr int kCmpZero = 32 * 16;                    // zero weights of input group 1
constexpr int kCmpW1 = 4 * 32 * 16;                  // [cin group][cout][8 cin]
constexpr int kCmpW2 = 4 * 16 * 16;
constexpr int kCmpAct = 2 * 4 * 128 * 16;            // [half][K group][row][8]
constexpr int kCmpSmem = kCmpHalo + kCmpRgb + kCmpW0 + kCmpZero + kCmpW1 + kCmpW2 + kCmpAct;
constexpr int kCmpCtas = 6;                          // CTAs per SM
static_assert(kCmpHalo % 16 == 0 && kCmpRgb % 16 == 0 && kCmpW0 % 16 == 0 && kCmpZero % 16 == 0 &&
              kCmpW1 % 16 == 0 && kCmpW2 % 16 == 0, "operands start on 16-byte boundaries");

__global__ void __launch_bounds__(128, kCmpCtas)
compact_fill_tc_kernel(ConvDims d, const uint4 *__restrict__ W0, const uint4 *__restrict__ W1,
                       const uint4 *__restrict__ W2, const float *__restrict__ bias,
                       uint32_t *__restrict__ status, FillIO io) {
  constexpr int HR = kCmpHR, HC = kCmpHC;
  constexpr int kGPer = (HR * HC + 127) / 128;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *const halo = smem;
  float4 *const rgb = reinterpret_cast<float4 *>(smem + kCmpHalo);
  uint8_t *const w0s = smem + kCmpHalo + kCmpRgb;
  uint8_t *const zs = w0s + kCmpW0;
  uint8_t *const w1s = zs + kCmpZero;
  uint8_t *const w2s = w1s + kCmpW1;
  uint8_t *const act = w2s + kCmpW2;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ float s_bias[80];   // b0 [32], b1 [32], b2 [16]
  const int t = threadIdx.x, warp = t >> 5;
  const int ty = t / kConvTW, tx = t % kConvTW;   // this thread's block within a half
  if (t < 80) s_bias[t] = bias[t];
  const int tiles_x = (d.W + kCmpTW - 1) / kCmpTW, tiles_y = (d.H + kCmpTH - 1) / kCmpTH;
  const int n_tiles = d.B * tiles_x * tiles_y;
  const int my_n = (int)blockIdx.x < n_tiles ? (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const int lsh = io.tile == 32 ? 5 : 4;   // pixel -> tile shift (tiles of 16 or 32 pixels)
  // a tile's origin, halo blocks (r, g, b of the top-left pixel, depth; zero outside the image)
  // and the levels of this thread's two blocks (4 outside the image), loaded into registers
  float4 gv[kGPer];
  int nb = 0, ny0 = 0, nx0 = 0, lv_next[2] = {4, 4};
  auto gather_load = [&](int k) {
    const int tt = (int)blockIdx.x + k * (int)gridDim.x;
    const int r = tt / tiles_x;
    nx0 = (tt - r * tiles_x) * kCmpTW;
    nb = r / tiles_y;
    ny0 = (r - nb * tiles_y) * kCmpTH;
    const float *img = io.img + (size_t)nb * io.H * io.W * 3;
    const float *dep = io.depth + (size_t)nb * io.H * io.W;
#pragma unroll
    for (int j = 0; j < kGPer; ++j) {
      const int q = t + 128 * j, rr = q / HC, c = q - rr * HC;
      const int y = ny0 - 1 + rr, x = nx0 - 1 + c;
      gv[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (q < HR * HC && y >= 0 && y < d.H && x >= 0 && x < d.W) {
        const unsigned src = (unsigned)(2 * y) * (unsigned)io.W + (unsigned)(2 * x);
        gv[j] = make_float4(img[3 * src], img[3 * src + 1], img[3 * src + 2], dep[src]);
      }
    }
    const uint8_t *lrow = io.levels + nb * io.n_tiles + ((2 * (ny0 + ty)) >> lsh) * io.tiles_x;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int y = ny0 + ty, x = nx0 + 8 * h + tx;
      lv_next[h] = y < d.H && x < d.W ? lrow[(2 * x) >> lsh] : 4;
    }
  };
  // the BF16 operand (r, g, b, depth / 8, then zeros: the conversion of block_input's first
  // group) ...
  auto store_operand = [&]() {
#pragma unroll
    for (int j = 0; j < kGPer; ++j) {
      const int q = t + 128 * j;
      if (q < HR * HC) {
        uint4 lo;
        __nv_bfloat162 *l2 = reinterpret_cast<__nv_bfloat162 *>(&lo);
        l2[0] = __floats2bfloat162_rn(gv[j].x, gv[j].y);
        l2[1] = __floats2bfloat162_rn(gv[j].z, gv[j].w * 0.125f);
        l2[2] = __floats2bfloat162_rn(0.0f, 0.0f);
        l2[3] = l2[2];
        *reinterpret_cast<uint4 *>(halo + (size_t)q * 16) = lo;
      }
    }
  };
  // ... and the FP32 colours
  auto store_colours = [&]() {
#pragma unroll
    for (int j = 0; j < kGPer; ++j) {
      const int q = t + 128 * j;
      if (q < HR * HC) rgb[q] = gv[j];
    }
  };
  if (warp == 0) tc::tmem_alloc(&s_tmem, 64);
  for (int i = t; i < kCmpW0 / 16; i += 128) {   // input group 0 of each tap: the first 32 of 64 rows
    const int tap = i / 32, row = i - tap * 32;
    reinterpret_cast<uint4 *>(w0s)[i] = __ldg(W0 + tap * 64 + row);
  }
  for (int i = t; i < kCmpZero / 16; i += 128) reinterpret_cast<uint4 *>(zs)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = t; i < kCmpW1 / 16; i += 128) reinterpret_cast<uint4 *>(w1s)[i] = __ldg(W1 + i);
  for (int i = t; i < kCmpW2 / 16; i += 128) reinterpret_cast<uint4 *>(w2s)[i] = __ldg(W2 + i);
  if (my_n > 0) {
    gather_load(0);
    store_operand();
  }
  tc::fence_proxy_async();
  if (t == 0) tc::mbar_init(&s_bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t h0 = tc::smem_u32(halo), a0 = tc::smem_u32(act);
  const uint32_t b0 = tc::smem_u32(w0s), b1 = tc::smem_u32(w1s), b2 = tc::smem_u32(w2s);
  uint32_t phase = 0;
  // one thread waits for the MMAs (bounded); the others wait at the barrier, issuing nothing
  auto wait_mma = [&]() {
    if (t == 0) {
      if (!tc::mbar_wait(&s_bar, phase)) atomicOr(status, kStatusTimeout);
      tc::fence_before_sync();
    }
    phase ^= 1u;
    __syncthreads();
    tc::fence_after_sync();
  };
  // bias (+ ReLU) of both halves' 32-column accumulators, rounded to BF16 as the next layer's
  // A operands
  auto to_act = [&](int boff) {
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      float v[32];
      tc::tmem_ld32(taddr + 32 * h, v);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint4 pk;
        __nv_bfloat162 *p2 = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          p2[c] = __floats2bfloat162_rn(fmaxf(v[g * 8 + 2 * c] + s_bias[boff + g * 8 + 2 * c], 0.0f),
                                        fmaxf(v[g * 8 + 2 * c + 1] + s_bias[boff + g * 8 + 2 * c + 1], 0.0f));
        *reinterpret_cast<uint4 *>(act + h * 8192 + g * 2048 + t * 16) = pk;
      }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  // the per-block layer (N = 16 or 32) of both halves, issued by thread 0
  auto issue_block_layer = [&](uint32_t bw0, int n) {
    const uint32_t idesc = tc::idesc_bf16_f32(128, n);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
        tc::mma_bf16(tmem + 32 * h, tc::smem_desc(a0 + h * 8192 + kk * 4096, 2048, 128),
                     tc::smem_desc(bw0 + kk * (2 * n * 16), n * 16, 128), idesc, kk > 0);
    tc::mma_commit(&s_bar);
  };
  const int bh = (io.H + 1) / 2, bw = (io.W + 1) / 2;   // blocks per column and row
  for (int k = 0; k < my_n; ++k) {
    const int b = nb, y0 = ny0, x0 = nx0, lv0 = lv_next[0], lv1 = lv_next[1];
    // operand k stored and fenced by every thread; the last tile's tensor-memory reads and
    // colour reads done
    const bool need = __syncthreads_or(lv0 < 4 || lv1 < 4) != 0;
    tc::fence_after_sync();
    store_colours();   // read by this tile's compose, after the barriers below
    if (need && t == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(128, 32);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int ky = tap / 3, kx = tap - 3 * ky;
          tc::mma_bf16(tmem + 32 * h, tc::smem_desc(h0 + (ky * HC + kx + 8 * h) * 16, 0, HC * 16),
                       tc::smem_desc(b0 + tap * 512, (9 - tap) * 512, 128), idesc, tap > 0);
        }
      tc::mma_commit(&s_bar);
    }
    if (k + 1 < my_n) gather_load(k + 1);   // in flight while this tile's layers run
    if (need) {
      wait_mma();
      to_act(0);
      if (t == 0) issue_block_layer(b1, 32);
      wait_mma();
      to_act(32);
      if (t == 0) issue_block_layer(b2, 16);
      wait_mma();
      const int y = y0 + ty, rd = min(y + 1, bh - 1) - y0 + 1, Y = 2 * y;
      float *const img = io.img + (size_t)b * io.H * io.W * 3;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int lv = h ? lv1 : lv0;
        float v[16];
        tc::tmem_ld16(taddr + 32 * h, v);
        if (lv >= 4) continue;   // outside the image or every pixel of the block rendered
        // the top-left pixels of the block, its right and lower neighbours and the diagonal one
        // (the last block repeated past the edge) from the halo's colours; then the same
        // arithmetic as compose_block
        const int cx = tx + 8 * h, x = x0 + cx;
        const int cr = min(x + 1, bw - 1) - x0 + 1;
        const float4 a = rgb[(ty + 1) * HC + cx + 1], right = rgb[(ty + 1) * HC + cr];
        const float4 down = rgb[rd * HC + cx + 1], diag = rgb[rd * HC + cr];
        const float av[3] = {a.x, a.y, a.z}, rv[3] = {right.x, right.y, right.z};
        const float dv[3] = {down.x, down.y, down.z}, gv3[3] = {diag.x, diag.y, diag.z};
        const int X = 2 * x;
        auto put = [&](int dy, int dx, const float *base, int s) {
          if (Y + dy >= io.H || X + dx >= io.W) return;
          float *o = img + 3 * ((unsigned)(Y + dy) * (unsigned)io.W + (unsigned)(X + dx));
#pragma unroll
          for (int c = 0; c < 3; ++c) o[c] = base[c] + (v[4 * c + s] + s_bias[64 + 4 * c + s]);
        };
        float bt[3], bb[3], bd[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          bt[c] = __fmul_rn(__fadd_rn(av[c], rv[c]), 0.5f);
          bb[c] = __fmul_rn(__fadd_rn(av[c], dv[c]), 0.5f);
          bd[c] = __fmul_rn(__fadd_rn(__fadd_rn(__fadd_rn(av[c], rv[c]), dv[c]), gv3[c]), 0.25f);
        }
        if (lv <= 2) put(0, 1, bt, 1);   // top-right: label 3, rendered from level 3
        float *const o1 = img + 3 * ((unsigned)(Y + 1) * (unsigned)io.W + (unsigned)X);
        if (lv <= 1 && Y + 1 < io.H && X + 1 < io.W && (reinterpret_cast<uintptr_t>(o1) & 7u) == 0) {
          // bottom-left and bottom-right: six consecutive floats, three 8-byte stores
          float2 *o2 = reinterpret_cast<float2 *>(o1);
          auto res = [&](int c, int s) { return v[4 * c + s] + s_bias[64 + 4 * c + s]; };
          o2[0] = make_float2(bb[0] + res(0, 2), bb[1] + res(1, 2));
          o2[1] = make_float2(bb[2] + res(2, 2), bd[0] + res(0, 3));
          o2[2] = make_float2(bd[1] + res(1, 3), bd[2] + res(2, 3));
        } else {
          if (lv <= 3) put(1, 0, bb, 2);   // bottom-left: label 4, rendered at level 4
          if (lv <= 1) put(1, 1, bd, 3);   // bottom-right: label 2, rendered from level 2
        }
      }
    }
    if (k + 1 < my_n) store_operand();   // layer 0 of this tile, if any, has completed
    tc::fence_proxy_async();
    tc::fence_before_sync();
  }
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// Weight gradient  dW[cout][cin][tap] += sum over pixels of X[pixel + tap][cin] dY[pixel][cout]
// as D[(tap, cin)][cout] = A[(tap, cin)][pixel] B[cout][pixel]^T with K = pixels: per 8 x 8
// pixel tile the CTA transposes the halo into A (K-major, one M-tile per 128 (tap, cin) rows)
// and dY into B, and accumulates in tensor memory over the tiles it owns; the bias gradient
// is summed alongside.  Partial results are added to the fp32 outputs with atomics.
constexpr int kWgTile = 8;   // 8 x 8 pixel tiles, K = 64 per tile

template <int CIN, int COUT>
constexpr int wgrad_mtiles() { return (9 * CIN + 127) / 128; }

template <int CIN, int COUT>
constexpr int wgrad_smem_bytes() {
  return wgrad_mtiles<CIN, COUT>() * 16384 + (COUT / 8) * 1024 + (CIN / 8) * (kWgTile + 2) * (kWgTile + 2) * 16;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
conv3x3_wgrad_tc_kernel(ConvDims d, const __nv_bfloat16 *__restrict__ X,
                        const __nv_bfloat16 *__restrict__ dY, float *__restrict__ dW,
                        float *__restrict__ db, int tiles_per_cta, uint32_t *__restrict__ status) {
  constexpr int CG = CIN / 8, MT = wgrad_mtiles<CIN, COUT>(), HR = kWgTile + 2, HC = kWgTile + 2;
  constexpr int ABYTES = MT * 16384, BBYTES = (COUT / 8) * 1024;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *as = smem, *bs = smem + ABYTES, *hs = smem + ABYTES + BBYTES;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int tx_n = (d.W + kWgTile - 1) / kWgTile, ty_n = (d.H + kWgTile - 1) / kWgTile;
  const int n_tiles = d.B * tx_n * ty_n;
  if (warp == 0) tc::tmem_alloc(&s_tmem, 128);
  if (t == 0) tc::mbar_init(&s_bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  constexpr int BG = COUT / 8;           // 8-channel groups of dY
  const int my_g = t % BG;               // every (pixel, group) entry of this thread has group my_g
  float dbl[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int issued = 0;
  for (int q = 0; q < tiles_per_cta; ++q) {
    const int tt = blockIdx.x * tiles_per_cta + q;
    if (tt >= n_tiles) break;
    const int b = tt / (tx_n * ty_n), rem = tt - b * (tx_n * ty_n);
    const int y0 = (rem / tx_n) * kWgTile, x0 = (rem % tx_n) * kWgTile;
    if (issued > 0) {   // the previous tile's MMAs still read A and B
      if (!tc::mbar_wait(&s_bar, (issued - 1) & 1) && lane == 0) atomicOr(status, kStatusTimeout);
      tc::fence_after_sync();
    }
    load_halo<CG>(hs, X, b, y0, x0, HR, HC, d.H, d.W);
    // B[cout][pixel]: entry e = (pixel, group of 8 couts)
    for (int e = t; e < 64 * BG; e += 128) {
      const int p = e / BG, g = e - (e / BG) * BG;
      const int y = y0 + p / kWgTile, x = x0 + (p % kWgTile);
      uint4 v = make_uint4(0, 0, 0, 0);
      if (y < d.H && x < d.W) v = __ldg(reinterpret_cast<const uint4 *>(dY + (((size_t)b * d.H + y) * d.W + x) * COUT) + g);
      const __nv_bfloat16 *vb = reinterpret_cast<const __nv_bfloat16 *>(&v);
      uint8_t *dst = bs + g * 1024 + (p >> 3) * 128 + (p & 7) * 2;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        *reinterpret_cast<__nv_bfloat16 *>(dst + c * 16) = vb[c];
        dbl[c] += __bfloat162float(vb[c]);
      }
    }
    __syncthreads();   // halo complete
    // A[(tap, cin)][pixel]: entry e = (pixel, tap, channel group)
    for (int e = t; e < 64 * 9 * CG; e += 128) {
      const int cg = e % CG, pt = e / CG;
      const int tap = pt % 9, p = pt / 9;
      const int ky = tap / 3, kx = tap - 3 * ky;
      const int oy = p / kWgTile, ox = p % kWgTile;
      const uint4 v = *reinterpret_cast<const uint4 *>(hs + ((size_t)(cg * HR + oy + ky) * HC + ox + kx) * 16);
      const __nv_bfloat16 *vb = reinterpret_cast<const __nv_bfloat16 *>(&v);
      const int row = tap * CIN + cg * 8;    // 8 consecutive rows: one core matrix's rows
      const int mt = row >> 7, i = row & 127;
      uint8_t *dst = as + mt * 16384 + (i >> 3) * 1024 + (p >> 3) * 128 + (p & 7) * 2;
#pragma unroll
      for (int c = 0; c < 8; ++c) *reinterpret_cast<__nv_bfloat16 *>(dst + c * 16) = vb[c];
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      const uint32_t a0 = tc::smem_u32(as), b0 = tc::smem_u32(bs);
      const uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
          tc::mma_bf16(tmem + mt * COUT, tc::smem_desc(a0 + mt * 16384 + kc * 256, 128, 1024),
                       tc::smem_desc(b0 + kc * 256, 128, 1024), idesc, issued > 0 || kc > 0);
      tc::mma_commit(&s_bar);
    }
    ++issued;
  }
  // bias gradient: lanes with the same channel group are BG apart within the warp
#pragma unroll
  for (int c = 0; c < 8; ++c)
    for (int o = BG; o < 32; o <<= 1) dbl[c] += __shfl_xor_sync(0xffffffffu, dbl[c], o);
  if (lane < BG)
#pragma unroll
    for (int c = 0; c < 8; ++c) atomicAdd(db + my_g * 8 + c, dbl[c]);
  if (issued > 0) {
    if (!tc::mbar_wait(&s_bar, (issued - 1) & 1) && lane == 0) atomicOr(status, kStatusTimeout);
    tc::fence_after_sync();
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      float v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + mt * COUT;
      if (COUT == 32) tc::tmem_ld32(taddr, v);
      else tc::tmem_ld16(taddr, v);
      const int row = mt * 128 + warp * 32 + lane;
      if (row < 9 * CIN) {
        const int tap = row / CIN, ci = row - tap * CIN;
#pragma unroll
        for (int co = 0; co < COUT; ++co) atomicAdd(dW + ((size_t)co * CIN + ci) * 9 + tap, v[co]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// ------------------------------------------------------- CUDA-core helpers of the network
// x0[b][y2][x2] = (r, g, b, depth / 8, 0 ...) of the top-left pixel of each 2x2 block.
__global__ void gather_input_kernel(const float *__restrict__ img, const float *__restrict__ depth, int B,
                                    int H, int W, __nv_bfloat16 *__restrict__ x0) {
  const int H2 = (H + 1) / 2, W2 = (W + 1) / 2;
  const size_t n = (size_t)B * H2 * W2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x2 = (int)(i % W2);
    const size_t r = i / W2;
    const int y2 = (int)(r % H2), b = (int)(r / H2);
    uint4 *dst = reinterpret_cast<uint4 *>(x0 + i * 16);
    dst[0] = block_input(img, depth, b, H, W, y2, x2);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// Base of sub-pixel (dx, dy) of block (x2, y2), colour c: the bilinear interpolation of the
// blocks' top-left pixels of img [B][H][W][3] -- a, right = (x2 + 1), down = (y2 + 1), diag --
// with the last block repeated past the edge: a; (a + right) / 2; (a + down) / 2;
// (((a + right) + down) + diag) / 4.  Where only top-left pixels are rendered it is the
// interpolating fill (Sec. 3.4 "inherit or interpolate").
__device__ __forceinline__ float base_px(const float *__restrict__ img, int b, int H, int W, int y2,
                                         int x2, int dy, int dx, int c) {
  const int H2 = (H + 1) / 2, W2 = (W + 1) / 2;
  const int xr = min(x2 + 1, W2 - 1), yd = min(y2 + 1, H2 - 1);
  auto tl = [&](int yy, int xx) { return img[3 * (((size_t)b * H + 2 * yy) * W + 2 * xx) + c]; };
  const float a = tl(y2, x2);
  if (dx == 0 && dy == 0) return a;
  if (dy == 0) return __fmul_rn(__fadd_rn(a, tl(y2, xr)), 0.5f);
  if (dx == 0) return __fmul_rn(__fadd_rn(a, tl(yd, x2)), 0.5f);
  return __fmul_rn(__fadd_rn(__fadd_rn(__fadd_rn(a, tl(y2, xr)), tl(yd, x2)), tl(yd, xr)), 0.25f);
}

// Prediction = bilinear base + residual of the sub-pixel; loss = mean squared error against
// the target; g_r = dL/dr (BF16, channels 12..15 zero).  loss_acc accumulates the sum of
// squared errors.
__global__ void loss_kernel(const float *__restrict__ r, const float *__restrict__ img,
                            const float *__restrict__ target, int B, int H, int W, float inv_count,
                            __nv_bfloat16 *__restrict__ g_r, float *__restrict__ loss_acc) {
  const int H2 = (H + 1) / 2, W2 = (W + 1) / 2;
  const size_t n = (size_t)B * H2 * W2;
  float acc = 0.0f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x2 = (int)(i % W2);
    const size_t rr = i / W2;
    const int y2 = (int)(rr % H2), b = (int)(rr / H2);
    float g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int dy = s >> 1, dx = s & 1;
      const int y = 2 * y2 + dy, x = 2 * x2 + dx;
      if (y >= H || x >= W) continue;
      const size_t q = ((size_t)b * H + y) * W + x;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float e = base_px(img, b, H, W, y2, x2, dy, dx, c) + r[i * 16 + c * 4 + s] - target[3 * q + c];
        acc += e * e;
        g[c * 4 + s] = 2.0f * e * inv_count;
      }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(g_r + i * 16);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint4 pk;
      __nv_bfloat162 *p2 = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
      for (int c = 0; c < 4; ++c) p2[c] = __floats2bfloat162_rn(g[h * 8 + 2 * c], g[h * 8 + 2 * c + 1]);
      dst[h] = pk;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, acc);
}

// Adam on the fp32 master parameters.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// BF16 packs of one layer's weights W[cout][cin][9]: forward [tap][cin/8][cout][8 cin] and the
// data-gradient conv's [tap'][cout/8][cin][8 cout] with W'[cin][cout][tap'] = W[cout][cin][8 - tap'].
// A per-block (1x1) layer, W[cout][cin] with taps = 1, is the centre tap (4) of a 3x3 pack whose
// other taps stay zero, so the 3x3 kernels train it unchanged.
__global__ void pack_kernel(const float *__restrict__ w, int cin, int cout, int taps,
                            __nv_bfloat16 *__restrict__ fwd, __nv_bfloat16 *__restrict__ bwd) {
  const int n = cin * cout * taps;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int tap = taps == 9 ? i % 9 : 4, rest = taps == 9 ? i / 9 : i;
    const int ci = rest % cin, co = rest / cin;
    const __nv_bfloat16 v = __float2bfloat16_rn(w[i]);
    fwd[((size_t)(tap * (cin / 8) + ci / 8) * cout + co) * 8 + (ci & 7)] = v;
    if (bwd) bwd[((size_t)((8 - tap) * (cout / 8) + co / 8) * cin + ci) * 8 + (co & 7)] = v;
  }
}

// dW[cout][cin] += the centre tap of a 3x3 weight gradient g[cout][cin][9].
__global__ void centre_tap_kernel(const float *__restrict__ g, int n, float *__restrict__ dW) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dW[i] += g[i * 9 + 4];
}

// Layer tables.  Residual network: ten 3x3 convolutions (16 -> 32, eight 32 -> 32, 32 -> 16).
// Compact network: 3x3 16 -> 32, then the per-block layers 32 -> 32 and 32 -> 16.
constexpr int kLayers = 10;   // the most layers of either network
int n_layers(int arch) { return arch == A3FR_CNN_COMPACT ? 3 : kLayers; }
int layer_in(int arch, int l) { return l == 0 ? 16 : 32; }
int layer_out(int arch, int l) { return l == n_layers(arch) - 1 ? 16 : 32; }
int layer_taps(int arch, int l) { return arch == A3FR_CNN_COMPACT && l > 0 ? 1 : 9; }

size_t weight_offset(int arch, int l) {
  size_t o = 0;
  for (int k = 0; k < l; ++k) o += (size_t)layer_in(arch, k) * layer_out(arch, k) * layer_taps(arch, k);
  return o;
}
size_t bias_offset(int arch, int l) {
  size_t o = weight_offset(arch, n_layers(arch));
  for (int k = 0; k < l; ++k) o += layer_out(arch, k);
  return o;
}
size_t n_params(int arch) { return bias_offset(arch, n_layers(arch)); }

int grid_1d(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace
}  // namespace a3fr

struct a3fr_cnn {
  int arch = A3FR_CNN_RESIDUAL;
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  float *wscratch = nullptr;   // a per-block layer's 3x3 weight gradient [32][32][9]
  __nv_bfloat16 *wf[a3fr::kLayers] = {}, *wb[a3fr::kLayers] = {};
  size_t cap_px = 0;
  __nv_bfloat16 *x0 = nullptr, *h[5] = {}, *t[4] = {}, *g_r = nullptr, *gA = nullptr, *gB = nullptr, *gT = nullptr;
  float *r = nullptr;
  float *loss_acc = nullptr;
  uint32_t *status = nullptr;
  int step = 0;
};

namespace a3fr {
namespace {

template <typename T>
void dfree2(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_acts(a3fr_cnn *n) {
  dfree2(n->x0);
  for (auto &p : n->h) dfree2(p);
  for (auto &p : n->t) dfree2(p);
  dfree2(n->g_r);
  dfree2(n->gA);
  dfree2(n->gB);
  dfree2(n->gT);
  dfree2(n->r);
  n->cap_px = 0;
}

int ensure_acts(a3fr_cnn *n, size_t px) {
  if (px <= n->cap_px) return A3FR_OK;
  free_acts(n);
  const size_t b16 = sizeof(__nv_bfloat16);
  bool ok = cudaMalloc(&n->x0, px * 16 * b16) == cudaSuccess &&
            cudaMalloc(&n->g_r, px * 16 * b16) == cudaSuccess &&
            cudaMalloc(&n->gA, px * 32 * b16) == cudaSuccess &&
            cudaMalloc(&n->gB, px * 32 * b16) == cudaSuccess &&
            cudaMalloc(&n->gT, px * 32 * b16) == cudaSuccess &&
            cudaMalloc(&n->r, px * 16 * sizeof(float)) == cudaSuccess;
  for (auto &p : n->h) ok = ok && cudaMalloc(&p, px * 32 * b16) == cudaSuccess;
  for (auto &p : n->t) ok = ok && cudaMalloc(&p, px * 32 * b16) == cudaSuccess;
  if (!ok) {
    free_acts(n);
    return A3FR_ERR_OOM;
  }
  n->cap_px = px;
  return A3FR_OK;
}

template <int CIN, int COUT, int SRC = kSrcTensor, int DST = kDstTensor>
cudaError_t conv(const ConvDims &d, const __nv_bfloat16 *X, const __nv_bfloat16 *W, const float *bias,
                 const __nv_bfloat16 *R, const __nv_bfloat16 *M, void *Y, int flags, uint32_t *status,
                 cudaStream_t s, const FillIO &io = FillIO{}) {
  constexpr int smem = conv_smem_bytes<CIN, COUT>();
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<CIN, COUT, SRC, DST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  const int tiles = d.B * ((d.W + kConvTW - 1) / kConvTW) * ((d.H + kConvTH - 1) / kConvTH);
  const int grid = tiles < 152 * 5 ? tiles : 152 * 5;
  conv3x3_tc_kernel<CIN, COUT, SRC, DST><<<grid, 128, smem, s>>>(d, X, reinterpret_cast<const uint4 *>(W), bias,
                                                                 R, M, Y, flags, status, io);
  return cudaGetLastError();
}

cudaError_t compact_fill(const ConvDims &d, const a3fr_cnn *n, uint32_t *status, cudaStream_t s, const FillIO &io) {
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(compact_fill_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kCmpSmem);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  const int tiles = d.B * ((d.W + kCmpTW - 1) / kCmpTW) * ((d.H + kCmpTH - 1) / kCmpTH);
  const int grid = tiles < 152 * kCmpCtas ? tiles : 152 * kCmpCtas;
  const int A = A3FR_CNN_COMPACT;
  // the per-block layers' weights: the centre tap (4) of their 3x3 packs [tap][cin/8][cout][8]
  const uint4 *w1 = reinterpret_cast<const uint4 *>(n->wf[1] + 4 * 32 * 32);
  const uint4 *w2 = reinterpret_cast<const uint4 *>(n->wf[2] + 4 * 32 * 16);
  compact_fill_tc_kernel<<<grid, 128, kCmpSmem, s>>>(d, reinterpret_cast<const uint4 *>(n->wf[0]), w1, w2,
                                                     n->params + bias_offset(A, 0), status, io);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad(const ConvDims &d, const __nv_bfloat16 *X, const __nv_bfloat16 *dY, float *dW, float *db,
                  uint32_t *status, cudaStream_t s) {
  constexpr int smem = wgrad_smem_bytes<CIN, COUT>();
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(conv3x3_wgrad_tc_kernel<CIN, COUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  const int tiles = d.B * ((d.H + kWgTile - 1) / kWgTile) * ((d.W + kWgTile - 1) / kWgTile);
  const int ctas = tiles < 152 * 3 ? tiles : 152 * 3;
  const int per = (tiles + ctas - 1) / ctas;
  conv3x3_wgrad_tc_kernel<CIN, COUT><<<ctas, 128, smem, s>>>(d, X, dY, dW, db, per, status);
  return cudaGetLastError();
}

#define CNN_CHECK(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return A3FR_ERR_CUDA;         \
  } while (0)

int pack_all(a3fr_cnn *n, cudaStream_t s) {
  for (int l = 0; l < n_layers(n->arch); ++l) {
    const int cin = layer_in(n->arch, l), cout = layer_out(n->arch, l), taps = layer_taps(n->arch, l);
    pack_kernel<<<grid_1d((size_t)cin * cout * taps), 256, 0, s>>>(n->params + weight_offset(n->arch, l), cin,
                                                                  cout, taps, n->wf[l], l > 0 ? n->wb[l] : nullptr);
    CNN_CHECK(cudaGetLastError());
  }
  return A3FR_OK;
}

// The prediction r (training, a3fr_cnn_forward: io null) or, for the fill (io set), the
// composed image.  Residual network, fill: the first convolution reads its input from the
// render and the last composes the skipped pixels, with neither x0 nor r stored.  Compact
// network, fill: one fused kernel (no activation tensors at all); training: the 3x3 kernels,
// the per-block layers as centre-tap packs.
int forward(a3fr_cnn *n, const float *img, const float *depth, int B, int H, int W, cudaStream_t s,
            const FillIO *io = nullptr) {
  const ConvDims d{B, (H + 1) / 2, (W + 1) / 2};
  const size_t px = (size_t)d.B * d.H * d.W;
  const int A = n->arch;
  if (A == A3FR_CNN_COMPACT && io) {
    CNN_CHECK(compact_fill(d, n, n->status, s, *io));
    return A3FR_OK;
  }
  const int rc = ensure_acts(n, px);
  if (rc != A3FR_OK) return rc;
  const float *P = n->params;
  if (io) {
    CNN_CHECK((conv<16, 32, kSrcImage>(d, nullptr, n->wf[0], P + bias_offset(A, 0), nullptr, nullptr, n->h[0],
                                       kEpiBias | kEpiRelu, n->status, s, *io)));
  } else {
    gather_input_kernel<<<grid_1d(px), 256, 0, s>>>(img, depth, B, H, W, n->x0);
    CNN_CHECK(cudaGetLastError());
    CNN_CHECK((conv<16, 32>(d, n->x0, n->wf[0], P + bias_offset(A, 0), nullptr, nullptr, n->h[0],
                            kEpiBias | kEpiRelu, n->status, s)));
  }
  if (A == A3FR_CNN_COMPACT) {
    CNN_CHECK((conv<32, 32>(d, n->h[0], n->wf[1], P + bias_offset(A, 1), nullptr, nullptr, n->t[0],
                            kEpiBias | kEpiRelu, n->status, s)));
    CNN_CHECK((conv<32, 16>(d, n->t[0], n->wf[2], P + bias_offset(A, 2), nullptr, nullptr, n->r,
                            kEpiBias | kEpiF32, n->status, s)));
    return A3FR_OK;
  }
  for (int b = 0; b < 4; ++b) {
    CNN_CHECK((conv<32, 32>(d, n->h[b], n->wf[1 + 2 * b], P + bias_offset(A, 1 + 2 * b), nullptr, nullptr,
                            n->t[b], kEpiBias | kEpiRelu, n->status, s)));
    CNN_CHECK((conv<32, 32>(d, n->t[b], n->wf[2 + 2 * b], P + bias_offset(A, 2 + 2 * b), n->h[b], nullptr,
                            n->h[b + 1], kEpiBias | kEpiResid, n->status, s)));
  }
  if (io) {
    CNN_CHECK((conv<32, 16, kSrcTensor, kDstCompose>(d, n->h[4], n->wf[9], P + bias_offset(A, 9), nullptr, nullptr,
                                                     nullptr, kEpiBias, n->status, s, *io)));
  } else {
    CNN_CHECK((conv<32, 16>(d, n->h[4], n->wf[9], P + bias_offset(A, 9), nullptr, nullptr, n->r,
                            kEpiBias | kEpiF32, n->status, s)));
  }
  return A3FR_OK;
}

// Weight gradient of a per-block layer: the 3x3 kernel into the scratch, its centre tap added
// to dW[cout][cin]; the bias gradient directly.
template <int CIN, int COUT>
int wgrad_1x1(a3fr_cnn *n, const ConvDims &d, const __nv_bfloat16 *X, const __nv_bfloat16 *dY, float *dW,
              float *db, cudaStream_t s) {
  CNN_CHECK(cudaMemsetAsync(n->wscratch, 0, sizeof(float) * CIN * COUT * 9, s));
  CNN_CHECK((wgrad<CIN, COUT>(d, X, dY, n->wscratch, db, n->status, s)));
  centre_tap_kernel<<<grid_1d((size_t)CIN * COUT), 256, 0, s>>>(n->wscratch, CIN * COUT, dW);
  CNN_CHECK(cudaGetLastError());
  return A3FR_OK;
}

// Gradients of the mean squared error of the prediction against target into n->grads.
int backward(a3fr_cnn *n, const float *img, const float *target, int B, int H, int W, cudaStream_t s) {
  const ConvDims d{B, (H + 1) / 2, (W + 1) / 2};
  const size_t px = (size_t)d.B * d.H * d.W;
  const int A = n->arch;
  float *G = n->grads;
  CNN_CHECK(cudaMemsetAsync(G, 0, sizeof(float) * n_params(A), s));
  CNN_CHECK(cudaMemsetAsync(n->loss_acc, 0, sizeof(float), s));
  loss_kernel<<<grid_1d(px), 256, 0, s>>>(n->r, img, target, B, H, W, 1.0f / (3.0f * B * H * W), n->g_r,
                                          n->loss_acc);
  CNN_CHECK(cudaGetLastError());
  if (A == A3FR_CNN_COMPACT) {
    // r = W2 t + b2;  t = ReLU(W1 h + b1);  h = ReLU(conv0(x0) + b0)
    int rc = wgrad_1x1<32, 16>(n, d, n->t[0], n->g_r, G + weight_offset(A, 2), G + bias_offset(A, 2), s);
    if (rc != A3FR_OK) return rc;
    CNN_CHECK((conv<16, 32>(d, n->g_r, n->wb[2], nullptr, nullptr, n->t[0], n->gA, kEpiMask, n->status, s)));
    rc = wgrad_1x1<32, 32>(n, d, n->h[0], n->gA, G + weight_offset(A, 1), G + bias_offset(A, 1), s);
    if (rc != A3FR_OK) return rc;
    CNN_CHECK((conv<32, 32>(d, n->gA, n->wb[1], nullptr, nullptr, n->h[0], n->gB, kEpiMask, n->status, s)));
    CNN_CHECK((wgrad<16, 32>(d, n->x0, n->gB, G + weight_offset(A, 0), G + bias_offset(A, 0), n->status, s)));
    return A3FR_OK;
  }
  CNN_CHECK((wgrad<32, 16>(d, n->h[4], n->g_r, G + weight_offset(A, 9), G + bias_offset(A, 9), n->status, s)));
  CNN_CHECK((conv<16, 32>(d, n->g_r, n->wb[9], nullptr, nullptr, nullptr, n->gA, 0, n->status, s)));
  __nv_bfloat16 *cur = n->gA, *nxt = n->gB;
  for (int b = 3; b >= 0; --b) {
    const int l2 = 2 + 2 * b, l1 = 1 + 2 * b;
    CNN_CHECK((wgrad<32, 32>(d, n->t[b], cur, G + weight_offset(A, l2), G + bias_offset(A, l2), n->status, s)));
    CNN_CHECK((conv<32, 32>(d, cur, n->wb[l2], nullptr, nullptr, n->t[b], n->gT, kEpiMask, n->status, s)));
    CNN_CHECK((wgrad<32, 32>(d, n->h[b], n->gT, G + weight_offset(A, l1), G + bias_offset(A, l1), n->status, s)));
    CNN_CHECK((conv<32, 32>(d, n->gT, n->wb[l1], nullptr, cur, b == 0 ? n->h[0] : nullptr, nxt,
                            kEpiResid | (b == 0 ? kEpiMask : 0), n->status, s)));
    __nv_bfloat16 *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  CNN_CHECK((wgrad<16, 32>(d, n->x0, cur, G + weight_offset(A, 0), G + bias_offset(A, 0), n->status, s)));
  return A3FR_OK;
}

int read_status(a3fr_cnn *n, cudaStream_t s) {
  uint32_t h = 0;
  CNN_CHECK(cudaMemcpyAsync(&h, n->status, sizeof h, cudaMemcpyDeviceToHost, s));
  CNN_CHECK(cudaStreamSynchronize(s));
  return h ? A3FR_ERR_TIMEOUT : A3FR_OK;
}

}  // namespace
}  // namespace a3fr

using namespace a3fr;

extern "C" int a3fr_tc_tile_gemm(const uint16_t *A, const uint16_t *B, float *D, int n, int k,
                                 int variant, void *stream) {
  if (!A || !B || !D || (n != 16 && n != 32) || k < 16 || k > 64 || k % 16 != 0 ||
      (variant != 0 && variant != 1))
    return A3FR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t *status = nullptr;
  if (cudaMalloc(&status, sizeof(uint32_t)) != cudaSuccess) return A3FR_ERR_OOM;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_tile_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
  if (e == cudaSuccess) {
    tc_tile_gemm_kernel<<<1, 128, kProbeSmem, st>>>(A, B, D, n, k, variant, status);
    e = cudaGetLastError();
  }
  uint32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(status);
  if (e != cudaSuccess) return A3FR_ERR_CUDA;
  return h ? A3FR_ERR_TIMEOUT : A3FR_OK;
}

extern "C" {

size_t a3fr_cnn_param_count(void) { return n_params(A3FR_CNN_RESIDUAL); }

size_t a3fr_cnn_arch_param_count(int arch) {
  return arch == A3FR_CNN_RESIDUAL || arch == A3FR_CNN_COMPACT ? n_params(arch) : 0;
}

int a3fr_cnn_create(a3fr_cnn **out) { return a3fr_cnn_create_arch(out, A3FR_CNN_RESIDUAL); }

int a3fr_cnn_create_arch(a3fr_cnn **out, int arch) {
  if (!out || (arch != A3FR_CNN_RESIDUAL && arch != A3FR_CNN_COMPACT)) return A3FR_ERR_INVALID_ARG;
  *out = nullptr;
  a3fr_cnn *n = new (std::nothrow) a3fr_cnn();
  if (!n) return A3FR_ERR_OOM;
  n->arch = arch;
  const size_t np = n_params(arch);
  bool ok = cudaMalloc(&n->params, np * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->grads, np * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->adam_m, np * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->adam_v, np * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->wscratch, 32 * 32 * 9 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->loss_acc, sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->status, sizeof(uint32_t)) == cudaSuccess;
  for (int l = 0; l < n_layers(arch) && ok; ++l) {   // 3x3 packs (a per-block layer: its centre tap)
    const size_t w = (size_t)layer_in(arch, l) * layer_out(arch, l) * 9 * sizeof(__nv_bfloat16);
    ok = cudaMalloc(&n->wf[l], w) == cudaSuccess && cudaMalloc(&n->wb[l], w) == cudaSuccess &&
         cudaMemset(n->wf[l], 0, w) == cudaSuccess && cudaMemset(n->wb[l], 0, w) == cudaSuccess;
  }
  if (ok) ok = cudaMemset(n->params, 0, np * sizeof(float)) == cudaSuccess &&
               cudaMemset(n->adam_m, 0, np * sizeof(float)) == cudaSuccess &&
               cudaMemset(n->adam_v, 0, np * sizeof(float)) == cudaSuccess &&
               cudaMemset(n->status, 0, sizeof(uint32_t)) == cudaSuccess;
  if (ok) ok = pack_all(n, nullptr) == A3FR_OK && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    a3fr_cnn_destroy(n);
    return A3FR_ERR_OOM;
  }
  *out = n;
  return A3FR_OK;
}

int a3fr_cnn_destroy(a3fr_cnn *n) {
  if (!n) return A3FR_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  free_acts(n);
  dfree2(n->params);
  dfree2(n->grads);
  dfree2(n->adam_m);
  dfree2(n->adam_v);
  dfree2(n->wscratch);
  dfree2(n->loss_acc);
  dfree2(n->status);
  for (int l = 0; l < kLayers; ++l) {
    dfree2(n->wf[l]);
    dfree2(n->wb[l]);
  }
  delete n;
  return A3FR_OK;
}

int a3fr_cnn_set_params(a3fr_cnn *n, const float *host, size_t count) {
  if (!n || !host || count != n_params(n->arch)) return A3FR_ERR_INVALID_ARG;
  CNN_CHECK(cudaMemcpy(n->params, host, count * sizeof(float), cudaMemcpyHostToDevice));
  CNN_CHECK(cudaMemset(n->adam_m, 0, count * sizeof(float)));
  CNN_CHECK(cudaMemset(n->adam_v, 0, count * sizeof(float)));
  n->step = 0;
  const int rc = pack_all(n, nullptr);
  if (rc != A3FR_OK) return rc;
  CNN_CHECK(cudaDeviceSynchronize());
  return A3FR_OK;
}

int a3fr_cnn_get_params(a3fr_cnn *n, float *host, size_t count) {
  if (!n || !host || count != n_params(n->arch)) return A3FR_ERR_INVALID_ARG;
  CNN_CHECK(cudaDeviceSynchronize());
  CNN_CHECK(cudaMemcpy(host, n->params, count * sizeof(float), cudaMemcpyDeviceToHost));
  return A3FR_OK;
}

int a3fr_cnn_forward(a3fr_cnn *n, const float *img, const float *depth, int b, int h, int w,
                     float *residual_out, void *stream) {
  if (!n || !img || !depth || b < 1 || h < 2 || w < 2) return A3FR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = forward(n, img, depth, b, h, w, s);
  if (rc != A3FR_OK) return rc;
  if (residual_out) {
    const size_t px = (size_t)b * ((h + 1) / 2) * ((w + 1) / 2);
    CNN_CHECK(cudaMemcpyAsync(residual_out, n->r, px * 16 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  return A3FR_OK;
}

int a3fr_cnn_grads(a3fr_cnn *n, const float *img, const float *depth, const float *target, int b, int h,
                   int w, float *host_grads, float *loss, void *stream) {
  if (!n || !img || !depth || !target || !host_grads || b < 1 || h < 2 || w < 2) return A3FR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = forward(n, img, depth, b, h, w, s);
  if (rc == A3FR_OK) rc = backward(n, img, target, b, h, w, s);
  if (rc != A3FR_OK) return rc;
  CNN_CHECK(cudaMemcpyAsync(host_grads, n->grads, n_params(n->arch) * sizeof(float), cudaMemcpyDeviceToHost, s));
  float acc = 0.0f;
  CNN_CHECK(cudaMemcpyAsync(&acc, n->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, s));
  rc = read_status(n, s);
  if (loss) *loss = acc / (3.0f * b * h * w);
  return rc;
}

int a3fr_cnn_train_step(a3fr_cnn *n, const float *img, const float *depth, const float *target, int b, int h,
                        int w, float lr, float *loss, void *stream) {
  if (!n || !img || !depth || !target || b < 1 || h < 2 || w < 2 || !(lr > 0.0f)) return A3FR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = forward(n, img, depth, b, h, w, s);
  if (rc == A3FR_OK) rc = backward(n, img, target, b, h, w, s);
  if (rc != A3FR_OK) return rc;
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f / (1.0f - powf(b1, (float)n->step)), c2 = 1.0f / (1.0f - powf(b2, (float)n->step));
  adam_kernel<<<grid_1d(n_params(n->arch)), 256, 0, s>>>(n->params, n->grads, n->adam_m, n->adam_v,
                                                         (int)n_params(n->arch), lr, b1, b2, 1e-8f, c1, c2);
  CNN_CHECK(cudaGetLastError());
  rc = pack_all(n, s);
  if (rc != A3FR_OK) return rc;
  if (loss) {
    float acc = 0.0f;
    CNN_CHECK(cudaMemcpyAsync(&acc, n->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, s));
    rc = read_status(n, s);
    *loss = acc / (3.0f * b * h * w);
    return rc;
  }
  return A3FR_OK;
}

int a3fr_cnn_fill(a3fr_cnn *n, a3fr_scene *scene, float *out_rgb, void *stream) {
  if (!n || !scene || !out_rgb) return A3FR_ERR_INVALID_ARG;
  FillView v{};
  if (!scene_fill_view(scene, &v)) return A3FR_ERR_NOT_READY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const FillIO io{v.depth, out_rgb, v.levels, v.height, v.width, v.tile, v.tiles_x, v.n_tiles};
  return forward(n, out_rgb, v.depth, v.eyes, v.height, v.width, s, &io);
}

}  // extern "C"
