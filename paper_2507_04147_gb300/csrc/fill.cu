// fill.cu -- the interpolating fill of a foveated render (Sec. 3.4, "inherit or interpolate"),
// a pass after the composite when the fovea asks for it (a3fr_fovea.fill = 1).
#include "common.cuh"

namespace a3fr {
namespace {

// Interpolating fill of a foveated render (Sec. 3.4, "inherit or interpolate"): every pixel its
// tile's level skipped becomes the mean of its rendered 4-neighbours (summed up, down, left,
// right), else of its rendered diagonal neighbours (up-left, up-right, down-left, down-right),
// else keeps the inherited top-left value.  Reads only rendered pixels and writes only skipped
// ones, so the pixels of one launch never race.
//
// One thread per 2x2 block at (x, y) = (2 x2, 2 y2).  A pixel is rendered when its label --
// top-left 0, bottom-right 1, top-right 2, bottom-left 3 -- is below the level of its tile.
// The thread loads the levels of the blocks around its own once (L[by][bx], block offsets
// -1..1; 0 outside the image: nothing rendered there); every neighbour of a skipped pixel lies
// at a fixed offset, so its label and block are compile-time constants.
struct FillCtx {
  const float *p;   // pixel (x, y) of the eye's image
  int L[3][3];      // levels of the blocks at offsets (bx - 1, by - 1)
  int room_x, room_y, W;   // pixels from x to the right edge, from y to the bottom edge; width
  float tl[2][2][3];       // colours of the top-left pixels at offsets (0|2, 0|2), if inside
};

template <int OX, int OY>
__device__ __forceinline__ bool fill_rendered(const FillCtx &c) {
  constexpr int bx = (OX + 2) >> 1, by = (OY + 2) >> 1;   // offsets -1 | 0, 1 | 2 -> 0 | 1 | 2
  constexpr int px = OX & 1, py = OY & 1;
  constexpr int lab = px == py ? px : (px ? 2 : 3);
  return OX < c.room_x && OY < c.room_y && lab < c.L[by][bx];   // negative offsets: L is 0 outside
}

template <int OX, int OY>
__device__ __forceinline__ void fill_add(const FillCtx &c, float &a0, float &a1, float &a2, int &cnt) {
  if (!fill_rendered<OX, OY>(c)) return;
  float q0, q1, q2;
  if constexpr (OX >= 0 && OY >= 0 && OX % 2 == 0 && OY % 2 == 0) {   // a top-left pixel: loaded
    q0 = c.tl[OY / 2][OX / 2][0];
    q1 = c.tl[OY / 2][OX / 2][1];
    q2 = c.tl[OY / 2][OX / 2][2];
  } else {
    const float *q = c.p + 3 * (OY * c.W + OX);
    q0 = q[0];
    q1 = q[1];
    q2 = q[2];
  }
  a0 = __fadd_rn(a0, q0);
  a1 = __fadd_rn(a1, q1);
  a2 = __fadd_rn(a2, q2);
  ++cnt;
}

template <int PX, int PY>
__device__ __forceinline__ void fill_px(const FillCtx &c, float *out_px) {
  if (PX >= c.room_x || PY >= c.room_y) return;
  float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
  int cnt = 0;
  fill_add<PX, PY - 1>(c, a0, a1, a2, cnt);   // up
  fill_add<PX, PY + 1>(c, a0, a1, a2, cnt);   // down
  fill_add<PX - 1, PY>(c, a0, a1, a2, cnt);   // left
  fill_add<PX + 1, PY>(c, a0, a1, a2, cnt);   // right
  if (!cnt) {
    fill_add<PX - 1, PY - 1>(c, a0, a1, a2, cnt);   // up-left
    fill_add<PX + 1, PY - 1>(c, a0, a1, a2, cnt);   // up-right
    fill_add<PX - 1, PY + 1>(c, a0, a1, a2, cnt);   // down-left
    fill_add<PX + 1, PY + 1>(c, a0, a1, a2, cnt);   // down-right
  }
  if (cnt) {
    const float n = (float)cnt;
    float *o = out_px + 3 * (PY * c.W + PX);
    o[0] = __fdiv_rn(a0, n);
    o[1] = __fdiv_rn(a1, n);
    o[2] = __fdiv_rn(a2, n);
  }
}

// Skipped pixels of a block: top-right (label 2) below level 3, bottom-left (label 3) below
// level 4, bottom-right (label 1) at level 1.
__global__ void __launch_bounds__(256)
fill_kernel(const CompositeParams *__restrict__ pp, const uint8_t *__restrict__ levels) {
  pdl_begin();
  const CompositeParams &p = *pp;
  float *out = p.out;
  const int sh = p.tile == 32 ? 5 : 4;   // tiles of 16 or 32 pixels
  const int W = p.width, H = p.height;
  const unsigned W2 = (unsigned)(W + 1) >> 1, H2 = (unsigned)(H + 1) >> 1;
  const unsigned total = (unsigned)p.n_eyes * W2 * H2;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const unsigned r = i / W2, x2 = i - r * W2;
    const unsigned e = r / H2, y2 = r - e * H2;
    const int x = (int)(2 * x2), y = (int)(2 * y2);
    const uint8_t *lv_e = levels + e * p.n_tiles;
    FillCtx c;
    c.W = W;
    c.room_x = W - x;
    c.room_y = H - y;
    c.p = out + 3 * ((size_t)e * H * W + (unsigned)y * (unsigned)W + (unsigned)x);
    // every load of the block at once: its level and its neighbours' (the block up-left is
    // never needed), and the top-left colours of the block and of the blocks right, below
    // and diagonal -- the neighbours a level-1 block interpolates from
#pragma unroll
    for (int by = 0; by < 3; ++by) {
      const int yy = y + 2 * (by - 1);
      const bool yin = yy >= 0 && yy < H;
      const int row = (yy >> sh) * p.tiles_x;
#pragma unroll
      for (int bx = 0; bx < 3; ++bx) {
        const int xx = x + 2 * (bx - 1);
        c.L[by][bx] = (yin && xx >= 0 && xx < W && !(by == 0 && bx == 0)) ? __ldg(lv_e + row + (xx >> sh)) : 0;
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const bool in = 2 * i < c.room_x && 2 * j < c.room_y;
        const float *q = c.p + 3 * (2 * j * W + 2 * i);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) c.tl[j][i][ch] = in ? q[ch] : 0.0f;
      }
    const int lv = c.L[1][1];
    if (lv >= 4) continue;
    float *o = out + 3 * ((size_t)e * H * W + (unsigned)y * (unsigned)W + (unsigned)x);
    if (lv <= 2) fill_px<1, 0>(c, o);
    if (lv <= 3) fill_px<0, 1>(c, o);
    if (lv <= 1) fill_px<1, 1>(c, o);
  }
}

}  // namespace

cudaError_t launch_fill(const CompositeParams &p, const CompositeParams *p_dev, const uint8_t *levels,
                        cudaStream_t s) {
  const size_t total = (size_t)p.n_eyes * ((p.height + 1) / 2) * ((p.width + 1) / 2);   // 2x2 blocks
  if (total == 0) return cudaSuccess;
  const size_t want = (total + 255) / 256;
  const int grid = (int)(want < 152 * 16 ? want : 152 * 16);
  {
    const cudaError_t e_ = launch_pdl(fill_kernel, grid, 256, 0, s, p_dev, levels);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

}  // namespace a3fr
