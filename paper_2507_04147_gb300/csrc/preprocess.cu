// preprocess.cu -- per-Gaussian projection of the 3DGS forward pass (Sec. 2.3,
// "Projection"): activation, camera transform, EWA covariance, conic, 3-sigma radius,
// tile rectangle and SH colour, for every eye in one launch.
//
// Design (GB300):
//  * one thread per Gaussian handles all eyes, so the parameters of a Gaussian are read
//    from HBM once per stereo frame and the eye-independent work (exp of the scales,
//    rotation, 3-D covariance, opacity) is done once;
//  * the block's contiguous slices of the structure-of-arrays inputs are staged into
//    shared memory with coalesced 16-byte loads (SH rows padded to an odd stride so the
//    per-thread reads are free of bank conflicts);
//  * every operation that feeds the depth key and the tile rectangle is an exactly
//    rounded fp32 operation in a fixed order (no FMA contraction), with the project's own
//    Cody-Waite + Taylor exp, so the integer outputs are reproducible bit for bit by any
//    IEEE fp32 implementation of the same sequence;
//  * it also writes the key of the per-frame depth sort of the Gaussians (the depth bits,
//    all ones when the Gaussian is culled), so that the instances can be emitted in depth
//    order and then sorted by tile alone.
#include "common.cuh"

namespace a3fr {
namespace {

// fp32 constants of the exp: 1/ln2, ln2 split into a 16-bit head 45426/2^16 (so k*head
// is exact for |k| < 2^8) and an fp32 tail, and 1/n! for n = 0..7.
__device__ __forceinline__ float exp_cw(float x) {
  x = fminf(x, 88.0f);
  x = fmaxf(x, -87.0f);
  const float k = rintf(fm(x, 0x1.715476p+0f));
  const float r = fs(fs(x, fm(k, 0x1.62e4p-1f)), fm(k, 0x1.7f7d1cp-20f));
  float p = 0x1.a01a02p-13f;
  p = fa(fm(p, r), 0x1.6c16c2p-10f);
  p = fa(fm(p, r), 0x1.111112p-7f);
  p = fa(fm(p, r), 0x1.555556p-5f);
  p = fa(fm(p, r), 0x1.555556p-3f);
  p = fa(fm(p, r), 0x1p-1f);
  p = fa(fm(p, r), 0x1p+0f);
  p = fa(fm(p, r), 0x1p+0f);
  const float scale = __int_as_float((static_cast<int>(k) + 127) << 23);
  return fm(p, scale);
}

// The SH basis of degree sqrt(K) - 1 at the unit direction (dx, dy, dz).
template <int K>
__device__ __forceinline__ void sh_basis(const ShConsts &c, float dx, float dy, float dz,
                                         float b[16]) {
  b[0] = c.c0;
  if constexpr (K > 1) {
    b[1] = fm(-c.c1, dy);
    b[2] = fm(c.c1, dz);
    b[3] = fm(-c.c1, dx);
  }
  if constexpr (K > 4) {
    const float xx = fm(dx, dx), yy = fm(dy, dy), zz = fm(dz, dz);
    b[4] = fm(c.c2a, fm(dx, dy));
    b[5] = fm(-c.c2a, fm(dy, dz));
    b[6] = fm(c.c2b, fs(fs(fm(2.0f, zz), xx), yy));
    b[7] = fm(-c.c2a, fm(dx, dz));
    b[8] = fm(c.c2c, fs(xx, yy));
    if constexpr (K > 9) {
      b[9] = fm(-c.c3a, fm(dy, fs(fm(3.0f, xx), yy)));
      b[10] = fm(c.c3b, fm(fm(dx, dy), dz));
      b[11] = fm(-c.c3c, fm(dy, fs(fs(fm(4.0f, zz), xx), yy)));
      b[12] = fm(c.c3d, fm(dz, fs(fs(fm(2.0f, zz), fm(3.0f, xx)), fm(3.0f, yy))));
      b[13] = fm(-c.c3c, fm(dx, fs(fs(fm(4.0f, zz), xx), yy)));
      b[14] = fm(c.c3e, fm(dz, fs(xx, yy)));
      b[15] = fm(-c.c3a, fm(dx, fs(xx, fm(3.0f, yy))));
    }
  }
}

// SH rows whose 3K floats are whole 16-byte chunks (degrees 1 and 3) are staged by cp.async
// without padding; with an even number of chunks per row (degree 3: 12) chunk m of thread t's
// row sits at m ^ ((t >> 1) & 3), so the eight threads of a quarter warp reading the same
// chunk index hit eight different 16-byte bank groups.
template <int K>
constexpr bool sh_chunked() { return (3 * K) % 4 == 0; }

template <int K>
__device__ __forceinline__ int sh_swz(int m, int t) {
  return ((3 * K / 4) % 2 == 0) ? (m ^ ((t >> 1) & 3)) : m;
}

// colour = max(0, sum_k b_k coef_k + 1/2) per channel, the sum over k in ascending order.
// row: the thread's SH row in shared memory (chunked layout when sh_chunked<K>(), else the
// padded scalar layout).
template <int K>
__device__ __forceinline__ void sh_colour(const ShConsts &c, const float *row, int t, float dx,
                                          float dy, float dz, float rgb[3]) {
  float b[16];
  sh_basis<K>(c, dx, dy, dz, b);
  float acc[3] = {0.0f, 0.0f, 0.0f};
  if constexpr (sh_chunked<K>()) {
    const float4 *row4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int m = 0; m < 3 * K / 4; ++m) {
      const float4 v = row4[sh_swz<K>(m, t)];
      const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int f = 4 * m + j;
        acc[f % 3] = fa(acc[f % 3], fm(b[f / 3], e[j]));
      }
    }
  } else {
#pragma unroll
    for (int f = 0; f < 3 * K; ++f) acc[f % 3] = fa(acc[f % 3], fm(b[f / 3], row[f]));
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaxf(0.0f, fa(acc[ch], 0.5f));
}

// Shared-memory stride of one Gaussian's SH row: 3K floats (chunked rows), else rounded up to
// an odd count so the per-thread scalar reads are free of bank conflicts.
template <int K>
constexpr int sh_stride() { return sh_chunked<K>() ? 3 * K : ((3 * K) % 2 == 0 ? 3 * K + 1 : 3 * K); }

// Cooperative coalesced copy of `count` floats starting at src into shared memory,
// laid out as rows of `row` floats at stride `stride`.  src is 16-byte aligned.
__device__ __forceinline__ void stage(float *dst, const float *__restrict__ src, int count,
                                      int row, int stride) {
  const int n4 = count >> 2;
  const float4 *src4 = reinterpret_cast<const float4 *>(src);
  // four independent 16-byte loads in flight per thread before the shared-memory stores
  for (int i0 = threadIdx.x; i0 < n4; i0 += 4 * blockDim.x) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = i < n4 ? __ldg(src4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n4) {
        const float e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int f = 4 * i + j;
          dst[(f / row) * stride + (f % row)] = e[j];
        }
      }
    }
  }
  for (int f = 4 * n4 + threadIdx.x; f < count; f += blockDim.x)
    dst[(f / row) * stride + (f % row)] = __ldg(src + f);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// Asynchronous copy of `count` floats from src to dst (both 16-byte aligned); a tail of
// fewer than four floats is copied with plain loads.
__device__ __forceinline__ void stage_async(float *dst, const float *__restrict__ src, int count) {
  const int n4 = count >> 2;
  for (int i = threadIdx.x; i < n4; i += blockDim.x) cp_async16(dst + 4 * i, src + 4 * i);
  for (int f = 4 * n4 + threadIdx.x; f < count; f += blockDim.x) dst[f] = __ldg(src + f);
}

// Asynchronous copy of `cnt` chunked SH rows into the swizzled shared-memory layout.
template <int K>
__device__ __forceinline__ void stage_sh_async(float *dst, const float *__restrict__ src, int cnt) {
  constexpr int kChunks = 3 * K / 4;
  for (int g = threadIdx.x; g < cnt * kChunks; g += blockDim.x) {
    const int t = g / kChunks, m = g - t * kChunks;
    cp_async16(dst + 4 * (t * kChunks + sh_swz<K>(m, t)), src + 4 * g);
  }
}

template <int K>
__global__ void __launch_bounds__(kPreThreads, 6)
preprocess_kernel(const PreParams *__restrict__ pp, int n, const float *__restrict__ means,
                  const float *__restrict__ log_scales, const float *__restrict__ quats,
                  const float *__restrict__ opacity_logits, const float *__restrict__ sh,
                  float *__restrict__ rec, ushort4 *__restrict__ rect,
                  uint32_t *__restrict__ touched, uint32_t *__restrict__ dkeys,
                  uint32_t *__restrict__ depth_count) {
  pdl_begin();
  constexpr int SS = sh_stride<K>();
  // per-render parameters: device memory (so a captured graph sees each render's cameras),
  // copied once per block into shared memory
  __shared__ PreParams s_p;
  static_assert(sizeof(PreParams) % 4 == 0 && sizeof(PreParams) / 4 <= kPreThreads, "PreParams copy");
  if (threadIdx.x < sizeof(PreParams) / 4)
    reinterpret_cast<uint32_t *>(&s_p)[threadIdx.x] = reinterpret_cast<const uint32_t *>(pp)[threadIdx.x];
  const PreParams &p = s_p;
  __shared__ __align__(16) float s_mean[kPreThreads * 3];
  __shared__ __align__(16) float s_scale[kPreThreads * 3];
  __shared__ float4 s_quat[kPreThreads];
  __shared__ __align__(16) float s_sh[kPreThreads * SS];

  // every copy of the block is in flight at once: one memory round trip per block
  const int i0 = blockIdx.x * kPreThreads;
  const int cnt = min(kPreThreads, n - i0);
  stage_async(s_mean, means + 3 * (size_t)i0, 3 * cnt);
  stage_async(s_scale, log_scales + 3 * (size_t)i0, 3 * cnt);
  stage_async(reinterpret_cast<float *>(s_quat), quats + 4 * (size_t)i0, 4 * cnt);
  if constexpr (sh_chunked<K>())
    stage_sh_async<K>(s_sh, sh + (size_t)3 * K * i0, cnt);
  else
    stage(s_sh, sh + (size_t)3 * K * i0, 3 * K * cnt, 3 * K, SS);
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();

  const int t = threadIdx.x;
  const int i = i0 + t;
  if (blockIdx.x == 0 && t == 0) depth_count[0] = (uint32_t)(p.n_eyes * n);
  uint32_t kmin = 0xffffffffu, kmax = 0u;   // depth-key range of this thread's visible entries
  uint32_t inst = 0u;                        // tile instances of this thread's entries
  if (i < n) {
    const float mx = s_mean[3 * t], my = s_mean[3 * t + 1], mz = s_mean[3 * t + 2];
    // activation shared by the eyes
    float s2[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float s = exp_cw(s_scale[3 * t + j]);
      s2[j] = fm(s, s);
    }
    float4 q = s_quat[t];
    const float qn = fsq(fa(fa(fa(fm(q.x, q.x), fm(q.y, q.y)), fm(q.z, q.z)), fm(q.w, q.w)));
    const float qw = fdv(q.x, qn), qx = fdv(q.y, qn), qy = fdv(q.z, qn), qz = fdv(q.w, qn);
    float R[3][3];
    R[0][0] = fs(1.0f, fm(2.0f, fa(fm(qy, qy), fm(qz, qz))));
    R[0][1] = fm(2.0f, fs(fm(qx, qy), fm(qw, qz)));
    R[0][2] = fm(2.0f, fa(fm(qx, qz), fm(qw, qy)));
    R[1][0] = fm(2.0f, fa(fm(qx, qy), fm(qw, qz)));
    R[1][1] = fs(1.0f, fm(2.0f, fa(fm(qx, qx), fm(qz, qz))));
    R[1][2] = fm(2.0f, fs(fm(qy, qz), fm(qw, qx)));
    R[2][0] = fm(2.0f, fs(fm(qx, qz), fm(qw, qy)));
    R[2][1] = fm(2.0f, fa(fm(qy, qz), fm(qw, qx)));
    R[2][2] = fs(1.0f, fm(2.0f, fa(fm(qx, qx), fm(qy, qy))));
    float S[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        S[j][k] = fa(fa(fm(fm(R[j][0], s2[0]), R[k][0]), fm(fm(R[j][1], s2[1]), R[k][1])),
                     fm(fm(R[j][2], s2[2]), R[k][2]));
    const float opacity = fdv(1.0f, fa(1.0f, exp_cw(-__ldg(opacity_logits + i))));
    const float *coef = s_sh + t * SS;

    for (int e = 0; e < p.n_eyes; ++e) {
      const CamParams &c = p.cam[e];
      float *o = rec + ((size_t)e * n + i) * kRec;
      ushort4 rc = make_ushort4(0, 0, 0, 0);
      uint32_t n_touched = 0;
      float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0, o2 = o0;
      const float tx = fa(fa(fa(fm(c.R[0], mx), fm(c.R[1], my)), fm(c.R[2], mz)), c.t[0]);
      const float ty = fa(fa(fa(fm(c.R[3], mx), fm(c.R[4], my)), fm(c.R[5], mz)), c.t[1]);
      const float tz = fa(fa(fa(fm(c.R[6], mx), fm(c.R[7], my)), fm(c.R[8], mz)), c.t[2]);
      bool vis = tz > c.znear;
      float u = 0.f, v = 0.f, a = 0.f, b = 0.f, cc = 0.f, det = 0.f, radius = 0.f;
      if (vis) {
        const float txz = fdv(tx, tz), tyz = fdv(ty, tz);
        const float xc = fm(fminf(c.limx, fmaxf(-c.limx, txz)), tz);
        const float yc = fm(fminf(c.limy, fmaxf(-c.limy, tyz)), tz);
        const float tz2 = fm(tz, tz);
        const float J00 = fdv(c.fx, tz), J02 = -fdv(fm(c.fx, xc), tz2);
        const float J11 = fdv(c.fy, tz), J12 = -fdv(fm(c.fy, yc), tz2);
        float T[2][3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          T[0][j] = fa(fm(J00, c.R[j]), fm(J02, c.R[6 + j]));
          T[1][j] = fa(fm(J11, c.R[3 + j]), fm(J12, c.R[6 + j]));
        }
        float U[2][3];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int l = 0; l < 3; ++l)
            U[r][l] = fa(fa(fm(T[r][0], S[0][l]), fm(T[r][1], S[1][l])), fm(T[r][2], S[2][l]));
        const float c00 = fa(fa(fm(U[0][0], T[0][0]), fm(U[0][1], T[0][1])), fm(U[0][2], T[0][2]));
        const float c01 = fa(fa(fm(U[0][0], T[1][0]), fm(U[0][1], T[1][1])), fm(U[0][2], T[1][2]));
        const float c11 = fa(fa(fm(U[1][0], T[1][0]), fm(U[1][1], T[1][1])), fm(U[1][2], T[1][2]));
        a = fa(c00, 0.3f);
        b = c01;
        cc = fa(c11, 0.3f);
        det = fs(fm(a, cc), fm(b, b));
        vis = det > 0.0f;
        if (vis) {
          const float mid = fm(0.5f, fa(a, cc));
          const float lam = fa(mid, fsq(fmaxf(0.1f, fs(fm(mid, mid), det))));
          radius = ceilf(fm(3.0f, fsq(lam)));
          u = fa(fm(c.fx, txz), c.cx);
          v = fa(fm(c.fy, tyz), c.cy);
          // x / tile as x * (1 / tile): the tile (16 or 32) is a power of two, so both are the
          // exact quotient
          const float rb = 1.0f / static_cast<float>(p.tile);
          const float ftx = static_cast<float>(p.tiles_x), fty = static_cast<float>(p.tiles_y);
          const float fx0 = fminf(ftx, fmaxf(0.0f, floorf(fm(fs(u, radius), rb))));
          const float fx1 = fminf(ftx, fmaxf(0.0f, fa(floorf(fm(fa(u, radius), rb)), 1.0f)));
          const float fy0 = fminf(fty, fmaxf(0.0f, floorf(fm(fs(v, radius), rb))));
          const float fy1 = fminf(fty, fmaxf(0.0f, fa(floorf(fm(fa(v, radius), rb)), 1.0f)));
          const int x0 = static_cast<int>(fx0), x1 = static_cast<int>(fx1);
          const int y0 = static_cast<int>(fy0), y1 = static_cast<int>(fy1);
          vis = x0 < x1 && y0 < y1;
          if (vis) {
            rc = make_ushort4(x0, y0, x1, y1);
            n_touched = static_cast<uint32_t>((x1 - x0) * (y1 - y0));
          }
        }
      }
      if (vis) {
        // colour along the unit direction from the eye centre C = -R^T t to the mean
        float C[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          C[j] = -fa(fa(fm(c.R[j], c.t[0]), fm(c.R[3 + j], c.t[1])), fm(c.R[6 + j], c.t[2]));
        float dx = fs(mx, C[0]), dy = fs(my, C[1]), dz = fs(mz, C[2]);
        const float dn = fsq(fa(fa(fm(dx, dx), fm(dy, dy)), fm(dz, dz)));
        dx = fdv(dx, dn);
        dy = fdv(dy, dn);
        dz = fdv(dz, dn);
        float rgb[3];
        sh_colour<K>(p.shc, coef, t, dx, dy, dz, rgb);
        const float inv = fdv(1.0f, det);
        o0 = make_float4(u, v, fm(cc, inv), fm(-b, inv));
        o1 = make_float4(fm(a, inv), opacity, rgb[0], rgb[1]);
        o2 = make_float4(rgb[2], tz, radius, 1.0f);
      }
      float4 *o4 = reinterpret_cast<float4 *>(o);
      o4[0] = o0;
      o4[1] = o1;
      o4[2] = o2;
      rect[(size_t)e * n + i] = rc;
      touched[(size_t)e * n + i] = n_touched;
      inst += n_touched;
      dkeys[(size_t)e * n + i] = vis ? __float_as_uint(tz) : 0xffffffffu;
      if (vis) {
        kmin = min(kmin, __float_as_uint(tz));
        kmax = max(kmax, __float_as_uint(tz));
      }
    }
  }
  // range of the visible depth keys: depth_count[1] = ~min, depth_count[3] = max (the counters
  // start at zero every render, so the minimum is kept as the maximum of the complement)
  // and the render's instance total: depth_count[4..5] as one 64-bit counter
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    inst += __shfl_xor_sync(0xffffffffu, inst, o);
  }
  __shared__ uint32_t s_range[2];
  __shared__ unsigned long long s_inst;
  if (t == 0) {
    s_range[0] = 0u;
    s_range[1] = 0u;
    s_inst = 0ull;
  }
  __syncthreads();
  if ((t & 31) == 0) {
    if (kmax != 0u) {
      atomicMax(&s_range[0], ~kmin);
      atomicMax(&s_range[1], kmax);
    }
    if (inst) atomicAdd(&s_inst, (unsigned long long)inst);
  }
  __syncthreads();
  if (t == 0 && s_range[1] != 0u) {
    atomicMax(depth_count + 1, s_range[0]);
    atomicMax(depth_count + 3, s_range[1]);
  }
  if (t == 0 && s_inst) atomicAdd(reinterpret_cast<unsigned long long *>(depth_count + 4), s_inst);
}

}  // namespace

cudaError_t launch_preprocess(const PreParams *p, int n, int sh_degree, const float *means,
                              const float *log_scales, const float *quats,
                              const float *opacity_logits, const float *sh, float *rec,
                              ushort4 *rect, uint32_t *touched, uint32_t *dkeys,
                              uint32_t *depth_count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (n + kPreThreads - 1) / kPreThreads;
  switch (sh_degree) {
    case 0:
      {
        const cudaError_t e_ = launch_pdl(preprocess_kernel<1>, blocks, kPreThreads, 0, s, p, n, means,
                                          log_scales, quats, opacity_logits, sh, rec, rect, touched, dkeys,
                                          depth_count);
        if (e_ != cudaSuccess) return e_;
      }
      break;
    case 1:
      {
        const cudaError_t e_ = launch_pdl(preprocess_kernel<4>, blocks, kPreThreads, 0, s, p, n, means,
                                          log_scales, quats, opacity_logits, sh, rec, rect, touched, dkeys,
                                          depth_count);
        if (e_ != cudaSuccess) return e_;
      }
      break;
    case 2:
      {
        const cudaError_t e_ = launch_pdl(preprocess_kernel<9>, blocks, kPreThreads, 0, s, p, n, means,
                                          log_scales, quats, opacity_logits, sh, rec, rect, touched, dkeys,
                                          depth_count);
        if (e_ != cudaSuccess) return e_;
      }
      break;
    default:
      {
        const cudaError_t e_ = launch_pdl(preprocess_kernel<16>, blocks, kPreThreads, 0, s, p, n, means,
                                          log_scales, quats, opacity_logits, sh, rec, rect, touched, dkeys,
                                          depth_count);
        if (e_ != cudaSuccess) return e_;
      }
      break;
  }
  return cudaGetLastError();
}

}  // namespace a3fr
