// cnn.cu -- tensor-core (tcgen05) kernels of the learned periphery: a small residual CNN in
// BF16 with FP32 accumulation that reconstructs full-resolution RGB from the quarter-density
// peripheral layer (the level-1 pixels of Sec. 3.4) and its depth.
//
// This file starts with the single-tile GEMM that validates the operand encodings (shared-
// memory descriptors, instruction descriptor, tensor-memory round trip) before the
// convolution kernels use them.
#include "../../include/a3fr.h"
#include "common.cuh"
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
