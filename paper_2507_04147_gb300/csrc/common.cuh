// Shared definitions of the CUDA translation units of libA3FR.so (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace a3fr {

// Floats per Gaussian record: u v conic_a conic_b conic_c opacity r g b depth radius visible.
constexpr int kRec = 12;
constexpr int kMaxEyes = 2;

// Bits of the device status word.
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;

// Preprocess block size; the instance scan works on the same blocking.
constexpr int kPreThreads = 128;

// Per-eye camera as the kernels see it (passed by value).
struct CamParams {
  float R[9];        // world -> camera rotation, row-major
  float t[3];
  float fx, fy, cx, cy, znear;
  float limx, limy;  // 1.3 * tan(fov / 2) per axis, computed on the host in fp32
  int width, height;
};

// Spherical-harmonic normalisations, rounded to fp32 on the host.
struct ShConsts {
  float c0, c1, c2a, c2b, c2c, c3a, c3b, c3c, c3d, c3e;
};

struct PreParams {
  CamParams cam[kMaxEyes];
  ShConsts shc;
  int n_eyes;
  int tile, tiles_x, tiles_y;
};

// Exactly rounded fp32 operations for the key path (never contracted into FMA).
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsq(float a) { return __fsqrt_rn(a); }

}  // namespace a3fr

// Kernel launchers defined in the .cu files (host side).
namespace a3fr {

cudaError_t launch_preprocess(const PreParams &p, int n, int sh_degree, const float *means,
                              const float *log_scales, const float *quats,
                              const float *opacity_logits, const float *sh, float *rec,
                              ushort4 *rect, uint32_t *touched, uint32_t *block_sums,
                              cudaStream_t s);

cudaError_t launch_scan_blocks(const uint32_t *block_sums, int n_blocks,
                               unsigned long long *block_offsets, uint32_t *counts,
                               uint32_t capacity, uint32_t *status, cudaStream_t s);

cudaError_t launch_emit_keys(int n, int n_eyes, int tiles_x, int n_tiles, const float *rec,
                             const ushort4 *rect, const uint32_t *touched,
                             const unsigned long long *block_offsets, uint32_t capacity,
                             uint64_t *keys, uint32_t *vals, cudaStream_t s);

size_t sort_workspace_bytes(size_t capacity);
// Sorts counts[0] pairs (device-resident count, at most capacity); returns in *result_in_alt
// whether the sorted data ended in the alt buffers.
cudaError_t launch_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                        const uint32_t *d_count, size_t capacity, int key_bits, void *workspace,
                        uint32_t *status, bool *result_in_alt, cudaStream_t s);

cudaError_t launch_tile_ranges(const uint64_t *keys, const uint32_t *d_count, size_t capacity,
                               uint2 *ranges, int n_ranges, cudaStream_t s);

struct CompositeParams {
  int n_eyes, width, height, tile, tiles_x, tiles_y, n_tiles;
  int full;                 // 1: every tile at level 4
  int n_layers;
  int level[4];
  float r2[kMaxEyes][3];    // squared layer radii per eye
};

cudaError_t launch_composite(const CompositeParams &p, const float *rec, int n,
                             const uint2 *ranges, const uint32_t *vals, const float *gaze,
                             float *out, uint8_t *levels, float *t_final, uint32_t *n_contrib,
                             unsigned long long *counters, cudaStream_t s);

}  // namespace a3fr
