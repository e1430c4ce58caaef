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

// Decoupled look-back (prefix sums chained across CTAs): one word per CTA, a flag -- the
// CTA's own aggregate, or its inclusive prefix -- above a 62-bit value.  Every wait is
// bounded: after kLookbackSpins polls the status word gets kStatusTimeout and the CTA goes
// on with what it has (its writes stay in bounds).
constexpr unsigned long long kAggFlag = 1ull << 62, kPrefixFlag = 2ull << 62;
constexpr unsigned long long kVal62 = (1ull << 62) - 1ull;
constexpr uint32_t kLookbackSpins = 1u << 22;   // polls 256 ns apart: about a second

__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Exclusive prefix of CTA b's aggregate over the CTAs before it, by one warp: windows of
// 32 predecessors (lane k reads CTA b-1-k) summed nearest first up to the first inclusive
// prefix; an unpublished predecessor is polled again after a back-off.
__device__ inline unsigned long long block_lookback(unsigned long long *lookback, int b, uint32_t *status) {
  const int lane = threadIdx.x & 31;
  unsigned long long excl = 0;
  int j = b - 1;
  uint32_t spins = 0;
  while (j >= 0) {
    const unsigned long long w = j - lane >= 0 ? ld_relaxed64(lookback + (j - lane)) : kPrefixFlag;
    const unsigned long long flag = w & ~kVal62;
    const unsigned ready = __ballot_sync(0xffffffffu, flag != 0ull);
    const unsigned pref = __ballot_sync(0xffffffffu, flag == kPrefixFlag);
    // lanes up to the nearest inclusive prefix, if every one of them is published
    const int lim = pref ? __ffs(pref) - 1 : 31;
    const unsigned need = lim == 31 ? 0xffffffffu : ((2u << lim) - 1u);
    if ((ready & need) != need) {
      if (++spins > kLookbackSpins) {
        if (lane == 0) atomicOr(status, kStatusTimeout);
        break;
      }
      __nanosleep(spins < 3 ? 32u << spins : 256u);
      continue;
    }
    unsigned long long v = lane <= lim ? (w & kVal62) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (pref) break;
    j -= 32;
  }
  return excl;
}

// Programmatic dependent launch: the kernels of a render run back to back in one stream, each
// launched with programmatic stream serialisation (launch_pdl), so the next kernel's CTAs can
// be scheduled while this one's last CTAs finish.  Every such kernel starts with pdl_begin():
// it lets the next kernel be scheduled once all of its own CTAs have started, then waits until
// the previous kernel has completed and its writes are visible -- before touching any memory.
// Both instructions are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}

// floor(r / w) for r < 2^21, 1 <= w < 2^16: the float estimate r * (1/w) is within 2^-23
// relative of r / w, i.e. within 1/4 of the quotient, so its truncation is off by at most one
// and one correction step gives the exact integer quotient.  (r is an instance index inside
// one Gaussian's tile rectangle, below the tiles of an eye.)
__device__ __forceinline__ uint32_t div_small(uint32_t r, uint32_t w) {
  uint32_t d = (uint32_t)((float)r * __frcp_rn((float)w));
  if (d * w > r) --d;
  else if ((d + 1u) * w <= r) ++d;
  return d;
}

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

// The falloff of the compositing step in base 2: with A = -0.5 log2(e) a, B = -log2(e) b,
// C = -0.5 log2(e) c for the conic (a, b, c), (A dx + B dy) dx + C dy^2 = power * log2(e),
// power = -0.5 (a dx^2 + c dy^2) - b dx dy.  Explicitly rounded, so the forward composite
// and its backward evaluate the same value bit for bit.
constexpr float kLog2e = 1.4426950408889634f;
__device__ __forceinline__ float falloff_log2(float A, float B, float C, float dx, float dy) {
  return __fmaf_rn(__fmaf_rn(A, dx, __fmul_rn(B, dy)), dx, __fmul_rn(__fmul_rn(C, dy), dy));
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// alpha = min(0.99, opacity * 2^pw)
__device__ __forceinline__ float blend_alpha(float opacity, float pw) {
  return fminf(0.99f, __fmul_rn(opacity, ex2_approx(pw)));
}

}  // namespace a3fr

// Kernel launchers defined in the .cu files (host side).
namespace a3fr {

constexpr int kMaxSortPasses = 8;

// Digit plan of a radix sort: `passes` digits of the same width, digit p = (key >> shift[p]) & mask.
struct SortPlan {
  int passes;
  int shift[kMaxSortPasses];
  uint32_t mask;
};

// Writes rec/rect per eye, touched[e*n + i], the depth-sort keys dkeys[e*n + i] (depth bits,
// 0xffffffff when culled), depth_count[0] = n_eyes * n and the visible key range
// (depth_count[1] = ~min, depth_count[3] = max, accumulated with atomics on zeroed counters).
cudaError_t launch_preprocess(const PreParams *p_dev, int n, int sh_degree, const float *means,
                              const float *log_scales, const float *quats,
                              const float *opacity_logits, const float *sh, float *rec,
                              ushort4 *rect, uint32_t *touched, uint32_t *dkeys,
                              uint32_t *depth_count, cudaStream_t s);

SortPlan sort_plan(int key_bits, int digit_bits_max);
// small_parts: 2048-key partitions for 32-bit keys (more CTAs for short inputs), else 4096.
size_t onesweep_part_size(bool wide_keys, bool small_parts);
size_t onesweep_lookback_bytes(size_t capacity, int passes, bool wide_keys, bool small_parts);
template <typename K>
cudaError_t launch_histogram(const K *keys, const uint32_t *d_count, size_t capacity,
                             const SortPlan &plan, uint32_t *hist, cudaStream_t s);
// The depth keys' histogram, which first rebases them in place when the visible range fits in
// 24 bits (visible: key - min, culled: 0xffffff; the order of the visible keys is unchanged and
// culled entries emit nothing), so that the top digit is 0 everywhere and the last pass is a
// copy.  range = {~min, -, max} as preprocess leaves it.
cudaError_t launch_depth_histogram(uint32_t *keys, const uint32_t *d_count, const uint32_t *range,
                                   size_t capacity, const SortPlan &plan, uint32_t *hist,
                                   cudaStream_t s);
// Sorts d_count[0] (<= capacity) pairs with `plan`; hist holds the digit counts of every
// pass, counters and lookback are zeroed scratch.  With implicit_vals the first pass takes
// each pair's value to be its input position.  *result_in_alt tells where the result is.
// drop_final_keys: the last pass writes only the values (the caller never reads the sorted
// keys), so the result buffer's keys are left as they were.  final_skip (zeroed by the caller):
// a last pass that is the identity (its digit the same for every key) is skipped and sets
// *final_skip; the result is then in the last pass's input buffers (see Entries).
template <typename K>
cudaError_t launch_onesweep(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt,
                            bool implicit_vals, const uint32_t *d_count, size_t capacity,
                            const SortPlan &plan, const uint32_t *hist, uint32_t *counters,
                            uint32_t *lookback, uint32_t *status, bool *result_in_alt,
                            cudaStream_t s, bool small_parts = false, bool drop_final_keys = false,
                            uint32_t *final_skip = nullptr);

// The 64-bit pair sort of the public API: workspace = histograms | counters | look-back.
size_t sort_workspace_bytes(size_t capacity);
cudaError_t launch_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                        const uint32_t *d_count, size_t capacity, int key_bits, void *workspace,
                        uint32_t *status, bool *result_in_alt, cudaStream_t s);

// The depth-sorted entries: buf[0], or buf[1] when *sel is set (the depth sort skipped its
// identity last pass, leaving the result in that pass's input).
struct Entries {
  const uint32_t *buf[2];
  const uint32_t *sel;
  __device__ __forceinline__ const uint32_t *get() const {
    return (sel != nullptr && *sel != 0u) ? buf[1] : buf[0];
  }
};

// Tile binning of the depth-ordered entries (see binning.cu): per-chunk tile counts
// (bin_count), tile ranges and per-chunk starts (bin_offsets), and the ordered placement of
// every instance at its final slot (bin_emit).
constexpr int kBinMaxChunks = 1536;   // bin_offsets stages chunks x 128 bytes per CTA
struct BinParams {
  int n_eyes, n, n_entries, tiles_x, tiles_y, n_tiles;
  int chunk;                // mean entries per chunk (sizing; bin_plan sets the bounds)
  int n_chunks;
  int row;                  // u32 cells per chunk row of h: tiles rounded up to 4 (16 bytes)
  int band_rows;            // tile rows (eye * tiles_y + y) per bin_emit band
  int n_bands;
  uint32_t capacity;
};
BinParams bin_params(int n_eyes, int n, int tiles_x, int tiles_y, uint32_t capacity);
size_t bin_chunk_cells(const BinParams &p);          // u32 cells of h: chunks x row
// Shared memory of bin_count (the difference grids) and of bin_emit (the cursors); the
// larger of the two, with bin_emit's static part, is checked against the device up front.
size_t bin_count_smem_bytes(int n_eyes, int tiles_x, int tiles_y);
size_t bin_emit_smem_bytes(const BinParams &p);
size_t bin_smem_bytes(int n_eyes, int tiles_x, int tiles_y);
// bounds[0..n_chunks] <- chunk c = entries [bounds[c], bounds[c + 1]), about equal
// instance counts; inst_total is the render's instance total (preprocess), lookback
// (bin_plan_lookback_bytes, zeroed by the caller) chains the CTAs' sums.
size_t bin_plan_lookback_bytes(int n_entries);
cudaError_t launch_bin_plan(const BinParams &p, Entries entries, const uint32_t *touched,
                            const unsigned long long *inst_total, unsigned long long *lookback,
                            uint32_t *bounds, uint32_t *status, cudaStream_t s);
// h[c][r] <- chunk c's instances of tile r.
cudaError_t launch_bin_count(const BinParams &p, Entries entries, const ushort4 *rect,
                             const uint32_t *bounds, uint32_t *h, cudaStream_t s);
// ranges, h[c][r] <- start slot of chunk c's instances of tile r, counts[0] kept, [1] first
// eye, [3] total; the capacity status when the total exceeds the capacity.  lookback
// (bin_lookback_bytes, zeroed by the caller) chains the CTAs' sums.
size_t bin_lookback_bytes(int n_eyes, int n_tiles);
cudaError_t launch_bin_offsets(const BinParams &p, uint32_t *h, unsigned long long *lookback,
                               uint2 *ranges, uint32_t *counts, uint32_t *status, cudaStream_t s);
// vals[slot] <- Gaussian index of every instance, each tile's run in entry order.
cudaError_t launch_bin_emit(const BinParams &p, Entries entries, const ushort4 *rect,
                            const uint32_t *bounds, const uint32_t *h, uint32_t *vals,
                            cudaStream_t s);

// The sort-based binning for renders with many tiles (binning_sorted.cu): per-tile counts
// -> ranges, emit of the depth-ordered instances, then a stable onesweep sort by tile.
// Emission of the tile instances of the depth-ordered entries (see binning_sorted.cu).
struct EmitParams {
  int n, n_entries, n_tiles, tiles_x;
  uint32_t capacity;
};
// Instance offsets of the depth-ordered entries: off[j] <- the instances of the entries before
// j (u32 [n_entries]); pstart[k] (k < n_parts) <- the entry holding instance slot k kGenPart,
// for every such slot below the total; lookback[n_blocks] <- the total, n_blocks = entries /
// 1024 rounded up.  lookback (emit_lookback_bytes) and ticket: zeroed by the caller.
constexpr int kGenPart = 4096;   // slots per partition of the generated tile-sort pass
size_t emit_lookback_bytes(int n_entries);
cudaError_t launch_emit_offsets(const EmitParams &p, Entries entries, const uint32_t *touched,
                                unsigned long long *lookback, uint32_t *off, uint32_t *pstart, int n_parts,
                                uint32_t *ticket, uint32_t *status, cudaStream_t s);
// The instance array those offsets describe (slot off[j] + r = tile r of entry j's rectangle,
// row-major), sorted stably by tile index: the onesweep sort of launch_onesweep whose first
// pass generates its (tile, Gaussian) pairs from the entries instead of reading them, so the
// unsorted instances are never stored.  Same buffers and result convention as
// launch_onesweep (keys/vals are the first pass's would-be input, unread).
struct EmitSource {
  Entries entries;
  const ushort4 *rect;
  const uint32_t *off, *pstart;
  const unsigned long long *total;
  int n_entries, n, n_tiles, tiles_x, n_parts;
};
cudaError_t launch_emit_onesweep(const EmitSource &src, uint32_t *keys, uint32_t *vals, uint32_t *keys_alt,
                                 uint32_t *vals_alt, const uint32_t *d_count, size_t capacity,
                                 const SortPlan &plan, const uint32_t *hist, uint32_t *counters,
                                 uint32_t *lookback, uint32_t *status, bool *result_in_alt,
                                 cudaStream_t s, bool drop_final_keys);

// Per-tile instance counts without enumerating instances: every tile rectangle adds
// +1/-1/-1/+1 at its four corners in a per-eye 2-D difference grid (tiles_y+1 rows of
// tiles_x+1), accumulated per CTA in shared memory and written out as partial grids
// (no global atomics), then summed by a reduction; the 2-D prefix sum is the count.
struct TileScanParams {
  int n_eyes, n, tiles_x, tiles_y, n_tiles;
  uint32_t capacity;
  SortPlan tile_plan;
};
int tile_count_blocks();
size_t tile_grid_cells(int n_eyes, int tiles_x, int tiles_y);
cudaError_t launch_tile_count(const TileScanParams &p, const ushort4 *rect, uint32_t *partials,
                              uint32_t *grid, cudaStream_t s);
// One CTA: counts -> ranges (exclusive scan over tiles, eye-major), tile-sort histograms and
// totals (counts[0] kept, [1..2] per eye, [3] total).  Grids that do not fit in shared
// memory are rejected by the caller up front.
size_t tile_scan_smem_bytes(int n_eyes, int tiles_x, int tiles_y);
cudaError_t launch_tile_scan(const TileScanParams &p, const uint32_t *grid, uint2 *ranges,
                             uint32_t *tile_hist, uint32_t *counts, uint32_t *status,
                             cudaStream_t s);

// keys[j] = tile << 32 | depth bits of the Gaussian vals[j] (for inspection), the tile of
// slot j found in the ranges.
cudaError_t launch_materialize_keys(const uint2 *ranges, int n_ranges, const uint32_t *vals,
                                    const float *rec, int n, int n_tiles, uint32_t count,
                                    uint64_t *keys, cudaStream_t s);

struct CompositeParams {
  int n_eyes, width, height, tile, tiles_x, tiles_y, n_tiles;
  int full;                 // 1: every tile at level 4
  int n_layers;
  int level[4];
  float r2[kMaxEyes][3];    // squared layer radii per eye
  int gaze_slot;            // mailbox-ring slot of the gaze (foveated renders)
  float *out;               // output image [eyes][H][W][3]
  float count_frac;         // count-based tile levels: fraction of heavy tiles per eye (0 = off)
};

// Per-render parameters, resident in device memory so that captured graphs stay valid: one
// host-to-device copy per render updates them.
struct DevParams {
  PreParams pre;
  CompositeParams comp;
};

// Per-round parameters of an incremental round, written on the device by round_begin.
struct RoundPlan {
  float r2[kMaxEyes][3];    // squared layer radii of this round, per eye
  float gaze[kMaxEyes][2];  // gaze of this round, per eye
  int active;               // 0: nothing to render this round
  int pad[3];
};

// Interpolating fill of the skipped pixels of a foveated render (after the composite).
cudaError_t launch_fill(const CompositeParams &p, const CompositeParams *p_dev, const uint8_t *levels,
                        cudaStream_t s);

// Bytes of the work plan of launch_composite for n_ranges = n_eyes * n_tiles.
size_t plan_bytes(int n_ranges);
// One composite: the work plan (tile levels and label intervals) and the compositing.
// Label intervals: a normal foveated render uses the gaze (round == nullptr, uniform == 0);
// the first round of a frame renders every tile at level `uniform` from label 0 and sets cur;
// a later round (round != nullptr) renders from cur up to the level of its gaze and radii,
// stores only those pixels, and raises cur; p.full renders every tile at level 4.  Ranges
// are clamped to kept[0] (the instances the sort kept).  32-pixel tiles: the plan cuts tiles
// into work items (plan32) and one persistent launch renders them all, heaviest first;
// 16-pixel tiles: the plan buckets tiles by label count (none for p.full) and one launch
// packs them into CTAs.  p (host copy) decides the launch shape; the kernels read p_dev (the
// same values).  *kernels (optional) receives the number of kernels launched.
cudaError_t launch_composite(const CompositeParams &p, const CompositeParams *p_dev,
                             const float *rec, int n, const uint2 *ranges, const uint32_t *kept,
                             const uint32_t *vals, const float *gaze, const RoundPlan *round,
                             int uniform, uint8_t *cur, uint32_t *plan, uint8_t *levels,
                             float *t_final, uint32_t *n_contrib, float *depth,
                             unsigned long long *counters, int batch_mult, uint32_t *thresholds,
                             cudaStream_t s, int *kernels = nullptr);

// Incremental rounds (Sec. 3.3, Alg. 1): state on the device, mailbox in mapped host memory.
struct RoundConfig {
  int n_eyes, n_exits, sir;
  float rf[kMaxEyes][3];     // final layer radii r_{f,N} per eye (pixels)
  float expected[8];         // E[dist(u_i, u_N)] per exit i = 1..N (pixels), index i - 1
  float step;                // SIR growth per speculative round (pixels)
  int n_layers;
};
struct RoundState {
  int last_exit;             // exit index of the last prediction consumed (0 = none)
  int rounds;
  int complete;
  int pad;
  float gaze[kMaxEyes][2];
  float r[kMaxEyes][3];      // current layer radii
};
// Mapped mailbox written by the host: seq is odd while a write is in progress.
struct Mailbox {
  unsigned int seq;
  int exit;
  float gaze[kMaxEyes][2];
};
// Status mirrored to mapped host memory after each round (read without a sync).
struct RoundStatus {
  int exit_consumed, complete, rounds, pad;
  float radius[3];
  float pad2;
};
}  // namespace a3fr

struct a3fr_scene;
namespace a3fr {
// Eyes rendered by a scene (eyes with a camera).
int scene_eyes(const a3fr_scene *s);

// What the learned periphery needs from a scene's last foveated render (keep_aux on):
// its expected depth and tile levels; false when there is no such render.
struct FillView {
  const float *depth;
  const uint8_t *levels;
  int eyes, width, height, tile, tiles_x, n_tiles;
};
bool scene_fill_view(a3fr_scene *s, FillView *v);

// Backward rasterizer (backward.cu).
struct BackwardParams {
  int n_eyes, n, width, height, tile, tiles_x, n_tiles;
};
size_t backward_g2d_floats(int n_eyes, int n);
cudaError_t launch_backward(const BackwardParams &bp, const PreParams *pre_dev, int sh_degree,
                            const float *means, const float *log_scales, const float *quats,
                            const float *opacity_logits, const float *sh, const float *rec,
                            const uint2 *ranges, const uint32_t *kept, const uint32_t *vals,
                            const uint8_t *levels, const float *t_final, const uint32_t *n_contrib,
                            const float *dl_drgb, float *g2d, float *d_means, float *d_log_scales,
                            float *d_quats, float *d_logits, float *d_sh, cudaStream_t s);

cudaError_t launch_round_begin(const RoundConfig &c, const Mailbox *mbox, RoundState *state,
                               RoundPlan *plan, RoundStatus *status, uint32_t *error_status,
                               cudaStream_t s);

}  // namespace a3fr
