// a3fr_api.cu -- the C ABI of libA3FR.so (declared in include/a3fr.h): scene objects,
// library-owned device workspace, the gaze mailbox, and the orchestration of one render:
//
//   preprocess -> depth sort -> binning (direct: chunk plan, per-chunk tile counts, ranges
//   and chunk starts, every instance to its slot; or sort-based: tile counts / ranges, emit,
//   stable sort by tile) -> [wait for the gaze event] -> plan + composite (level map, blend,
//   inherit or interpolate)
//
// all enqueued on the caller's stream without a host synchronisation (except the very
// first render of a scene created with automatic capacity, which measures the instance
// count once).  Only the composite depends on the gaze, so projection, binning and the
// sort overlap whatever produces the gaze (Sec. 3.3.3, Sec. 4.3: the preprocessing can
// start before gaze tracking finishes).
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "../../include/a3fr.h"
#include "common.cuh"

using namespace a3fr;

namespace {

constexpr int kSlots = 8;  // gaze mailbox ring depth
thread_local std::string g_detail;

int cuda_fail(cudaError_t e, const char *what) {
  g_detail = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? A3FR_ERR_OOM : A3FR_ERR_CUDA;
}

#define A3FR_CHECK(call)                          \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

struct a3fr_scene {
  a3fr_scene_desc desc{};
  a3fr_camera cams[kMaxEyes]{};
  bool cam_set[kMaxEyes]{false, false};

  // per-Gaussian and per-tile workspace, sized for (n_eyes, W, H)
  int alloc_eyes = 0, W = 0, H = 0, TX = 0, TY = 0, n_tiles = 0;
  float *rec = nullptr;
  ushort4 *rect = nullptr;
  uint32_t *touched = nullptr;
  uint32_t *dkeys[2] = {nullptr, nullptr};   // depth-sort keys (ping-pong)
  uint32_t *dvals[2] = {nullptr, nullptr};   // depth-sorted entries e * n + i
  uint2 *ranges = nullptr;
  uint32_t *bin_h = nullptr;                 // per-chunk tile counts, then starts (binning.cu)
  // the sort-based binning (binning_sorted.cu), for renders with more than
  // kBinDirectMaxTiles tiles: difference grids, instance tile keys, the sort's second buffers
  int binning = A3FR_BINNING_AUTO;
  bool sorted_bin = false;
  uint32_t *tile_partials = nullptr;
  uint32_t *tkeys[2] = {nullptr, nullptr};
  uint32_t *vals_alt = nullptr;
  uint32_t *tile_lb = nullptr;               // the tile sort's look-back (capacity-sized)
  uint32_t *pstart = nullptr;                // first entry of every tile-sort partition
  size_t tile_lb_bytes = 0;
  uint32_t *plan = nullptr;                  // tiles bucketed by level (foveated composite)
  uint8_t *levels = nullptr;
  float *t_final = nullptr;
  uint32_t *n_contrib = nullptr;
  float *depth = nullptr;                    // expected depth per pixel (keep_aux only)
  // instance workspace
  size_t capacity = 0;
  bool auto_capacity = false;
  uint32_t *vals = nullptr;                  // Gaussian index of each instance, by tile
  // per-frame scratch, zeroed at the start of every render (see frame_layout)
  void *frame_ws = nullptr;
  size_t frame_ws_bytes = 0;
  uint32_t *counts = nullptr;                // [0] kept, [1..2] per eye, [3] total, [4] entries
  // persistent device state: status | counters[3] (evaluations, staged, blends) | thresholds[2]
  uint32_t *status = nullptr;
  unsigned long long *counters = nullptr;
  uint32_t *thresholds = nullptr;            // per-eye heavy-tile count thresholds
  void *small = nullptr;
  // gaze mailbox ring
  float *gaze_dev = nullptr;
  float *gaze_pinned = nullptr;
  cudaEvent_t gaze_written[kSlots]{};
  cudaEvent_t gaze_consumed[kSlots]{};
  bool slot_written[kSlots]{};
  bool slot_consumed[kSlots]{};
  int gaze_seq = -1;

  cudaStream_t last_stream = nullptr;
  int last_eyes = 0;
  bool keep_aux = false;
  uint64_t renders = 0;
  uint64_t launches = 0;

  // stage timing ring: events[slot][A3FR_N_STAGES + 1]
  int timing_ring = 0;
  cudaEvent_t *timing_events = nullptr;
  uint64_t timed_renders = 0;

  // incremental rounds (Sec. 3.3): the frame's precompute is kept between rounds
  bool round_ready = false;
  a3fr_fovea round_fovea{};
  RoundConfig round_cfg{};
  uint8_t *cur_level = nullptr;              // [eye * tiles] levels rendered so far
  RoundState *round_state = nullptr;         // device
  RoundPlan *round_plan = nullptr;           // device
  Mailbox *mbox_host = nullptr;              // mapped pinned host memory
  Mailbox *mbox_dev = nullptr;
  RoundStatus *status_host = nullptr;        // mapped pinned host memory
  RoundStatus *status_dev = nullptr;
  std::mutex mbox_mutex;
  bool mbox_stalled = false;                 // a write begun and not finished (fault injection)
  float *out_round = nullptr;                // the canvas of the frame's rounds

  // per-render parameters: device copy, pinned staging ring, completion of the last render
  DevParams *params_dev = nullptr;
  DevParams *params_pinned = nullptr;        // [kSlots]
  cudaEvent_t params_copied[kSlots]{};
  bool params_used[kSlots]{};
  uint64_t params_seq = 0;
  cudaEvent_t render_done = nullptr;
  bool render_done_recorded = false;

  // CUDA graphs of the precompute and of the composite (foveated / full)
  bool graph_mode = false;
  bool capturing = false;    // a graph capture is in progress (stage marks are not recorded)
  uint64_t alloc_gen = 1;                    // bumped whenever a workspace buffer moves
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t g_pre = nullptr, g_fov = nullptr, g_full = nullptr;
  uint64_t g_pre_key = 0, g_fov_key = 0, g_full_key = 0;
  uint64_t g_pre_launches = 0;               // kernels in the precompute graph

  int batch_mult = 1;                        // Gaussians staged per thread per composite batch

  // backward: what the last render leaves for it (0 none, 1 full, 2 foveated; keep_aux only)
  int bw_mode = 0;
  float *g2d = nullptr;                      // [eye][n][9] per-Gaussian image-space gradients
  size_t g2d_floats = 0;
};

namespace {

int n_eyes_of(const a3fr_scene *s) { return s->cam_set[1] ? 2 : (s->cam_set[0] ? 1 : 0); }

constexpr int kDepthPasses = 4;   // 32-bit depth keys, 8-bit digits

// AUTO binning: direct placement up to this many tiles (all eyes), the sort-based binning
// above.  Each direct-binning warp walks one chunk of entries serially; with many tiles the
// chunk table (chunks x tiles) caps the chunk count, the chains grow and the stable radix
// sort by tile is faster (3M clustered stereo 2064x2208, 8,970 tiles: 0.54 vs 0.80 ms).
constexpr int kBinDirectMaxTiles = 6144;

int tile_bits_for(int n_ranges) {
  int bits = 1;
  while ((1ll << bits) < (long long)n_ranges) ++bits;
  return bits;
}


// Byte offsets inside frame_ws; everything in it starts at zero every render.
struct FrameLayout {
  size_t counts = 0;                 // counts[0..7] u32 ([6]: emit's block counter), [8..9] the u64 instance total, [10] the depth sort's skipped last pass
  size_t depth_hist = 64;            // kMaxSortPasses x 256 u32
  size_t depth_ctr = 64 + 8192;      // kMaxSortPasses u32 (+pad)
  size_t tile_hist = 64 + 8192 + 64; // sort-based binning: the tile sort's histograms, counters
  size_t tile_ctr = 64 + 8192 + 64 + 8192;
  size_t depth_lb = 0, bin_lb = 0, plan_lb = 0, bounds = 0, emit_lb = 0, tile_diff = 0, total = 0;
};

FrameLayout frame_layout(size_t entries, int eyes, int tiles_x, int tiles_y) {
  FrameLayout L;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  L.depth_lb = up(L.tile_ctr + 64);
  L.bin_lb = up(L.depth_lb + onesweep_lookback_bytes(entries, kDepthPasses, false, false));
  L.plan_lb = up(L.bin_lb + bin_lookback_bytes(eyes, tiles_x * tiles_y));
  L.bounds = up(L.plan_lb + bin_plan_lookback_bytes((int)entries));
  L.emit_lb = up(L.bounds + sizeof(uint32_t) * (kBinMaxChunks + 1));
  L.tile_diff = up(L.emit_lb + emit_lookback_bytes((int)entries));
  L.total = up(L.tile_diff + sizeof(uint32_t) * tile_grid_cells(eyes, tiles_x, tiles_y));
  return L;
}

void free_frame_buffers(a3fr_scene *s) {
  dfree(s->rec);
  dfree(s->rect);
  dfree(s->touched);
  for (int b = 0; b < 2; ++b) {
    dfree(s->dkeys[b]);
    dfree(s->dvals[b]);
  }
  dfree(s->ranges);
  dfree(s->bin_h);
  dfree(s->tile_partials);
  dfree(s->plan);
  dfree(s->cur_level);
  s->round_ready = false;
  dfree(s->levels);
  dfree(s->t_final);
  dfree(s->depth);
  dfree(s->n_contrib);
  s->alloc_eyes = 0;
}

void free_sort_buffers(a3fr_scene *s) {
  for (int b = 0; b < 2; ++b) dfree(s->tkeys[b]);
  dfree(s->vals_alt);
  dfree(s->tile_lb);
  dfree(s->pstart);
  s->tile_lb_bytes = 0;
}

void free_instance_buffers(a3fr_scene *s) {
  dfree(s->vals);
  free_sort_buffers(s);
}

// The sort-based binning's instance buffers: tile keys (ping-pong), the second value buffer
// and the tile sort's look-back, all sized by the capacity.
int ensure_sort_buffers(a3fr_scene *s) {
  if (!s->sorted_bin || s->capacity == 0) {
    free_sort_buffers(s);
    return A3FR_OK;
  }
  if (s->vals_alt) return A3FR_OK;
  const int passes = sort_plan(tile_bits_for(s->alloc_eyes * s->n_tiles), 8).passes;
  for (int b = 0; b < 2; ++b) A3FR_CHECK(cudaMalloc(&s->tkeys[b], sizeof(uint32_t) * s->capacity));
  A3FR_CHECK(cudaMalloc(&s->vals_alt, sizeof(uint32_t) * s->capacity));
  s->tile_lb_bytes = onesweep_lookback_bytes(s->capacity, passes, false, false);
  A3FR_CHECK(cudaMalloc(&s->tile_lb, s->tile_lb_bytes));
  A3FR_CHECK(cudaMalloc(&s->pstart, sizeof(uint32_t) * (s->capacity / kGenPart + 2)));
  return A3FR_OK;
}

// (Re)allocate frame_ws for the current entry count and capacity.
int ensure_frame_ws(a3fr_scene *s) {
  const size_t entries = (size_t)s->alloc_eyes * (size_t)(s->desc.n > 0 ? s->desc.n : 1);
  const FrameLayout L = frame_layout(entries, s->alloc_eyes, s->TX, s->TY);
  if (s->frame_ws && s->frame_ws_bytes >= L.total) return A3FR_OK;
  if (s->frame_ws) {
    A3FR_CHECK(cudaDeviceSynchronize());
    dfree(s->frame_ws);
  }
  s->alloc_gen++;
  A3FR_CHECK(cudaMalloc(&s->frame_ws, L.total));
  A3FR_CHECK(cudaMemset(s->frame_ws, 0, L.total));
  s->frame_ws_bytes = L.total;
  s->counts = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(s->frame_ws) + L.counts);
  return A3FR_OK;
}

int alloc_instances(a3fr_scene *s, size_t capacity) {
  s->alloc_gen++;
  free_instance_buffers(s);
  s->capacity = capacity;
  if (capacity > 0) A3FR_CHECK(cudaMalloc(&s->vals, sizeof(uint32_t) * capacity));
  if (s->alloc_eyes) {
    const int rc = ensure_sort_buffers(s);
    if (rc != A3FR_OK) return rc;
    return ensure_frame_ws(s);
  }
  return A3FR_OK;
}

int ensure_frame_buffers(a3fr_scene *s, int eyes, int W, int H) {
  if (s->alloc_eyes == eyes && s->W == W && s->H == H) return A3FR_OK;
  // a size change: wait for any render still using the old buffers
  if (s->alloc_eyes) A3FR_CHECK(cudaDeviceSynchronize());
  free_frame_buffers(s);
  s->alloc_gen++;
  const int n = s->desc.n;
  const int tile = s->desc.tile;
  {
    int dev = 0, max_optin = 0;
    A3FR_CHECK(cudaGetDevice(&dev));
    A3FR_CHECK(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    s->sorted_bin = s->binning == A3FR_BINNING_SORTED ||
                    (s->binning == A3FR_BINNING_AUTO && (long long)eyes * tx * ty > kBinDirectMaxTiles);
    const size_t need = s->sorted_bin ? tile_scan_smem_bytes(eyes, tx, ty) + 9216 : bin_smem_bytes(eyes, tx, ty);
    if (need > (size_t)max_optin) return A3FR_ERR_INVALID_ARG;
  }
  s->W = W;
  s->H = H;
  s->TX = (W + tile - 1) / tile;
  s->TY = (H + tile - 1) / tile;
  s->n_tiles = s->TX * s->TY;
  const size_t nn = (n > 0 ? (size_t)n : 1) * eyes;
  A3FR_CHECK(cudaMalloc(&s->rec, sizeof(float) * kRec * nn));
  A3FR_CHECK(cudaMalloc(&s->rect, sizeof(ushort4) * nn));
  A3FR_CHECK(cudaMalloc(&s->touched, sizeof(uint32_t) * nn));
  for (int b = 0; b < 2; ++b) {
    A3FR_CHECK(cudaMalloc(&s->dkeys[b], sizeof(uint32_t) * nn));
    A3FR_CHECK(cudaMalloc(&s->dvals[b], sizeof(uint32_t) * nn));
  }
  A3FR_CHECK(cudaMalloc(&s->ranges, sizeof(uint2) * (size_t)s->n_tiles * eyes));
  if (s->sorted_bin)
    A3FR_CHECK(cudaMalloc(&s->tile_partials, sizeof(uint32_t) * (size_t)tile_count_blocks() *
                                                 tile_grid_cells(eyes, s->TX, s->TY)));
  else
    A3FR_CHECK(cudaMalloc(&s->bin_h, sizeof(uint32_t) *
                                         bin_chunk_cells(bin_params(eyes, n > 0 ? n : 1, s->TX, s->TY, 0))));
  A3FR_CHECK(cudaMalloc(&s->plan, plan_bytes(s->n_tiles * eyes)));
  A3FR_CHECK(cudaMalloc(&s->cur_level, (size_t)s->n_tiles * eyes));
  A3FR_CHECK(cudaMalloc(&s->levels, (size_t)s->n_tiles * eyes));
  A3FR_CHECK(cudaMalloc(&s->t_final, sizeof(float) * (size_t)W * H * eyes));
  A3FR_CHECK(cudaMalloc(&s->n_contrib, sizeof(uint32_t) * (size_t)W * H * eyes));
  A3FR_CHECK(cudaMalloc(&s->depth, sizeof(float) * (size_t)W * H * eyes));
  A3FR_CHECK(cudaMemset(s->ranges, 0, sizeof(uint2) * (size_t)s->n_tiles * eyes));
  A3FR_CHECK(cudaMemset(s->levels, 0, (size_t)s->n_tiles * eyes));
  s->alloc_eyes = eyes;
  const int rc = ensure_sort_buffers(s);
  if (rc != A3FR_OK) return rc;
  return ensure_frame_ws(s);
}

CamParams cam_params(const a3fr_camera &c) {
  CamParams p{};
  const float *w = c.world_to_cam;
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) p.R[3 * r + k] = w[4 * r + k];
    p.t[r] = w[4 * r + 3];
  }
  p.fx = c.fx;
  p.fy = c.fy;
  p.cx = c.cx;
  p.cy = c.cy;
  p.znear = c.znear;
  // 1.3 tan(fov / 2), rounded step by step in fp32 (this file is built without contraction)
  const float half_w = 0.5f * (float)c.width, half_h = 0.5f * (float)c.height;
  const float tx = half_w / c.fx, ty = half_h / c.fy;
  p.limx = 1.3f * tx;
  p.limy = 1.3f * ty;
  p.width = c.width;
  p.height = c.height;
  return p;
}

ShConsts sh_consts() {
  const double PI = 3.14159265358979323846;
  ShConsts k;
  k.c0 = (float)(0.5 * std::sqrt(1.0 / PI));
  k.c1 = (float)std::sqrt(3.0 / (4.0 * PI));
  k.c2a = (float)(0.5 * std::sqrt(15.0 / PI));
  k.c2b = (float)(0.25 * std::sqrt(5.0 / PI));
  k.c2c = (float)(0.25 * std::sqrt(15.0 / PI));
  k.c3a = (float)(0.25 * std::sqrt(35.0 / (2.0 * PI)));
  k.c3b = (float)(0.5 * std::sqrt(105.0 / PI));
  k.c3c = (float)(0.25 * std::sqrt(21.0 / (2.0 * PI)));
  k.c3d = (float)(0.25 * std::sqrt(7.0 / PI));
  k.c3e = (float)(0.25 * std::sqrt(105.0 / PI));
  return k;
}

// Squared radius of layer boundary k (Eq. 1 with rho d = fx): f tan(theta_k + dtheta).
float layer_radius2(float fx, float theta_deg, float dtheta_deg) {
  const double PI = 3.14159265358979323846;
  const float r = (float)((double)fx * std::tan(((double)theta_deg + (double)dtheta_deg) * PI / 180.0));
  return r * r;
}

void free_timing(a3fr_scene *s) {
  if (s->timing_events) {
    for (int i = 0; i < s->timing_ring * (A3FR_N_STAGES + 1); ++i)
      if (s->timing_events[i]) cudaEventDestroy(s->timing_events[i]);
    delete[] s->timing_events;
  }
  s->timing_events = nullptr;
  s->timing_ring = 0;
  s->timed_renders = 0;
}

// Records the boundary event k (0..A3FR_N_STAGES) of the current timed render.  Nothing is
// recorded into a graph being captured: a graph-mode render records its events around the
// graph launches instead (render()).
cudaError_t mark(a3fr_scene *s, int k, cudaStream_t stream) {
  if (!s->timing_ring || s->capturing) return cudaSuccess;
  const int slot = (int)(s->timed_renders % (uint64_t)s->timing_ring);
  return cudaEventRecord(s->timing_events[slot * (A3FR_N_STAGES + 1) + k], stream);
}

CompositeParams composite_params(const a3fr_scene *s, int eyes, const a3fr_fovea *fv) {
  CompositeParams cp{};
  cp.n_eyes = eyes;
  cp.width = s->W;
  cp.height = s->H;
  cp.tile = s->desc.tile;
  cp.tiles_x = s->TX;
  cp.tiles_y = s->TY;
  cp.n_tiles = s->n_tiles;
  cp.full = fv ? 0 : 1;
  if (fv) {
    cp.n_layers = fv->n_layers;
    for (int k = 0; k < 4; ++k) cp.level[k] = fv->level[k];
    cp.count_frac = fv->count_frac;
    for (int e = 0; e < eyes; ++e)
      for (int k = 0; k < 3; ++k)
        cp.r2[e][k] = layer_radius2(s->cams[e].fx, fv->theta_deg[k], fv->dtheta_deg);
  } else {
    cp.n_layers = 1;
    cp.level[0] = 4;
  }
  return cp;
}

enum class Mode { kFull, kFoveated, kFirstRound };

// Writes the mailbox under its sequence lock (any host thread).  While a stalled write is
// open (a3fr_stall_mailbox) the payload is updated but the sequence stays odd: the GPU sees
// a write in progress until the stall ends.
void post_mailbox(a3fr_scene *s, int exit, const float *gaze, int eyes) {
  std::lock_guard<std::mutex> lock(s->mbox_mutex);
  Mailbox *m = s->mbox_host;
  const unsigned int seq = __atomic_load_n(&m->seq, __ATOMIC_RELAXED);
  if (!s->mbox_stalled) {
    __atomic_store_n(&m->seq, seq + 1u, __ATOMIC_RELAXED);
    std::atomic_thread_fence(std::memory_order_release);
  }
  __atomic_store_n(&m->exit, exit, __ATOMIC_RELAXED);
  for (int q = 0; q < kMaxEyes; ++q)
    for (int k = 0; k < 2; ++k) {
      const float v = (gaze && q < eyes) ? gaze[2 * q + k] : 0.0f;
      __atomic_store(&m->gaze[q][k], &v, __ATOMIC_RELAXED);
    }
  if (!s->mbox_stalled) __atomic_store_n(&m->seq, seq + 2u, __ATOMIC_RELEASE);
}

// Opens (stall != 0) or closes a mailbox write that stays in progress: the sequence is made
// odd and left so, as when the tracker thread is descheduled in the middle of a write.
void stall_mailbox(a3fr_scene *s, bool stall) {
  std::lock_guard<std::mutex> lock(s->mbox_mutex);
  if (stall == s->mbox_stalled) return;
  Mailbox *m = s->mbox_host;
  const unsigned int seq = __atomic_load_n(&m->seq, __ATOMIC_RELAXED);
  if (stall) {
    __atomic_store_n(&m->seq, seq + 1u, __ATOMIC_RELAXED);
    std::atomic_thread_fence(std::memory_order_release);
  } else {
    __atomic_store_n(&m->seq, seq + 1u, __ATOMIC_RELEASE);
  }
  s->mbox_stalled = stall;
}

// Copies the per-render parameters to the device (pinned staging ring), after the previous
// render of the scene is done with them.
int upload_params(a3fr_scene *s, const DevParams &hp, cudaStream_t stream) {
  const int slot = (int)(s->params_seq++ % kSlots);
  if (s->params_used[slot]) A3FR_CHECK(cudaEventSynchronize(s->params_copied[slot]));
  s->params_pinned[slot] = hp;
  if (s->render_done_recorded) A3FR_CHECK(cudaStreamWaitEvent(stream, s->render_done, 0));
  A3FR_CHECK(cudaMemcpyAsync(s->params_dev, s->params_pinned + slot, sizeof(DevParams),
                             cudaMemcpyHostToDevice, stream));
  A3FR_CHECK(cudaEventRecord(s->params_copied[slot], stream));
  s->params_used[slot] = true;
  return A3FR_OK;
}

int finish_render(a3fr_scene *s, cudaStream_t stream) {
  A3FR_CHECK(cudaEventRecord(s->render_done, stream));
  s->render_done_recorded = true;
  return A3FR_OK;
}

PreParams pre_params(const a3fr_scene *s, int eyes) {
  PreParams pp{};
  for (int e = 0; e < eyes; ++e) pp.cam[e] = cam_params(s->cams[e]);
  pp.shc = sh_consts();
  pp.n_eyes = eyes;
  pp.tile = s->desc.tile;
  pp.tiles_x = s->TX;
  pp.tiles_y = s->TY;
  return pp;
}

// First render of an automatic-capacity scene: read the instance count once, size the
// instance buffers for twice that, and fix the kept count and the status of this render.
int size_instances(a3fr_scene *s, cudaStream_t stream) {
  uint32_t cnt[8];
  A3FR_CHECK(cudaMemcpyAsync(cnt, s->counts, sizeof cnt, cudaMemcpyDeviceToHost, stream));
  A3FR_CHECK(cudaStreamSynchronize(stream));
  size_t want = 2 * (size_t)cnt[3] + (1u << 16);
  if (want >= (1u << 30)) want = (1u << 30) - 1;
  const int rc = alloc_instances(s, want);
  if (rc != A3FR_OK) return rc;
  cnt[0] = cnt[3] < s->capacity ? cnt[3] : (uint32_t)s->capacity;
  A3FR_CHECK(cudaMemcpyAsync(s->counts, cnt, sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
  A3FR_CHECK(cudaMemsetAsync(s->status, 0, sizeof(uint32_t), stream));
  A3FR_CHECK(cudaStreamSynchronize(stream));
  return A3FR_OK;
}

// The sort-based binning (renders with more than kBinDirectMaxTiles tiles): tile counts ->
// ranges and the tile sort's histograms, emit of the depth-ordered instances, stable
// onesweep by tile index.  The sort's result lands in s->vals.
int enqueue_bin_sorted(a3fr_scene *s, int eyes, Entries entries, const FrameLayout &L,
                       cudaStream_t stream, bool allow_resize, uint64_t *launches) {
  const int n = s->desc.n;
  const SortPlan tile_plan = sort_plan(tile_bits_for(eyes * s->n_tiles), 8);
  unsigned char *ws = static_cast<unsigned char *>(s->frame_ws);
  uint32_t *counts = s->counts;
  uint32_t *tile_hist = reinterpret_cast<uint32_t *>(ws + L.tile_hist);
  uint32_t *tile_ctr = reinterpret_cast<uint32_t *>(ws + L.tile_ctr);
  unsigned long long *emit_lb = reinterpret_cast<unsigned long long *>(ws + L.emit_lb);
  uint32_t *tile_diff = reinterpret_cast<uint32_t *>(ws + L.tile_diff);
  TileScanParams tp{};
  tp.n_eyes = eyes;
  tp.n = n;
  tp.tiles_x = s->TX;
  tp.tiles_y = s->TY;
  tp.n_tiles = s->n_tiles;
  tp.capacity = (uint32_t)s->capacity;
  tp.tile_plan = tile_plan;
  if (n > 0) {
    A3FR_CHECK(launch_tile_count(tp, s->rect, s->tile_partials, tile_diff, stream));
    *launches += 2;
  }
  A3FR_CHECK(launch_tile_scan(tp, tile_diff, s->ranges, tile_hist, counts, s->status, stream));
  ++*launches;
  if (allow_resize && s->auto_capacity && s->capacity == 0 && n > 0) {
    const int rc = size_instances(s, stream);
    if (rc != A3FR_OK) return rc;
  }
  A3FR_CHECK(mark(s, A3FR_STAGE_EMIT, stream));
  if (n > 0 && s->capacity > 0) {
    EmitParams ep{};
    ep.n = n;
    ep.n_entries = eyes * n;
    ep.n_tiles = s->n_tiles;
    ep.tiles_x = s->TX;
    ep.capacity = (uint32_t)s->capacity;
    // an odd number of passes ends in the second buffers: start there so it ends in vals
    uint32_t *v0 = tile_plan.passes % 2 ? s->vals_alt : s->vals;
    uint32_t *v1 = tile_plan.passes % 2 ? s->vals : s->vals_alt;
    A3FR_CHECK(cudaMemsetAsync(s->tile_lb, 0, s->tile_lb_bytes, stream));
    // the entries' instance offsets go to the depth sort's first key buffer, free once the
    // depth sort has run
    uint32_t *off = s->dkeys[0];
    const int n_parts = (int)((s->capacity + kGenPart - 1) / kGenPart);
    A3FR_CHECK(launch_emit_offsets(ep, entries, s->touched, emit_lb, off, s->pstart, n_parts, counts + 6,
                                   s->status, stream));
    EmitSource src{};
    src.entries = entries;
    src.rect = s->rect;
    src.off = off;
    src.pstart = s->pstart;
    src.total = emit_lb + (ep.n_entries + 1023) / 1024;
    src.n_parts = n_parts;
    src.n_entries = ep.n_entries;
    src.n = n;
    src.n_tiles = s->n_tiles;
    src.tiles_x = s->TX;
    bool in_alt = false;
    A3FR_CHECK(launch_emit_onesweep(src, s->tkeys[0], v0, s->tkeys[1], v1, counts, s->capacity, tile_plan,
                                    tile_hist, tile_ctr, s->tile_lb, s->status, &in_alt, stream,
                                    /*drop_final_keys=*/true));
    *launches += 1 + tile_plan.passes;
  }
  return A3FR_OK;
}

// The precompute of a render: projection, depth sort and binning (tile ranges and the
// instances in tile order).  allow_resize: the first render of an automatic-capacity scene
// measures the instance count (one host synchronisation) and sizes the instance buffers.
int enqueue_pre(a3fr_scene *s, int eyes, cudaStream_t stream, bool allow_resize,
                uint64_t *launches) {
  const int n = s->desc.n;
  const int n_entries = eyes * n;
  const SortPlan depth_plan = sort_plan(32, 8);
  const FrameLayout L = frame_layout((size_t)(n_entries > 0 ? n_entries : eyes), eyes, s->TX, s->TY);
  unsigned char *ws = static_cast<unsigned char *>(s->frame_ws);
  uint32_t *counts = s->counts;
  uint32_t *depth_hist = reinterpret_cast<uint32_t *>(ws + L.depth_hist);
  uint32_t *depth_ctr = reinterpret_cast<uint32_t *>(ws + L.depth_ctr);
  uint32_t *depth_lb = reinterpret_cast<uint32_t *>(ws + L.depth_lb);
  unsigned long long *bin_lb = reinterpret_cast<unsigned long long *>(ws + L.bin_lb);
  unsigned long long *plan_lb = reinterpret_cast<unsigned long long *>(ws + L.plan_lb);
  uint32_t *bounds = reinterpret_cast<uint32_t *>(ws + L.bounds);
  const unsigned long long *inst_total = reinterpret_cast<const unsigned long long *>(counts + 8);

  A3FR_CHECK(mark(s, A3FR_STAGE_PREPROCESS, stream));
  A3FR_CHECK(cudaMemsetAsync(s->frame_ws, 0, L.total, stream));
  if (n > 0) {
    A3FR_CHECK(launch_preprocess(&s->params_dev->pre, n, s->desc.sh_degree, s->desc.means,
                                 s->desc.log_scales, s->desc.quats, s->desc.opacity_logits,
                                 s->desc.sh, s->rec, s->rect, s->touched, s->dkeys[0], counts + 4,
                                 stream));
    ++*launches;
  }
  // depth sort of the (eye, Gaussian) entries: 4 passes, result back in dkeys[0]/dvals[0]
  A3FR_CHECK(mark(s, A3FR_STAGE_DEPTH_SORT, stream));
  if (n > 0) {
    A3FR_CHECK(launch_depth_histogram(s->dkeys[0], counts + 4, counts + 5, (size_t)n_entries,
                                      depth_plan, depth_hist, stream));
    bool in_alt = false;
    A3FR_CHECK(launch_onesweep<uint32_t>(s->dkeys[0], s->dvals[0], s->dkeys[1], s->dvals[1], true,
                                         counts + 4, (size_t)n_entries, depth_plan, depth_hist,
                                         depth_ctr, depth_lb, s->status, &in_alt, stream, false,
                                         /*drop_final_keys=*/true, /*final_skip=*/counts + 10));
    *launches += 1 + depth_plan.passes;
  }
  // the last pass's digit (the top 8 bits of the rebased depth) is often one bucket: that pass
  // then writes nothing and sets counts[10], and the kernels below read its input instead
  const Entries entries{{s->dvals[depth_plan.passes % 2], s->dvals[(depth_plan.passes + 1) % 2]},
                        counts + 10};
  A3FR_CHECK(mark(s, A3FR_STAGE_BIN, stream));
  if (s->sorted_bin) return enqueue_bin_sorted(s, eyes, entries, L, stream, allow_resize, launches);
  // per-chunk tile counts -> tile ranges, per-chunk starts, totals
  BinParams bp = bin_params(eyes, n, s->TX, s->TY, (uint32_t)s->capacity);
  A3FR_CHECK(launch_bin_plan(bp, entries, s->touched, inst_total, plan_lb, bounds, s->status, stream));
  A3FR_CHECK(launch_bin_count(bp, entries, s->rect, bounds, s->bin_h, stream));
  A3FR_CHECK(launch_bin_offsets(bp, s->bin_h, bin_lb, s->ranges, counts, s->status, stream));
  *launches += 3;
  if (allow_resize && s->auto_capacity && s->capacity == 0 && n > 0) {
    // first render: read the instance count once, then size the instance buffer (the
    // starts in bin_h do not depend on the capacity)
    const int rc = size_instances(s, stream);
    if (rc != A3FR_OK) return rc;
    bp.capacity = (uint32_t)s->capacity;
  }
  // every instance straight to its slot, each tile's run in depth order
  A3FR_CHECK(mark(s, A3FR_STAGE_EMIT, stream));
  if (n > 0 && s->capacity > 0) {
    A3FR_CHECK(launch_bin_emit(bp, entries, s->rect, bounds, s->bin_h, s->vals, stream));
    ++*launches;
  }
  return A3FR_OK;
}

// The composite of a render (plan + composite, or composite alone for full resolution).
int enqueue_comp(a3fr_scene *s, const CompositeParams &cp, int uniform, uint8_t *cur, bool fill,
                 cudaStream_t stream, uint64_t *launches) {
  A3FR_CHECK(mark(s, A3FR_STAGE_COMPOSITE, stream));
  int kernels = 0;
  A3FR_CHECK(launch_composite(cp, &s->params_dev->comp, s->rec, s->desc.n, s->ranges, s->counts,
                              s->vals, s->gaze_dev, nullptr, uniform, cur, s->plan, s->levels,
                              s->keep_aux ? s->t_final : nullptr,
                              s->keep_aux ? s->n_contrib : nullptr,
                              s->keep_aux ? s->depth : nullptr, s->counters, s->batch_mult, s->thresholds, stream, &kernels));
  *launches += (uint64_t)kernels;
  if (fill) {
    A3FR_CHECK(launch_fill(cp, &s->params_dev->comp, s->levels, stream));
    ++*launches;
  }
  A3FR_CHECK(mark(s, A3FR_N_STAGES, stream));
  return A3FR_OK;
}

// Captures `fn` (enqueuing on a stream) into an executable graph.
template <typename F>
int capture(a3fr_scene *s, cudaGraphExec_t *exec, uint64_t *kernels, F fn) {
  if (*exec) {
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  A3FR_CHECK(cudaStreamBeginCapture(s->capture_stream, cudaStreamCaptureModeRelaxed));
  *kernels = 0;
  s->capturing = true;
  const int rc = fn(s->capture_stream, kernels);
  s->capturing = false;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s->capture_stream, &g);
  if (rc != A3FR_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  const cudaError_t ei = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate");
  return A3FR_OK;
}

int render(a3fr_scene *s, const a3fr_fovea *fv, float *out, cudaStream_t stream, Mode mode) {
  s->round_ready = false;   // any render replaces the precompute that rounds build on
  const int eyes = n_eyes_of(s);
  if (eyes == 0 || out == nullptr) return A3FR_ERR_INVALID_ARG;
  const a3fr_camera &c0 = s->cams[0];
  if (eyes == 2 && (s->cams[1].width != c0.width || s->cams[1].height != c0.height))
    return A3FR_ERR_INVALID_ARG;
  if (fv) {
    if (fv->n_layers < 1 || fv->n_layers > 4) return A3FR_ERR_INVALID_ARG;
    for (int k = 0; k < fv->n_layers; ++k)
      if (fv->level[k] < 1 || fv->level[k] > 4) return A3FR_ERR_INVALID_ARG;
    if (fv->fill != 0 && fv->fill != 1) return A3FR_ERR_INVALID_ARG;
    if (!(fv->count_frac >= 0.0f && fv->count_frac <= 1.0f)) return A3FR_ERR_INVALID_ARG;
    if (mode == Mode::kFoveated && s->gaze_seq < 0) return A3FR_ERR_NOT_READY;
  }
  int rc = ensure_frame_buffers(s, eyes, c0.width, c0.height);
  if (rc != A3FR_OK) return rc;

  DevParams hp{};
  hp.pre = pre_params(s, eyes);
  hp.comp = composite_params(s, eyes, mode == Mode::kFull ? nullptr : fv);
  hp.comp.out = out;
  int slot = -1;
  if (mode == Mode::kFoveated) {
    slot = s->gaze_seq % kSlots;
    hp.comp.gaze_slot = slot;
  }
  rc = upload_params(s, hp, stream);
  if (rc != A3FR_OK) return rc;

  uint64_t launches = 0;
  // with stage timing on, a graph-mode render times its two graphs: the precompute graph as
  // the preprocess stage (the depth sort, bin and emit stages then read zero) and the
  // composite graph as the composite stage
  const bool graphs = s->graph_mode && s->capacity > 0 && mode != Mode::kFirstRound &&
                      s->desc.n > 0;
  if (graphs) {
    const uint64_t key = s->alloc_gen * 4 + (s->keep_aux ? 2 : 0) + (uint64_t)eyes;
    if (!s->g_pre || s->g_pre_key != key) {
      rc = capture(s, &s->g_pre, &s->g_pre_launches, [&](cudaStream_t cs, uint64_t *l) {
        return enqueue_pre(s, eyes, cs, false, l);
      });
      if (rc != A3FR_OK) return rc;
      s->g_pre_key = key;
    }
    A3FR_CHECK(mark(s, A3FR_STAGE_PREPROCESS, stream));
    A3FR_CHECK(cudaGraphLaunch(s->g_pre, stream));
    launches += s->g_pre_launches;
  } else {
    rc = enqueue_pre(s, eyes, stream, true, &launches);
    if (rc != A3FR_OK) return rc;
  }

  int uniform = 0;
  uint8_t *cur = nullptr;
  if (mode == Mode::kFoveated) {
    A3FR_CHECK(cudaStreamWaitEvent(stream, s->gaze_written[slot], 0));
  } else if (mode == Mode::kFirstRound) {
    // round 1 renders every tile at the peripheral level (Fig. 6: rendering starts at
    // peripheral resolution) and starts the frame's round state afresh
    uniform = fv->level[fv->n_layers - 1];
    cur = s->cur_level;
    A3FR_CHECK(cudaMemsetAsync(s->round_state, 0, sizeof(RoundState), stream));
    post_mailbox(s, 0, nullptr, eyes);
  }
  const bool fill = mode == Mode::kFoveated && fv->fill == 1;
  if (graphs) {
    const bool by_count = mode == Mode::kFoveated && fv->count_frac > 0.0f;
    const uint64_t key = s->alloc_gen * 16 + (by_count ? 8 : 0) + (fill ? 4 : 0) + (s->keep_aux ? 2 : 0) +
                         (uint64_t)eyes;
    cudaGraphExec_t *g = mode == Mode::kFull ? &s->g_full : &s->g_fov;
    uint64_t *gk = mode == Mode::kFull ? &s->g_full_key : &s->g_fov_key;
    if (!*g || *gk != key) {
      uint64_t k = 0;
      rc = capture(s, g, &k, [&](cudaStream_t cs, uint64_t *l) {
        return enqueue_comp(s, hp.comp, 0, nullptr, fill, cs, l);
      });
      if (rc != A3FR_OK) return rc;
      *gk = key;
    }
    for (int k = A3FR_STAGE_DEPTH_SORT; k <= A3FR_STAGE_COMPOSITE; ++k)
      A3FR_CHECK(mark(s, k, stream));
    A3FR_CHECK(cudaGraphLaunch(*g, stream));
    A3FR_CHECK(mark(s, A3FR_N_STAGES, stream));
    launches += (mode == Mode::kFull ? 1 : 2) + (fill ? 1 : 0);
  } else {
    rc = enqueue_comp(s, hp.comp, uniform, cur, fill, stream, &launches);
    if (rc != A3FR_OK) return rc;
  }
  if (mode == Mode::kFoveated) {
    A3FR_CHECK(cudaEventRecord(s->gaze_consumed[slot], stream));
    s->slot_consumed[slot] = true;
  }
  rc = finish_render(s, stream);
  if (rc != A3FR_OK) return rc;
  s->last_stream = stream;
  s->last_eyes = eyes;
  s->renders++;
  s->launches += launches;
  if (s->timing_ring) s->timed_renders++;
  if (mode == Mode::kFirstRound) {
    s->round_ready = true;
    s->out_round = out;
  }
  s->bw_mode = !s->keep_aux ? 0 : (mode == Mode::kFull ? 1 : (mode == Mode::kFoveated ? 2 : 0));
  return A3FR_OK;
}

// One later round: round_begin (mailbox, Eq. 3' / Eq. 4) + plan + composite of new labels.
int render_round(a3fr_scene *s, float *out, cudaStream_t stream) {
  if (!s->round_ready || out == nullptr) return A3FR_ERR_NOT_READY;
  const int eyes = s->last_eyes;
  DevParams hp{};
  hp.pre = pre_params(s, eyes);
  hp.comp = composite_params(s, eyes, &s->round_fovea);
  hp.comp.out = out;
  int rc = upload_params(s, hp, stream);
  if (rc != A3FR_OK) return rc;
  A3FR_CHECK(launch_round_begin(s->round_cfg, s->mbox_dev, s->round_state, s->round_plan,
                                s->status_dev, s->status, stream));
  int kernels = 0;
  A3FR_CHECK(launch_composite(hp.comp, &s->params_dev->comp, s->rec, s->desc.n, s->ranges,
                              s->counts, s->vals, s->gaze_dev, s->round_plan, 0, s->cur_level,
                              s->plan, s->levels, s->keep_aux ? s->t_final : nullptr,
                              s->keep_aux ? s->n_contrib : nullptr,
                              s->keep_aux ? s->depth : nullptr, s->counters, s->batch_mult, s->thresholds, stream, &kernels));
  rc = finish_render(s, stream);
  if (rc != A3FR_OK) return rc;
  s->launches += 1 + (uint64_t)kernels;   // round_begin, plan, composite
  s->last_stream = stream;
  s->bw_mode = 0;
  return A3FR_OK;
}

}  // namespace

int a3fr::scene_eyes(const a3fr_scene *s) { return n_eyes_of(s); }

bool a3fr::scene_fill_view(a3fr_scene *s, FillView *v) {
  if (!s || !v || s->bw_mode != 2 || s->last_eyes == 0) return false;
  v->depth = s->depth;
  v->levels = s->levels;
  v->eyes = s->last_eyes;
  v->width = s->cams[0].width;
  v->height = s->cams[0].height;
  v->tile = s->desc.tile;
  v->tiles_x = s->TX;
  v->n_tiles = s->n_tiles;
  return true;
}

extern "C" {

int a3fr_create_scene(const a3fr_scene_desc *desc, size_t instance_capacity, a3fr_scene **out) {
  if (!desc || !out) return A3FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (desc->n < 0 || desc->n >= (1 << 30) || desc->sh_degree < 0 || desc->sh_degree > 3 ||
      desc->reserved != 0)
    return A3FR_ERR_INVALID_ARG;
  const int tile = desc->tile == 0 ? 16 : desc->tile;
  if (tile != 16 && tile != 32) return A3FR_ERR_INVALID_ARG;
  if (instance_capacity >= (1u << 30)) return A3FR_ERR_INVALID_ARG;
  if (desc->n > 0) {
    const void *ptrs[5] = {desc->means, desc->log_scales, desc->quats, desc->opacity_logits,
                           desc->sh};
    for (const void *p : ptrs)
      if (p == nullptr || !aligned16(p)) return A3FR_ERR_INVALID_ARG;
  }
  a3fr_scene *s = new (std::nothrow) a3fr_scene();
  if (!s) return A3FR_ERR_OOM;
  s->desc = *desc;
  s->desc.tile = tile;
  s->auto_capacity = instance_capacity == 0;
  int rc = A3FR_OK;
  auto fail = [&](int code) {
    a3fr_destroy_scene(s);
    return code;
  };
  cudaError_t e = cudaMalloc(&s->small, 256);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(state)"));
  unsigned char *sm = static_cast<unsigned char *>(s->small);
  s->status = reinterpret_cast<uint32_t *>(sm + 16);
  s->counters = reinterpret_cast<unsigned long long *>(sm + 32);
  s->thresholds = reinterpret_cast<uint32_t *>(sm + 64);
  if ((e = cudaMemset(s->small, 0, 256)) != cudaSuccess) return fail(cuda_fail(e, "cudaMemset"));
  if ((e = cudaMalloc(&s->gaze_dev, sizeof(float) * 4 * kSlots)) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMalloc(gaze)"));
  if ((e = cudaMemset(s->gaze_dev, 0, sizeof(float) * 4 * kSlots)) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMemset(gaze)"));
  if ((e = cudaMallocHost(&s->gaze_pinned, sizeof(float) * 4 * kSlots)) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMallocHost(gaze)"));
  for (int k = 0; k < kSlots; ++k) {
    if ((e = cudaEventCreateWithFlags(&s->gaze_written[k], cudaEventDisableTiming)) != cudaSuccess)
      return fail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaEventCreateWithFlags(&s->gaze_consumed[k], cudaEventDisableTiming)) != cudaSuccess)
      return fail(cuda_fail(e, "cudaEventCreate"));
  }
  if ((e = cudaMalloc(&s->params_dev, sizeof(DevParams))) != cudaSuccess ||
      (e = cudaMallocHost(&s->params_pinned, sizeof(DevParams) * kSlots)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->render_done, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMalloc(params)"));
  for (int k = 0; k < kSlots; ++k)
    if ((e = cudaEventCreateWithFlags(&s->params_copied[k], cudaEventDisableTiming)) != cudaSuccess)
      return fail(cuda_fail(e, "cudaEventCreate(params)"));
  if ((e = cudaMalloc(&s->round_state, sizeof(RoundState))) != cudaSuccess ||
      (e = cudaMalloc(&s->round_plan, sizeof(RoundPlan))) != cudaSuccess ||
      (e = cudaMemset(s->round_state, 0, sizeof(RoundState))) != cudaSuccess ||
      (e = cudaMemset(s->round_plan, 0, sizeof(RoundPlan))) != cudaSuccess)
    return fail(cuda_fail(e, "cudaMalloc(round state)"));
  if ((e = cudaHostAlloc(&s->mbox_host, sizeof(Mailbox), cudaHostAllocMapped)) != cudaSuccess ||
      (e = cudaHostAlloc(&s->status_host, sizeof(RoundStatus), cudaHostAllocMapped)) != cudaSuccess)
    return fail(cuda_fail(e, "cudaHostAlloc(mailbox)"));
  std::memset(s->mbox_host, 0, sizeof(Mailbox));
  std::memset(s->status_host, 0, sizeof(RoundStatus));
  if ((e = cudaHostGetDevicePointer(&s->mbox_dev, s->mbox_host, 0)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&s->status_dev, s->status_host, 0)) != cudaSuccess)
    return fail(cuda_fail(e, "cudaHostGetDevicePointer(mailbox)"));
  if (!s->auto_capacity) {
    rc = alloc_instances(s, instance_capacity);
    if (rc != A3FR_OK) return fail(rc);
  }
  *out = s;
  return A3FR_OK;
}

int a3fr_destroy_scene(a3fr_scene *s) {
  if (!s) return A3FR_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  free_timing(s);
  free_frame_buffers(s);
  free_instance_buffers(s);
  dfree(s->frame_ws);
  dfree(s->g2d);
  dfree(s->gaze_dev);
  dfree(s->round_state);
  dfree(s->round_plan);
  dfree(s->params_dev);
  if (s->params_pinned) cudaFreeHost(s->params_pinned);
  for (int k = 0; k < kSlots; ++k)
    if (s->params_copied[k]) cudaEventDestroy(s->params_copied[k]);
  if (s->render_done) cudaEventDestroy(s->render_done);
  if (s->g_pre) cudaGraphExecDestroy(s->g_pre);
  if (s->g_fov) cudaGraphExecDestroy(s->g_fov);
  if (s->g_full) cudaGraphExecDestroy(s->g_full);
  if (s->capture_stream) cudaStreamDestroy(s->capture_stream);
  if (s->mbox_host) cudaFreeHost(s->mbox_host);
  if (s->status_host) cudaFreeHost(s->status_host);
  if (s->small) cudaFree(s->small);
  if (s->gaze_pinned) cudaFreeHost(s->gaze_pinned);
  for (int k = 0; k < kSlots; ++k) {
    if (s->gaze_written[k]) cudaEventDestroy(s->gaze_written[k]);
    if (s->gaze_consumed[k]) cudaEventDestroy(s->gaze_consumed[k]);
  }
  delete s;
  return A3FR_OK;
}

int a3fr_set_camera(a3fr_scene *s, int eye, const a3fr_camera *cam) {
  if (!s || !cam || eye < 0 || eye >= kMaxEyes) return A3FR_ERR_INVALID_ARG;
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return A3FR_ERR_INVALID_ARG;
  if (!(cam->fx > 0.0f) || !(cam->fy > 0.0f) || !(cam->znear > 0.0f)) return A3FR_ERR_INVALID_ARG;
  s->cams[eye] = *cam;
  s->cam_set[eye] = true;
  return A3FR_OK;
}

int a3fr_set_gaze(a3fr_scene *s, const float *gaze_px, void *side_stream) {
  if (!s || !gaze_px) return A3FR_ERR_INVALID_ARG;
  const int eyes = n_eyes_of(s);
  if (eyes == 0) return A3FR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(side_stream);
  const int slot = (s->gaze_seq + 1) % kSlots;
  // the pinned staging slot is reused only after its previous copy finished
  if (s->slot_written[slot]) A3FR_CHECK(cudaEventSynchronize(s->gaze_written[slot]));
  // the device slot is overwritten only after the render that read it
  if (s->slot_consumed[slot]) A3FR_CHECK(cudaStreamWaitEvent(st, s->gaze_consumed[slot], 0));
  float *h = s->gaze_pinned + 4 * slot;
  for (int k = 0; k < 4; ++k) h[k] = k < 2 * eyes ? gaze_px[k] : 0.0f;
  A3FR_CHECK(cudaMemcpyAsync(s->gaze_dev + 4 * slot, h, sizeof(float) * 4,
                             cudaMemcpyHostToDevice, st));
  A3FR_CHECK(cudaEventRecord(s->gaze_written[slot], st));
  s->slot_written[slot] = true;
  s->gaze_seq++;
  return A3FR_OK;
}

int a3fr_render_foveated(a3fr_scene *s, const a3fr_fovea *fovea, float *out_rgb, void *stream) {
  if (!s || !fovea) return A3FR_ERR_INVALID_ARG;
  return render(s, fovea, out_rgb, static_cast<cudaStream_t>(stream), Mode::kFoveated);
}

int a3fr_render_full(a3fr_scene *s, float *out_rgb, void *stream) {
  if (!s) return A3FR_ERR_INVALID_ARG;
  return render(s, nullptr, out_rgb, static_cast<cudaStream_t>(stream), Mode::kFull);
}

int a3fr_begin_frame(a3fr_scene *s, const a3fr_fovea *fovea, const a3fr_rounds *rounds,
                     float *out_rgb, void *stream) {
  if (!s || !fovea || !rounds || !out_rgb) return A3FR_ERR_INVALID_ARG;
  if (rounds->n_exits < 1 || rounds->n_exits > A3FR_MAX_EXITS || !(rounds->sir_step_px >= 0.0f))
    return A3FR_ERR_INVALID_ARG;
  for (int i = 0; i < rounds->n_exits; ++i)
    if (!(rounds->expected_dist_px[i] >= 0.0f)) return A3FR_ERR_INVALID_ARG;
  const int eyes = n_eyes_of(s);
  if (eyes == 0) return A3FR_ERR_INVALID_ARG;
  RoundConfig c{};
  c.n_eyes = eyes;
  c.n_exits = rounds->n_exits;
  c.sir = rounds->sir != 0;
  c.step = rounds->sir_step_px;
  c.n_layers = fovea->n_layers;
  for (int i = 0; i < rounds->n_exits; ++i) c.expected[i] = rounds->expected_dist_px[i];
  for (int e = 0; e < eyes; ++e)
    for (int k = 0; k < 3; ++k) c.rf[e][k] = std::sqrt(layer_radius2(s->cams[e].fx,
                                                                        fovea->theta_deg[k],
                                                                        fovea->dtheta_deg));
  s->round_ready = false;
  const int rc = render(s, fovea, out_rgb, static_cast<cudaStream_t>(stream), Mode::kFirstRound);
  if (rc != A3FR_OK) return rc;
  s->round_fovea = *fovea;
  s->round_cfg = c;
  return A3FR_OK;
}

int a3fr_post_prediction(a3fr_scene *s, int exit_index, const float *gaze_px) {
  if (!s || !gaze_px || exit_index < 1 || exit_index > A3FR_MAX_EXITS) return A3FR_ERR_INVALID_ARG;
  const int eyes = n_eyes_of(s);
  if (eyes == 0) return A3FR_ERR_INVALID_ARG;
  post_mailbox(s, exit_index, gaze_px, eyes);
  return A3FR_OK;
}

int a3fr_stall_mailbox(a3fr_scene *s, int stall) {
  if (!s) return A3FR_ERR_INVALID_ARG;
  stall_mailbox(s, stall != 0);
  return A3FR_OK;
}

int a3fr_render_round(a3fr_scene *s, float *out_rgb, void *stream) {
  if (!s) return A3FR_ERR_INVALID_ARG;
  return render_round(s, out_rgb, static_cast<cudaStream_t>(stream));
}

int a3fr_get_round_status(a3fr_scene *s, a3fr_round_status *out) {
  if (!s || !out) return A3FR_ERR_INVALID_ARG;
  const volatile RoundStatus *v = s->status_host;
  out->exit_consumed = v->exit_consumed;
  out->complete = v->complete;
  out->rounds = v->rounds;
  for (int k = 0; k < 3; ++k) out->radius_px[k] = v->radius[k];
  return A3FR_OK;
}

int a3fr_set_graph_mode(a3fr_scene *s, int on) {
  if (!s) return A3FR_ERR_INVALID_ARG;
  s->graph_mode = on != 0;
  return A3FR_OK;
}

int a3fr_set_keep_aux(a3fr_scene *s, int keep) {
  if (!s) return A3FR_ERR_INVALID_ARG;
  s->keep_aux = keep != 0;
  return A3FR_OK;
}

int a3fr_get_stats(a3fr_scene *s, a3fr_stats *st, int reset) {
  if (!s || !st) return A3FR_ERR_INVALID_ARG;
  A3FR_CHECK(cudaStreamSynchronize(s->last_stream));
  unsigned char buf[256];
  A3FR_CHECK(cudaMemcpy(buf, s->small, sizeof buf, cudaMemcpyDeviceToHost));
  uint32_t counts[4] = {0, 0, 0, 0};
  if (s->counts) A3FR_CHECK(cudaMemcpy(counts, s->counts, sizeof counts, cudaMemcpyDeviceToHost));
  uint32_t status;
  unsigned long long ctr[3];
  std::memcpy(&status, buf + 16, sizeof status);
  std::memcpy(ctr, buf + 32, sizeof ctr);
  std::memset(st, 0, sizeof *st);
  st->status = status;
  st->n_eyes = s->last_eyes;
  st->instances = counts[0];
  st->instances_eye[0] = counts[1];
  st->instances_eye[1] = s->last_eyes > 1 ? counts[3] - counts[1] : 0;
  st->capacity = (int64_t)s->capacity;
  st->evaluations = ctr[0];
  st->records_staged = ctr[1];
  st->contributions = ctr[2];
  st->renders = s->renders;
  st->kernel_launches = s->launches;
  if (reset) {
    A3FR_CHECK(cudaMemset(s->status, 0, sizeof(uint32_t)));
    A3FR_CHECK(cudaMemset(s->counters, 0, 3 * sizeof(unsigned long long)));
    s->renders = 0;
    s->launches = 0;
  }
  return A3FR_OK;
}

int a3fr_set_stage_timing(a3fr_scene *s, int ring) {
  if (!s || ring < 0 || ring > 65536) return A3FR_ERR_INVALID_ARG;
  if (s->timing_ring) A3FR_CHECK(cudaStreamSynchronize(s->last_stream));
  free_timing(s);
  if (ring == 0) return A3FR_OK;
  const int count = ring * (A3FR_N_STAGES + 1);
  s->timing_events = new (std::nothrow) cudaEvent_t[count]();
  if (!s->timing_events) return A3FR_ERR_OOM;
  s->timing_ring = ring;
  for (int i = 0; i < count; ++i) {
    cudaError_t e = cudaEventCreate(&s->timing_events[i]);
    if (e != cudaSuccess) {
      free_timing(s);
      return cuda_fail(e, "cudaEventCreate(timing)");
    }
  }
  return A3FR_OK;
}

int a3fr_get_stage_times(a3fr_scene *s, int max_renders, float *ms, int *n_out) {
  if (!s || !ms || !n_out || max_renders < 0) return A3FR_ERR_INVALID_ARG;
  *n_out = 0;
  if (!s->timing_ring) return A3FR_OK;
  A3FR_CHECK(cudaStreamSynchronize(s->last_stream));
  uint64_t avail = s->timed_renders < (uint64_t)s->timing_ring ? s->timed_renders
                                                                 : (uint64_t)s->timing_ring;
  if (avail > (uint64_t)max_renders) avail = (uint64_t)max_renders;
  for (uint64_t r = 0; r < avail; ++r) {
    const uint64_t idx = s->timed_renders - avail + r;
    const int slot = (int)(idx % (uint64_t)s->timing_ring);
    cudaEvent_t *ev = s->timing_events + slot * (A3FR_N_STAGES + 1);
    for (int k = 0; k < A3FR_N_STAGES; ++k) {
      float t = 0.0f;
      A3FR_CHECK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
      ms[r * A3FR_N_STAGES + k] = t;
    }
  }
  *n_out = (int)avail;
  return A3FR_OK;
}

int a3fr_copy_buffer(a3fr_scene *s, int which, void *dst, size_t bytes, size_t *needed,
                     void *stream) {
  if (!s) return A3FR_ERR_INVALID_ARG;
  const int eyes = s->alloc_eyes;
  const size_t n = (size_t)s->desc.n;
  const void *src = nullptr;
  size_t size = 0;
  uint32_t cnt = 0;
  if (which == A3FR_BUF_KEYS || which == A3FR_BUF_VALUES) {
    A3FR_CHECK(cudaStreamSynchronize(s->last_stream));
    if (s->counts) A3FR_CHECK(cudaMemcpy(&cnt, s->counts, sizeof cnt, cudaMemcpyDeviceToHost));
  }
  switch (which) {
    case A3FR_BUF_RECORDS: src = s->rec; size = sizeof(float) * kRec * n * eyes; break;
    case A3FR_BUF_RECTS: src = s->rect; size = sizeof(ushort4) * n * eyes; break;
    case A3FR_BUF_KEYS: size = sizeof(uint64_t) * cnt; break;   // built on demand below
    case A3FR_BUF_VALUES: src = s->vals; size = sizeof(uint32_t) * cnt; break;
    case A3FR_BUF_RANGES: src = s->ranges; size = sizeof(uint2) * (size_t)s->n_tiles * eyes; break;
    case A3FR_BUF_LEVELS: src = s->levels; size = (size_t)s->n_tiles * eyes; break;
    case A3FR_BUF_T_FINAL: src = s->t_final; size = sizeof(float) * (size_t)s->W * s->H * eyes; break;
    case A3FR_BUF_N_CONTRIB: src = s->n_contrib; size = sizeof(uint32_t) * (size_t)s->W * s->H * eyes; break;
    case A3FR_BUF_DEPTH: src = s->depth; size = sizeof(float) * (size_t)s->W * s->H * eyes; break;
    default: return A3FR_ERR_INVALID_ARG;
  }
  if (needed) *needed = size;
  if (dst == nullptr) return bytes == 0 ? A3FR_OK : A3FR_ERR_INVALID_ARG;
  if (bytes > size) return A3FR_ERR_INVALID_ARG;
  if (bytes == 0) return A3FR_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (which == A3FR_BUF_KEYS) {
    // the render sorts tile indices; the 64-bit (tile << 32 | depth bits) keys are rebuilt
    A3FR_CHECK(launch_materialize_keys(s->ranges, eyes * s->n_tiles, s->vals, s->rec, s->desc.n,
                                       s->n_tiles,
                                       (uint32_t)(bytes / sizeof(uint64_t)),
                                       static_cast<uint64_t *>(dst), st));
    return A3FR_OK;
  }
  A3FR_CHECK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
  return A3FR_OK;
}

size_t a3fr_sort_pairs_workspace_bytes(size_t n) { return sort_workspace_bytes(n) + 256; }

int a3fr_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                    size_t n, int key_bits, void *workspace, size_t workspace_bytes,
                    void *stream) {
  if (n == 0) return A3FR_OK;
  if (!keys || !vals || !keys_alt || !vals_alt || !workspace) return A3FR_ERR_INVALID_ARG;
  if (key_bits < 1 || key_bits > 64 || n >= (1u << 30)) return A3FR_ERR_INVALID_ARG;
  if (workspace_bytes < a3fr_sort_pairs_workspace_bytes(n)) return A3FR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the first 256 bytes hold the device-resident count and the status word
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *d_count = reinterpret_cast<uint32_t *>(ws);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws + 16);
  const uint32_t n32 = (uint32_t)n;
  A3FR_CHECK(cudaMemsetAsync(ws, 0, 256, st));
  A3FR_CHECK(cudaMemcpyAsync(d_count, &n32, sizeof n32, cudaMemcpyHostToDevice, st));
  bool in_alt = false;
  A3FR_CHECK(launch_sort(keys, vals, keys_alt, vals_alt, d_count, n, key_bits, ws + 256, status,
                         &in_alt, st));
  if (in_alt) {
    A3FR_CHECK(cudaMemcpyAsync(keys, keys_alt, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
    A3FR_CHECK(cudaMemcpyAsync(vals, vals_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
  }
  // a look-back wait that gave up leaves partitions scattered to wrong offsets: read the
  // status word once the sort has finished and report it
  uint32_t host_status = 0;
  A3FR_CHECK(cudaMemcpyAsync(&host_status, status, sizeof host_status, cudaMemcpyDeviceToHost, st));
  A3FR_CHECK(cudaStreamSynchronize(st));
  return (host_status & kStatusTimeout) ? A3FR_ERR_TIMEOUT : A3FR_OK;
}

const char *a3fr_error_string(int code) {
  switch (code) {
    case A3FR_OK: return "A3FR_OK";
    case A3FR_ERR_INVALID_ARG: return "A3FR_ERR_INVALID_ARG: invalid argument";
    case A3FR_ERR_CUDA: return "A3FR_ERR_CUDA: a CUDA runtime call failed";
    case A3FR_ERR_OOM: return "A3FR_ERR_OOM: out of memory";
    case A3FR_ERR_CAPACITY: return "A3FR_ERR_CAPACITY: instance capacity exceeded";
    case A3FR_ERR_TIMEOUT: return "A3FR_ERR_TIMEOUT: a bounded device wait gave up";
    case A3FR_ERR_NOT_READY: return "A3FR_ERR_NOT_READY: no gaze has been posted";
    default: return "unknown A3FR error code";
  }
}

const char *a3fr_last_error_detail(void) { return g_detail.c_str(); }


int a3fr_backward(a3fr_scene *s, const float *dl_drgb, const a3fr_grads *g, void *stream) {
  if (!s || !dl_drgb || !g) return A3FR_ERR_INVALID_ARG;
  const int n = s->desc.n;
  if (n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
    return A3FR_ERR_INVALID_ARG;
  if (s->bw_mode == 0 || s->last_eyes == 0) return A3FR_ERR_NOT_READY;
  if (n == 0) return A3FR_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int eyes = s->last_eyes;
  const size_t need = backward_g2d_floats(eyes, n);
  if (s->g2d_floats < need) {
    dfree(s->g2d);
    s->g2d_floats = 0;
    cudaError_t e = cudaMalloc(&s->g2d, sizeof(float) * need);
    if (e != cudaSuccess) {
      s->g2d = nullptr;
      return cuda_fail(e, "cudaMalloc(backward workspace)");
    }
    s->g2d_floats = need;
  }
  BackwardParams bp{};
  bp.n_eyes = eyes;
  bp.n = n;
  bp.width = s->cams[0].width;
  bp.height = s->cams[0].height;
  bp.tile = s->desc.tile;
  bp.tiles_x = s->TX;
  bp.n_tiles = s->n_tiles;
  A3FR_CHECK(launch_backward(bp, &s->params_dev->pre, s->desc.sh_degree, s->desc.means,
                             s->desc.log_scales, s->desc.quats, s->desc.opacity_logits, s->desc.sh,
                             s->rec, s->ranges, s->counts, s->vals,
                             s->bw_mode == 2 ? s->levels : nullptr, s->t_final, s->n_contrib,
                             dl_drgb, s->g2d, g->means, g->log_scales, g->quats, g->opacity_logits,
                             g->sh, st));
  s->launches += 2;
  return A3FR_OK;
}


int a3fr_set_tile(a3fr_scene *s, int tile) {
  if (!s || (tile != 16 && tile != 32)) return A3FR_ERR_INVALID_ARG;
  if (s->desc.tile == tile) return A3FR_OK;
  A3FR_CHECK(cudaDeviceSynchronize());
  free_frame_buffers(s);
  if (s->auto_capacity) {   // the instance count changes with the tile: measure it again
    free_instance_buffers(s);
    s->capacity = 0;
  }
  s->desc.tile = tile;
  s->alloc_gen++;
  s->bw_mode = 0;
  return A3FR_OK;
}

int a3fr_set_binning(a3fr_scene *s, int mode) {
  if (!s || mode < A3FR_BINNING_AUTO || mode > A3FR_BINNING_SORTED) return A3FR_ERR_INVALID_ARG;
  if (s->binning == mode) return A3FR_OK;
  A3FR_CHECK(cudaDeviceSynchronize());
  free_frame_buffers(s);
  free_sort_buffers(s);
  s->binning = mode;
  s->alloc_gen++;
  s->bw_mode = 0;
  return A3FR_OK;
}

int a3fr_set_batch(a3fr_scene *s, int batch_mult) {
  if (!s || (batch_mult != 1 && batch_mult != 2)) return A3FR_ERR_INVALID_ARG;
  if (s->batch_mult != batch_mult) {
    s->batch_mult = batch_mult;
    s->alloc_gen++;   // captured composite graphs hold the kernel choice
  }
  return A3FR_OK;
}

int a3fr_autotune(a3fr_scene *s, const a3fr_fovea *fovea, float *out_rgb, int timed_renders,
                  void *stream, a3fr_tune_result *result) {
  if (!s || !fovea || !out_rgb || !result || timed_renders < 1) return A3FR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  *result = a3fr_tune_result{};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return A3FR_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return A3FR_ERR_CUDA;
  }
  const int tiles[2] = {16, 32}, mults[2] = {1, 2};
  float best = 1e30f;
  int rc = A3FR_OK;
  for (int ti = 0; ti < 2 && rc == A3FR_OK; ++ti) {
    for (int mi = 0; mi < 2 && rc == A3FR_OK; ++mi) {
      rc = a3fr_set_tile(s, tiles[ti]);
      if (rc == A3FR_OK) rc = a3fr_set_batch(s, mults[mi]);
      for (int w = 0; w < 2 && rc == A3FR_OK; ++w) rc = a3fr_render_foveated(s, fovea, out_rgb, stream);
      if (rc != A3FR_OK) break;
      if (cudaEventRecord(e0, st) != cudaSuccess) { rc = A3FR_ERR_CUDA; break; }
      for (int r = 0; r < timed_renders && rc == A3FR_OK; ++r) rc = a3fr_render_foveated(s, fovea, out_rgb, stream);
      if (rc != A3FR_OK) break;
      float ms = 0.0f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = A3FR_ERR_CUDA;
        break;
      }
      ms /= (float)timed_renders;
      result->ms[ti][mi] = ms;
      if (ms < best) {
        best = ms;
        result->tile = tiles[ti];
        result->batch_mult = mults[mi];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != A3FR_OK) return rc;
  rc = a3fr_set_tile(s, result->tile);
  if (rc == A3FR_OK) rc = a3fr_set_batch(s, result->batch_mult);
  return rc;
}

}  // extern "C"
