/*
 * a3fr.h -- C ABI of libA3FR.so, the GB300 (sm_103a) foveated 3D Gaussian Splatting
 * forward rasterizer of A3FR (arXiv 2507.04147).
 *
 * What one render computes (per eye), in the paper's order:
 *   projection of every Gaussian to a 2-D ellipse and its tile overlap (Sec. 2.3,
 *   "Projection"), a per-tile depth sort (Sec. 2.3, "Sorting"), front-to-back
 *   volume rendering of each pixel (Sec. 2.3, "Rasterization"), with the tiles
 *   labelled by eccentricity from the gaze (Eq. 1, Sec. 3.4) so that a level-k tile
 *   renders k of the 4 pixels of every 2x2 block and the other pixels inherit the
 *   block's top-left pixel or are interpolated (Sec. 3.4, Sec. 3.5).  All foveation layers of all eyes
 *   form one canvas, written in one pass.
 *
 * Conventions shared by every entry point:
 *   - Every call returns A3FR_OK (0) or a negative A3FR_ERR_* code; nothing is thrown
 *     across the ABI and the library never exits the process.
 *   - Pointers documented as DEVICE point to global memory of the current CUDA
 *     device; pointers documented as HOST are ordinary host memory.
 *   - `stream` arguments are cudaStream_t handles passed as void* (NULL = the legacy
 *     default stream).  Rendering is asynchronous on that stream; the caller keeps
 *     inputs alive and outputs untouched until the stream reaches the render.
 *   - Device-side failures (instance-capacity overflow, a bounded wait that gave up)
 *     set bits of a per-scene status word; a3fr_get_stats reads it.
 *   - One scene is used by one host thread at a time.
 */
#ifndef A3FR_H
#define A3FR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define A3FR_OK 0
#define A3FR_ERR_INVALID_ARG (-1) /* a null pointer, a size out of range, an unset camera */
#define A3FR_ERR_CUDA (-2)        /* a CUDA runtime call failed; see a3fr_last_error_detail */
#define A3FR_ERR_OOM (-3)         /* device or pinned-host allocation failed */
#define A3FR_ERR_CAPACITY (-4)    /* more tile-Gaussian instances than the scene's capacity */
#define A3FR_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define A3FR_ERR_NOT_READY (-6)   /* render_foveated before any set_gaze */

/* bits of a3fr_stats.status */
#define A3FR_STATUS_CAPACITY 1u   /* some instances were dropped: the image is incomplete */
#define A3FR_STATUS_TIMEOUT 2u    /* a look-back wait (radix sort, binning) gave up */

typedef struct a3fr_scene a3fr_scene; /* opaque, library-owned */

/* The Gaussians of a scene (Sec. 2.3: position, scales, rotation, opacity, SH colour).
 * All arrays are DEVICE fp32, caller-owned and borrowed: they must stay allocated and
 * unchanged while the scene renders.  Arrays must be 16-byte aligned. */
typedef struct {
  int32_t n;                    /* number of Gaussians, 0 <= n < 2^30 */
  int32_t sh_degree;            /* 0..3 */
  int32_t tile;                 /* tile edge in pixels: 16 or 32 (0 selects 16) */
  int32_t reserved;             /* must be 0 */
  const float *means;           /* [n][3] world position */
  const float *log_scales;      /* [n][3] log standard deviation per axis */
  const float *quats;           /* [n][4] rotation (w, x, y, z); normalised by the library */
  const float *opacity_logits;  /* [n] opacity = sigmoid(logit) */
  const float *sh;              /* [n][(sh_degree+1)^2][3] SH coefficients, channel fastest */
} a3fr_scene_desc;

/* Pinhole camera: x_cam = R x_world + t with world_to_cam = [R | t] row-major 3x4;
 * pixel (i, j) samples the image plane at (i, j); +z forward, +y down. */
typedef struct {
  int32_t width, height;        /* pixels, 1..16384 */
  float fx, fy, cx, cy;         /* focal lengths and principal point, pixels */
  float znear;                  /* Gaussians with camera depth <= znear are culled */
  float world_to_cam[12];
} a3fr_camera;

/* Foveation layers (Eq. 1, Sec. 3.4).  Layer k < n_layers-1 covers the tiles whose
 * nearest pixel centre lies within r_k = fx * tan(theta_deg[k] + dtheta_deg) pixels
 * of the gaze (and not within an inner layer); the last layer covers the rest.
 * Layer k renders its tiles at pixel-density level level[k] in 1..4. */
typedef struct {
  int32_t n_layers;             /* 1..4 */
  float theta_deg[3];           /* increasing eccentricity boundaries, degrees */
  float dtheta_deg;             /* gaze-tracking error margin of Eq. 1, degrees */
  int32_t level[4];             /* e.g. {4, 2, 1} for three layers */
  int32_t fill;                 /* skipped pixels (Sec. 3.4 "inherit or interpolate"): 0 inherit the
                                   block's top-left pixel; 1 interpolate: the mean of the pixel's
                                   rendered 4-neighbours (up, down, left, right), else of its rendered
                                   diagonal neighbours, else the top-left pixel (a3fr_render_foveated
                                   only; rounds inherit) */
  float count_frac;             /* tile levels by Gaussian count (Sec. 3.6, 4.6: tiles sorted by their
                                   number of Gaussians, resolution adjusted): per eye, the
                                   floor(count_frac * tiles) tiles with the most instances (every tile
                                   whose count is >= the k-th largest) drop one level if their level is
                                   2 or 3; 0 = off; in [0, 1].  a3fr_render_foveated only
                                   (the rounds API ignores it). */
} a3fr_fovea;

typedef struct {
  uint32_t status;              /* A3FR_STATUS_* bits accumulated since the last reset */
  int32_t n_eyes;               /* eyes rendered by the last render */
  int64_t instances;            /* tile-Gaussian pairs of the last render (all eyes) */
  int64_t instances_eye[2];     /* the same per eye */
  int64_t capacity;             /* instance capacity of the scene */
  uint64_t evaluations;         /* (pixel, Gaussian) evaluations since the last reset: each
                                   rendered pixel's position in its tile's list where it
                                   stopped (or the list length); counted by renders with
                                   keep_aux on only (0 otherwise) */
  uint64_t records_staged;      /* Gaussian records staged by tile blocks since the reset */
  uint64_t renders;             /* renders since the last reset */
  uint64_t kernel_launches;     /* kernels this library launched since the last reset */
  uint64_t contributions;       /* (pixel, Gaussian) blends since the last reset, counted by
                                   renders with keep_aux on only (0 otherwise) */
} a3fr_stats;

/* Create a scene over caller-owned Gaussians.  instance_capacity bounds the number of
 * tile-Gaussian pairs per render over all eyes; 0 sizes it at the first render from the
 * measured count (that render synchronises once).  *out receives the scene. */
int a3fr_create_scene(const a3fr_scene_desc *desc, size_t instance_capacity, a3fr_scene **out);

/* Free the scene and its library-owned device workspace (synchronises the device). */
int a3fr_destroy_scene(a3fr_scene *scene);

/* Set the camera of eye 0 or 1 (copied; HOST struct).  The eyes rendered are 0..k where
 * k is the highest eye with a camera; all eyes must have the same width and height. */
int a3fr_set_camera(a3fr_scene *scene, int eye, const a3fr_camera *camera);

/* Post the gaze of every eye, HOST float[n_eyes][2] in pixels, into the scene's device
 * mailbox: an asynchronous host-to-device copy on side_stream followed by an event.  A
 * later render_foveated waits for that event before its first gaze-dependent step
 * (Sec. 3.3.3: the latest gaze prediction is stored in GPU memory). */
int a3fr_set_gaze(a3fr_scene *scene, const float *gaze_px, void *side_stream);

/* Render every eye foveated into out_rgb, DEVICE fp32 [n_eyes][height][width][3]. */
int a3fr_render_foveated(a3fr_scene *scene, const a3fr_fovea *fovea, float *out_rgb,
                         void *stream);

/* Render every eye at full resolution (every tile at level 4, no gaze), same layout. */
int a3fr_render_full(a3fr_scene *scene, float *out_rgb, void *stream);

/* Synchronise the scene's last stream and report counters; reset != 0 clears them. */
int a3fr_get_stats(a3fr_scene *scene, a3fr_stats *stats, int reset);

/* ---- incremental rendering rounds (Sec. 3.3, Algorithm 1) ----
 * A frame is rendered in rounds while the gaze tracker refines its prediction: the first
 * round does the buffered precompute (projection, sorts, tile ranges; Sec. 3.5) and renders
 * every tile at the peripheral level; each later round reads the latest prediction u_i from a
 * mailbox in mapped host memory when it runs on the GPU and renders only the pixels its
 * region adds (labels above each tile's current level), never a pixel twice. */
#define A3FR_MAX_EXITS 8

typedef struct {
  int32_t n_exits;                 /* N, the number of tracker exits, 1..A3FR_MAX_EXITS */
  int32_t sir;                     /* 1: speculative rounds when no new prediction arrived */
  float expected_dist_px[A3FR_MAX_EXITS]; /* E[dist(u_i, u_N)] in pixels, exit i at [i-1];
                                      the last one should be 0 */
  float sir_step_px;               /* growth of the radii per speculative round, pixels */
} a3fr_rounds;

typedef struct {
  int32_t exit_consumed;           /* exit of the prediction the last round used, 0 = none */
  int32_t complete;                /* 1 once the final exit's region has been rendered */
  int32_t rounds;                  /* rounds that rendered something, this frame */
  float radius_px[3];              /* layer radii of eye 0 in the last round */
} a3fr_round_status;

/* Round 1 of a frame: the full precompute for the current cameras and every tile rendered at
 * the peripheral level (fovea->level[n_layers - 1]) into out_rgb (DEVICE [eyes][H][W][3],
 * which later rounds keep refining).  Clears the mailbox and the round state.  The final
 * layer radii are those of `fovea` (Eq. 1). */
int a3fr_begin_frame(a3fr_scene *scene, const a3fr_fovea *fovea, const a3fr_rounds *rounds,
                     float *out_rgb, void *stream);

/* Post prediction u_i (exit_index i in 1..N, HOST float[eyes][2] pixels) into the mailbox.
 * Callable from any host thread at any time, without a CUDA call (sequence-locked write into
 * mapped pinned memory). */
int a3fr_post_prediction(a3fr_scene *scene, int exit_index, const float *gaze_px);

/* One later round on `stream` (after a3fr_begin_frame, same out_rgb).  When it runs, a new
 * prediction u_i renders the region of radii max(0, r_{k,N} - E_i) around u_i (Eq. 3'); with
 * no new prediction and SIR on, the region around the last prediction u_j grows by
 * sir_step_px up to r_{k,N} + E_j (Eq. 4); otherwise nothing is rendered.  Returns
 * A3FR_ERR_NOT_READY without a begun frame. */
int a3fr_render_round(a3fr_scene *scene, float *out_rgb, void *stream);

/* Status of the last completed round, read from mapped host memory (no synchronisation). */
int a3fr_get_round_status(a3fr_scene *scene, a3fr_round_status *status);

/* Fault injection on the host (Sec. 3.3: the tracker runs on a CPU that other work can slow
 * down).  stall != 0 begins a write of the prediction mailbox and leaves it unfinished, as
 * when the tracker thread is descheduled in the middle of a write: the sequence word stays
 * odd, and predictions posted meanwhile update the payload without publishing it.  A round
 * that runs meanwhile polls the mailbox a bounded number of times (2^16), then gives up,
 * sets A3FR_STATUS_TIMEOUT in the scene's status word (a3fr_get_stats) and keeps the last
 * prediction it consumed -- with SIR on it grows the region around that prediction (Eq. 4)
 * instead of waiting.  stall == 0 finishes the write and publishes the latest payload.
 * Nothing on the GPU hangs or faults. */
int a3fr_stall_mailbox(a3fr_scene *scene, int stall);

/* ---- one frame of Algorithm 1, natively timed ---- */
#define A3FR_DRIVE_A3FR 0  /* rounds overlapped with tracking (SIR per rounds->sir) */
#define A3FR_DRIVE_SFR 1   /* sequential: wait for the final prediction, then render foveated */
#define A3FR_DRIVE_FRR 2   /* full resolution, no tracking */

typedef struct {
  int32_t mode;                    /* A3FR_DRIVE_* */
  int32_t n_exits;                 /* must equal rounds->n_exits */
  const float *predictions;        /* HOST [n_exits][eyes][2]: u_1..u_N in pixels */
  const double *exit_time_us;      /* HOST [n_exits]: time each prediction is ready, unloaded */
  double load_period_us;           /* > 0: tracker intervals in every odd period are stretched */
  double load_factor;              /*   by this factor (alternating CPU load, Sec. 4.5) */
  int32_t max_rounds;              /* bound on the rounds launched after the first */
} a3fr_frame_driver;

typedef struct {
  double latency_us;               /* frame start -> completion of its last needed GPU work */
  double tracker_end_us;           /* when the tracker thread posted its last prediction */
  int32_t rounds;                  /* rounds launched after the first (1 for SFR/FRR) */
  int32_t exit_per_round[16];      /* exit consumed by each of the first 16 rounds */
  double round_end_us[16];         /* completion time of each of the first 16 rounds */
} a3fr_frame_result;

/* Render one frame the way Algorithm 1 runs its two processes: a host thread posts
 * drv->predictions at drv->exit_time_us (process 1) while this thread begins the frame and
 * launches rounds until the final prediction's region is rendered (process 2); a round
 * without a new prediction speculates (Eq. 4) when rounds->sir is set and the region can
 * still grow, otherwise this thread waits for the next prediction.  SFR and FRR modes run the
 * sequential and full-resolution baselines with the same clock.  Synchronous; the cameras
 * must be set. */
int a3fr_run_frame(a3fr_scene *scene, const a3fr_fovea *fovea, const a3fr_rounds *rounds,
                   const a3fr_frame_driver *driver, float *out_rgb, void *stream,
                   a3fr_frame_result *result);

/* Graph mode (default off): renders replay two captured CUDA graphs -- the precompute and
 * the composite (foveated or full) -- instead of launching ~20 operations each; the gaze wait
 * sits between them, so the precompute still overlaps the tracker.  Per-render parameters
 * (cameras, layer radii, gaze slot, output pointer) live in device memory and one copy per
 * render updates them.  Graphs are captured at the first render that can use them and again
 * whenever a workspace buffer moves; the first render of an automatic-capacity scene and
 * the rounds API launch directly (with stage timing on, a graph-mode render is timed around
 * its two graphs: see a3fr_set_stage_timing). */
int a3fr_set_graph_mode(a3fr_scene *scene, int on);

/* ------------------------------------------------------------------ tiling and tuning
 * Tile size (16 or 32 pixels; the paper tiles 32 x 32, Sec. 3.5): with 32, every label of a
 * tile is its own 256-thread CTA and only the labels a tile's level needs are launched.  The
 * per-thread staging batch (1 or 2 Gaussians per thread per shared-memory batch) trades
 * barrier count for shared memory.  Changing either invalidates the scene's buffers and
 * captured graphs (the next render reallocates); synchronous. */
int a3fr_set_tile(a3fr_scene *scene, int tile);
int a3fr_set_batch(a3fr_scene *scene, int batch_mult);

/* Binning path (Sec. 2.3 tile binning; both give the same tile lists bit for bit).  DIRECT:
 * the depth-ordered entries cut into chunks, per-chunk tile counts and start slots, every
 * instance placed at its slot by ordered ranks (no sort over the instances).  SORTED: tile
 * counts, emit of the depth-ordered instances, a stable radix sort by tile.  AUTO (default):
 * DIRECT up to 6,144 tiles over all eyes, SORTED above (where it is faster).  Changing it invalidates the scene's buffers (the next render reallocates);
 * synchronous.  Invalid mode: A3FR_ERR_INVALID_ARG. */
#define A3FR_BINNING_AUTO 0
#define A3FR_BINNING_DIRECT 1
#define A3FR_BINNING_SORTED 2
int a3fr_set_binning(a3fr_scene *scene, int mode);

typedef struct {
  int32_t tile, batch_mult;   /* the configuration chosen (and left set on the scene) */
  float ms[2][2];             /* mean foveated render time per (tile 16|32, batch 1|2) */
} a3fr_tune_result;

/* Autotuner (not in the paper, which fixes its tiling by hand): renders the scene foveated
 * with the current cameras and gaze under every (tile, batch) configuration -- 2 warm-up
 * and timed_renders timed renders each, CUDA events on `stream` -- and keeps the fastest.
 * out_rgb as for a3fr_render_foveated; synchronous. */
int a3fr_autotune(a3fr_scene *scene, const a3fr_fovea *fovea, float *out_rgb, int timed_renders,
                  void *stream, a3fr_tune_result *result);

/* ---------------------------------------------------------------- backward rasterizer
 * Gradients of L = sum(dl_drgb * image) with respect to the scene parameters, for the last
 * render of this scene (3DGS training, Sec. 4.1 "Training": the rasterizer's forward pass
 * differentiated through compositing, projection and SH colour of Sec. 2.3).
 *
 * grads: DEVICE pointers, caller-owned, same layouts and sizes as the scene description
 *   (means [n][3], log_scales [n][3], quats [n][4], opacity_logits [n], sh [n][(deg+1)^2][3]);
 *   every element is overwritten (culled Gaussians get zeros).  With two eyes the
 *   gradients of both eyes' images are summed.
 * dl_drgb: DEVICE fp32 [n_eyes][height][width][3], the gradient of L with respect to the
 *   image the last render wrote.  For a foveated render, an inherited pixel's gradient is
 *   passed to the top-left pixel of its block (the pixel it copies).
 * Preconditions: the last render of the scene was a3fr_render_full or a3fr_render_foveated
 *   with keep_aux on (its final transmittance and last contributor per pixel are what the
 *   backward walks from; per-pixel transmittance is recomputed back to front, not stored),
 *   no round has run since, the scene's parameter arrays are unchanged since that render,
 *   and `stream` is ordered after it.  Otherwise A3FR_ERR_NOT_READY.
 * Asynchronous on `stream`; per-Gaussian partial sums are accumulated with float atomics,
 *   so the last bits of a gradient may differ from run to run.  Allocates a workspace of
 *   36 bytes per eye and Gaussian on first use. */
typedef struct {
  float *means, *log_scales, *quats, *opacity_logits, *sh;
} a3fr_grads;

int a3fr_backward(a3fr_scene *scene, const float *dl_drgb, const a3fr_grads *grads, void *stream);

/* ------------------------------------------------------------ tensor-core building block
 * No counterpart in the paper: the single-tile BF16 GEMM on the fifth-generation tensor
 * cores (tcgen05) that the learned-periphery kernels are built from, exported so that its
 * operand encodings can be checked on their own.  D[128][n] = A[128][k] * B[n][k]^T with
 * A, B bf16 (uint16 bit patterns) and D fp32, all DEVICE, row-major, caller-owned;
 * n in {16, 32}, k in {16, 32, 48, 64}; variant 0 is the descriptor layout the library uses,
 * variant 1 swaps its two stride fields (a wrong layout gives wrong numbers, never an
 * out-of-bounds access).  Synchronous; A3FR_ERR_TIMEOUT if the MMA never completed. */
int a3fr_tc_tile_gemm(const uint16_t *A, const uint16_t *B, float *D, int n, int k, int variant,
                      void *stream);

/* ------------------------------------------------------------------- learned periphery
 * Not in the paper (its un-rendered pixels "inherit or interpolate", Sec. 3.4): a small
 * residual CNN that predicts the pixels a foveated render skipped from the quarter-density
 * layer (the top-left pixel of every 2x2 block, which every level renders) and its expected
 * depth.  Network: 3x3 conv 16->32 + ReLU; four residual blocks (3x3 conv 32->32 + ReLU,
 * 3x3 conv 32->32, skip); 3x3 conv 32->16 whose channel c*4 + 2*dy + dx is the correction
 * of colour c at sub-pixel (dx, dy) of the block, added to the base: the bilinear
 * interpolation of the top-left pixels (the block's a, its right neighbour's, the one below,
 * the diagonal one; the last block repeated past the edge) -- a at (0, 0), (a + right) / 2,
 * (a + down) / 2, (((a + right) + down) + diag) / 4 -- i.e. the interpolating fill where
 * only top-left pixels are rendered.
 * BF16 weights and activations, FP32 accumulation, all convolutions on the tensor cores
 * (tcgen05); inputs (r, g, b, depth/8) per block.  Parameters: fp32, layer by layer the
 * weights [out][in][3][3] (layer 0's input channels 4..15 unused), then the biases; the
 * library keeps Adam state for training.  The object owns its device memory; one object per
 * host thread. */
typedef struct a3fr_cnn a3fr_cnn;

/* Architectures.  RESIDUAL: the network above.  COMPACT: 3x3 conv 16->32 + ReLU, per-block
 * layer 32->32 + ReLU, per-block layer 32->16 (same output channels and base) -- its fill is
 * one fused kernel with every activation kept on chip.  Parameters, layer by layer, the
 * weights ([out][in][3][3] for 3x3 layers, [out][in] for per-block ones), then the biases. */
#define A3FR_CNN_RESIDUAL 0
#define A3FR_CNN_COMPACT 1

size_t a3fr_cnn_param_count(void);                      /* of the RESIDUAL network */
size_t a3fr_cnn_arch_param_count(int arch);             /* 0 for an unknown architecture */
int a3fr_cnn_create(a3fr_cnn **out);                    /* RESIDUAL, zero parameters */
/* A3FR_ERR_INVALID_ARG for an unknown architecture. */
int a3fr_cnn_create_arch(a3fr_cnn **out, int arch);
int a3fr_cnn_destroy(a3fr_cnn *net);
/* host fp32 [a3fr_cnn_arch_param_count(arch of net)]; set resets the Adam state; both
 * synchronous; A3FR_ERR_INVALID_ARG when count differs */
int a3fr_cnn_set_params(a3fr_cnn *net, const float *host, size_t count);
int a3fr_cnn_get_params(a3fr_cnn *net, float *host, size_t count);
/* img: DEVICE fp32 [b][h][w][3], depth: DEVICE fp32 [b][h][w] (expected depth).  Runs the
 * network on the top-left pixels; residual_out (optional, DEVICE fp32 [b][(h+1)/2][(w+1)/2][16])
 * receives the per-block corrections.  Asynchronous on stream. */
int a3fr_cnn_forward(a3fr_cnn *net, const float *img, const float *depth, int b, int h, int w,
                     float *residual_out, void *stream);
/* Mean squared error of the prediction (base + correction at every pixel) against
 * target (DEVICE fp32 [b][h][w][3]) and its gradient with respect to every parameter, into
 * host_grads (host fp32 [a3fr_cnn_arch_param_count(arch of net)]) and *loss; synchronous. */
int a3fr_cnn_grads(a3fr_cnn *net, const float *img, const float *depth, const float *target, int b,
                   int h, int w, float *host_grads, float *loss, void *stream);
/* One Adam step (beta 0.9 / 0.999) on the same loss; *loss (optional) makes it synchronous.
 * A3FR_ERR_TIMEOUT if a tensor-core wait gave up (the step's numbers are then unreliable). */
int a3fr_cnn_train_step(a3fr_cnn *net, const float *img, const float *depth, const float *target,
                        int b, int h, int w, float lr, float *loss, void *stream);
/* Learned fill of the scene's last render, which must be a3fr_render_foveated with keep_aux
 * on (for its depth) writing out_rgb: rendered pixels are kept, every skipped pixel becomes its
 * base plus the network's correction.  A3FR_ERR_NOT_READY otherwise.
 * Asynchronous on stream (ordered after the render). */
int a3fr_cnn_fill(a3fr_cnn *net, a3fr_scene *scene, float *out_rgb, void *stream);

/* Keep per-pixel transmittance and contributor counts of the next renders (aux buffers,
 * see a3fr_copy_buffer); off by default because they cost 8 bytes per pixel. */
int a3fr_set_keep_aux(a3fr_scene *scene, int keep);

/* Stages of a render timed by a3fr_set_stage_timing, in launch order. */
#define A3FR_STAGE_PREPROCESS 0  /* projection, EWA, SH colour, tile rectangles, histograms */
#define A3FR_STAGE_DEPTH_SORT 1  /* onesweep sort of the (eye, Gaussian) entries by depth */
#define A3FR_STAGE_BIN 2         /* chunk plan, per-chunk tile counts, tile ranges, chunk starts */
#define A3FR_STAGE_EMIT 3        /* every (tile, Gaussian) instance to its slot, depth order */
#define A3FR_STAGE_COMPOSITE 4   /* level map + front-to-back blending + inheritance */
#define A3FR_N_STAGES 5

/* Record CUDA events around every stage of the next renders on their stream, keeping the
 * last `ring` renders (0 turns timing off and frees the events).  A render in graph mode
 * (a3fr_set_graph_mode) replays two graphs and is timed around them: the precompute graph
 * (and, foveated, the wait for the gaze) as A3FR_STAGE_PREPROCESS, the composite graph as
 * A3FR_STAGE_COMPOSITE; its DEPTH_SORT, BIN and EMIT stages read zero. */
int a3fr_set_stage_timing(a3fr_scene *scene, int ring);

/* Synchronise and write the stage durations (ms) of the last min(max_renders, available)
 * timed renders, oldest first, into HOST ms[k][A3FR_N_STAGES]; *n_out (HOST) receives k. */
int a3fr_get_stage_times(a3fr_scene *scene, int max_renders, float *ms, int *n_out);

/* Internal buffers of the last render that a3fr_copy_buffer can copy out. */
#define A3FR_BUF_RECORDS 1    /* fp32 [n_eyes][n][12]: u v conic(a b c) opacity r g b depth radius visible */
#define A3FR_BUF_RECTS 2      /* uint16 [n_eyes][n][4]: tile x0 y0 x1 y1, half-open */
#define A3FR_BUF_KEYS 3       /* uint64 [instances]: sorted (eye*tiles + tile) << 32 | depth bits */
#define A3FR_BUF_VALUES 4     /* uint32 [instances]: Gaussian index of each sorted key */
#define A3FR_BUF_RANGES 5     /* uint32 [n_eyes*tiles][2]: [start, end) of each tile's run */
#define A3FR_BUF_LEVELS 6     /* uint8 [n_eyes*tiles]: pixel-density level of each tile */
#define A3FR_BUF_T_FINAL 7    /* fp32 [n_eyes][height][width] (keep_aux only) */
#define A3FR_BUF_N_CONTRIB 8  /* uint32 [n_eyes][height][width] (keep_aux only) */
#define A3FR_BUF_DEPTH 9      /* fp32 [n_eyes][height][width]: expected depth sum(alpha T z) (keep_aux only) */

/* Copy `bytes` bytes of internal buffer `which` (A3FR_BUF_*) of the last render into the
 * DEVICE buffer dst, asynchronously on `stream`.  *needed (HOST, may be NULL) receives the
 * buffer's size; bytes larger than that is an error. */
int a3fr_copy_buffer(a3fr_scene *scene, int which, void *dst, size_t bytes, size_t *needed,
                     void *stream);

/* ---- building blocks on caller buffers (also used by the scene path) ---- */

/* Workspace bytes a3fr_sort_pairs needs for n pairs. */
size_t a3fr_sort_pairs_workspace_bytes(size_t n);

/* Stable least-significant-digit radix sort (8-bit digits, one onesweep pass per digit)
 * of n (key, value) pairs by the low key_bits bits of the keys (1..64): the 3DGS depth
 * sort keyed by tile and depth (Sec. 2.3, "Sorting").  keys/vals (DEVICE uint64/uint32
 * [n]) hold the input and receive the result; keys_alt/vals_alt (DEVICE, [n]) and the
 * DEVICE workspace of a3fr_sort_pairs_workspace_bytes(n) bytes are scratch.  Bits above
 * key_bits must be zero.  The sort runs on `stream`, and the call returns once it has
 * finished there: it synchronises the stream to read the device status word (bytes 16..19
 * of the workspace), and returns A3FR_ERR_TIMEOUT when a bounded look-back wait gave up --
 * the pairs are then not validly ordered.  n >= 2^30 returns A3FR_ERR_INVALID_ARG. */
int a3fr_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                    size_t n, int key_bits, void *workspace, size_t workspace_bytes,
                    void *stream);

/* Largest n accepted by a3fr_sort_pairs_noalloc. */
#define A3FR_NOALLOC_MAX_PAIRS 262144

/* The sort of a3fr_sort_pairs for callers that cannot allocate device memory -- for example
 * a real-time render thread that cannot absorb the device-wide synchronisation cudaMalloc
 * and cudaFree may cause, or code inside an engine that owns all device memory through its
 * own allocator.  The paper has no counterpart; this is a library convenience.
 *
 * keys/vals (DEVICE uint64/uint32 [n]) hold the input and receive the result, as in
 * a3fr_sort_pairs; nothing else is passed in.  The scratch (ping-pong buffers, histograms,
 * look-back words) is one fixed file-scope device array of 4,194,560 bytes (4.0 MiB:
 * 12 bytes per pair of A3FR_NOALLOC_MAX_PAIRS, 1 MiB of histograms and look-back words,
 * 256 bytes of count and status), which every GPU that loads the library holds until the
 * process exits.  This call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.
 *  - n > A3FR_NOALLOC_MAX_PAIRS returns A3FR_ERR_CAPACITY and does no work.
 *  - Like a3fr_sort_pairs, the call returns once the sort has finished on `stream` (it
 *    synchronises the stream to read the status word from the array) and returns
 *    A3FR_ERR_TIMEOUT when a bounded look-back wait gave up.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    with that device current; make that first call before any stream capture.
 *  - Every call shares the one array, so calls whose work overlaps on the GPU (on different
 *    streams, or from different threads) race and corrupt each other's results; serialise
 *    them, e.g. on one stream.  The array keeps the last call's contents; each call clears
 *    what must start at zero. */
int a3fr_sort_pairs_noalloc(uint64_t *keys, uint32_t *vals, size_t n, int key_bits,
                            void *stream);

/* Human-readable name of an A3FR_* code (static storage). */
const char *a3fr_error_string(int code);

/* Detail of the last A3FR_ERR_CUDA raised on the calling thread (static storage). */
const char *a3fr_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* A3FR_H */
