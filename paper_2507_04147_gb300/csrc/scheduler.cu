// scheduler.cu -- a3fr_run_frame: one frame of Algorithm 1 with its two processes in
// parallel, natively timed.
//
// Process 1 (gaze tracking) is a host thread that posts the early-exit predictions
// u_1..u_N into the scene's mailbox at their exit times (optionally slowed down by an
// alternating CPU load, Sec. 4.5).  Process 2 (rendering) is the calling thread: it begins
// the frame (precompute + peripheral round) and keeps launching rounds; each round picks up
// the newest prediction when it runs on the GPU.  With speculative rounds off, process 2
// waits for the next prediction before each round.  The frame ends when the round that used
// the final prediction has completed.
//
// For comparison (Sec. 4.3) the same driver runs the two baselines under the same clock:
// SFR waits for the final prediction and then renders the foveated frame; FRR renders the
// full-resolution frame without waiting for the tracker.
#include <atomic>
#include <chrono>
#include <thread>

#include "../../include/a3fr.h"
#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double us_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
}

void wait_until_us(Clock::time_point t0, double t_us) {
  while (us_since(t0) < t_us) {
    const double left = t_us - us_since(t0);
    if (left > 200.0) std::this_thread::sleep_for(std::chrono::microseconds((int64_t)(left - 100.0)));
    else std::this_thread::yield();
  }
}

// Polls an event instead of blocking, to see completion as early as possible.
cudaError_t spin_event(cudaEvent_t ev) {
  while (true) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e != cudaErrorNotReady) return e;
    std::this_thread::yield();
  }
}

}  // namespace

extern "C" int a3fr_run_frame(a3fr_scene *scene, const a3fr_fovea *fovea,
                              const a3fr_rounds *rounds, const a3fr_frame_driver *drv,
                              float *out_rgb, void *stream, a3fr_frame_result *result) {
  if (!scene || !fovea || !rounds || !drv || !out_rgb || !result) return A3FR_ERR_INVALID_ARG;
  if (drv->n_exits < 1 || drv->n_exits > A3FR_MAX_EXITS || drv->n_exits != rounds->n_exits ||
      !drv->predictions || !drv->exit_time_us || drv->max_rounds < 1)
    return A3FR_ERR_INVALID_ARG;
  if (drv->mode < A3FR_DRIVE_A3FR || drv->mode > A3FR_DRIVE_FRR) return A3FR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return A3FR_ERR_CUDA;
  *result = a3fr_frame_result{};
  const int eyes = a3fr::scene_eyes(scene);
  if (eyes == 0) {
    cudaEventDestroy(ev);
    return A3FR_ERR_INVALID_ARG;
  }

  std::atomic<int> posted{0};
  const Clock::time_point t0 = Clock::now();
  auto tracker = [&]() {
    double t = 0.0, prev = 0.0;
    for (int i = 0; i < drv->n_exits; ++i) {
      double dt = drv->exit_time_us[i] - prev;
      prev = drv->exit_time_us[i];
      if (drv->load_period_us > 0.0 && ((int64_t)(t / drv->load_period_us) & 1))
        dt *= drv->load_factor;   // the heavily loaded half of each period
      t += dt;
      wait_until_us(t0, t);
      a3fr_post_prediction(scene, i + 1, drv->predictions + (size_t)i * eyes * 2);
      posted.store(i + 1, std::memory_order_release);
    }
  };

  int rc = A3FR_OK;
  std::thread th;
  if (drv->mode == A3FR_DRIVE_FRR) {
    rc = a3fr_render_full(scene, out_rgb, stream);
    if (rc == A3FR_OK && cudaEventRecord(ev, st) == cudaSuccess && spin_event(ev) == cudaSuccess)
      result->latency_us = us_since(t0);
    else if (rc == A3FR_OK)
      rc = A3FR_ERR_CUDA;
    result->rounds = 1;
  } else if (drv->mode == A3FR_DRIVE_SFR) {
    th = std::thread(tracker);
    while (posted.load(std::memory_order_acquire) < drv->n_exits) std::this_thread::yield();
    const float *u_n = drv->predictions + (size_t)(drv->n_exits - 1) * eyes * 2;
    rc = a3fr_set_gaze(scene, u_n, stream);
    if (rc == A3FR_OK) rc = a3fr_render_foveated(scene, fovea, out_rgb, stream);
    if (rc == A3FR_OK && cudaEventRecord(ev, st) == cudaSuccess && spin_event(ev) == cudaSuccess)
      result->latency_us = us_since(t0);
    else if (rc == A3FR_OK)
      rc = A3FR_ERR_CUDA;
    result->rounds = 1;
  } else {
    rc = a3fr_begin_frame(scene, fovea, rounds, out_rgb, stream);
    if (rc == A3FR_OK) th = std::thread(tracker);
    int last_seen = 0;
    float last_r = -1.0f;
    bool idle = true;   // the last round had nothing left to render
    for (int r = 0; rc == A3FR_OK && r < drv->max_rounds; ++r) {
      if (!rounds->sir || idle) {
        // without speculation, before the first prediction, and once the speculative region
        // has reached its maximum (Eq. 4), the GPU waits for the tracker's next prediction
        while (posted.load(std::memory_order_acquire) <= last_seen) std::this_thread::yield();
      }
      rc = a3fr_render_round(scene, out_rgb, stream);
      if (rc != A3FR_OK) break;
      if (cudaEventRecord(ev, st) != cudaSuccess || spin_event(ev) != cudaSuccess) {
        rc = A3FR_ERR_CUDA;
        break;
      }
      a3fr_round_status rs{};
      a3fr_get_round_status(scene, &rs);
      if (result->rounds < 16) {
        result->exit_per_round[result->rounds] = rs.exit_consumed;
        result->round_end_us[result->rounds] = us_since(t0);
      }
      result->rounds++;
      idle = rs.exit_consumed == last_seen && rs.radius_px[0] == last_r;
      last_seen = rs.exit_consumed;
      last_r = rs.radius_px[0];
      if (rs.complete) {
        result->latency_us = us_since(t0);
        break;
      }
    }
  }
  if (th.joinable()) th.join();
  result->tracker_end_us = us_since(t0);
  cudaEventDestroy(ev);
  return rc;
}
