// round.cu -- the start of one incremental rendering round (Sec. 3.3, Algorithm 1).
//
// The gaze tracker posts its early-exit predictions u_i into a mailbox in mapped (pinned,
// device-visible) host memory at any time; a round reads the LATEST one when it runs on the
// GPU (Sec. 3.3.3: the latest prediction is stored where the GPU can read it, and the GPU
// picks it up when a round completes).  One thread:
//   * reads the mailbox under its sequence lock (bounded retries, then a status bit);
//   * a new prediction u_i sets the round's gaze and the layer radii
//       r_{k,i} = max(0, r_{k,N} - E[dist(u_i, u_N)])                       (Eq. 3')
//     so that the region rendered now lies inside the final one in expectation;
//   * with no new prediction, speculative incremental rendering (SIR) keeps growing the
//     region around the last prediction u_j by a fixed step, up to
//       r^max_{k,j} = r_{k,N} + E[dist(u_j, u_N)]                          (Eq. 4);
//     without SIR the round renders nothing;
//   * the frame is complete once the final exit's region has been rendered;
//   * the round's gaze and squared radii go to the plan kernel, the state to device memory
//     and a status copy to mapped host memory (readable by the host without a sync).
#include "common.cuh"

namespace a3fr {
namespace {

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int *p) {
  return *reinterpret_cast<const volatile unsigned int *>(p);
}

__global__ void round_begin_kernel(RoundConfig c, const Mailbox *__restrict__ mbox,
                                   RoundState *__restrict__ st, RoundPlan *__restrict__ plan,
                                   RoundStatus *__restrict__ status, uint32_t *__restrict__ err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int exit = st->last_exit;
  float g[kMaxEyes][2] = {{0.f, 0.f}, {0.f, 0.f}};
  bool ok = false;
  const volatile Mailbox *vm = mbox;
  for (int tries = 0; tries < (1 << 16) && !ok; ++tries) {
    const unsigned int s1 = ld_volatile_u32(&mbox->seq);
    if (s1 & 1u) {
      __nanosleep(64);
      continue;
    }
    __threadfence_system();
    const int e = vm->exit;
    float h[kMaxEyes][2];
    for (int q = 0; q < kMaxEyes; ++q) {
      h[q][0] = vm->gaze[q][0];
      h[q][1] = vm->gaze[q][1];
    }
    __threadfence_system();
    if (ld_volatile_u32(&mbox->seq) == s1) {
      ok = true;
      exit = e;
      for (int q = 0; q < kMaxEyes; ++q) {
        g[q][0] = h[q][0];
        g[q][1] = h[q][1];
      }
    }
  }
  if (!ok) atomicOr(err, kStatusTimeout);   // keep the previous prediction

  RoundPlan rp{};
  rp.active = 0;
  if (ok && exit > st->last_exit && exit <= c.n_exits) {
    st->last_exit = exit;
    const float e = c.expected[exit - 1];
    for (int q = 0; q < c.n_eyes; ++q) {
      st->gaze[q][0] = g[q][0];
      st->gaze[q][1] = g[q][1];
      for (int k = 0; k < 3; ++k) st->r[q][k] = fmaxf(0.0f, c.rf[q][k] - e);
    }
    rp.active = 1;
  } else if (c.sir && st->last_exit > 0 && !st->complete) {
    const float e = c.expected[st->last_exit - 1];
    for (int q = 0; q < c.n_eyes; ++q)
      for (int k = 0; k < 3; ++k) st->r[q][k] = fminf(st->r[q][k] + c.step, c.rf[q][k] + e);
    rp.active = 1;
  }
  if (rp.active) {
    for (int q = 0; q < c.n_eyes; ++q) {
      rp.gaze[q][0] = st->gaze[q][0];
      rp.gaze[q][1] = st->gaze[q][1];
      for (int k = 0; k < 3; ++k) rp.r2[q][k] = st->r[q][k] * st->r[q][k];
    }
    st->rounds += 1;
  }
  if (st->last_exit == c.n_exits) st->complete = 1;
  *plan = rp;
  volatile RoundStatus *vs = status;
  vs->exit_consumed = st->last_exit;
  vs->complete = st->complete;
  vs->rounds = st->rounds;
  for (int k = 0; k < 3; ++k) vs->radius[k] = st->r[0][k];
  __threadfence_system();
}

}  // namespace

cudaError_t launch_round_begin(const RoundConfig &c, const Mailbox *mbox, RoundState *state,
                               RoundPlan *plan, RoundStatus *status, uint32_t *error_status,
                               cudaStream_t s) {
  round_begin_kernel<<<1, 32, 0, s>>>(c, mbox, state, plan, status, error_status);
  return cudaGetLastError();
}

}  // namespace a3fr
