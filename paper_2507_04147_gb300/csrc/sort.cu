// sort.cu -- stable LSD radix sort of (64-bit key, 32-bit value) pairs: the per-tile
// depth sort of 3DGS (Sec. 2.3, "Sorting"), run on the (tile << 32 | depth bits) keys so
// that one global sort orders every tile's Gaussians front to back.
//
// Algorithm: onesweep (Adinets & Merrill, "Onesweep: A Faster Least Significant Digit
// Radix Sort for GPUs", 2022).  One histogram kernel reads the keys once and counts all
// 8-bit digits of all passes; then each pass is ONE kernel that
//   1. takes a partition index from an atomic counter (so partitions start in order),
//   2. ranks its keys stably inside the CTA with warp-level multisplit
//      (__match_any_sync + per-warp digit counters),
//   3. publishes its per-digit counts and resolves the exclusive prefix of every digit by
//      decoupled look-back over earlier partitions (flag + 30-bit count in one word),
//   4. stages the keys in shared memory in digit order and writes them out in runs.
// Every look-back wait is bounded: after kSpinLimit polls the CTA records
// kStatusTimeout in the status word and continues, so a scheduling anomaly can corrupt
// an output but never hang the GPU.  Partitions beyond the device-resident count exit at
// once, so the grid can be sized for the capacity without a host synchronisation.
#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kKPT = 12;
constexpr int kPart = kThreads * kKPT;            // keys per partition
constexpr int kRadix = 256;
constexpr int kMaxPasses = 8;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr uint32_t kSpinLimit = 1u << 20;

// Workspace: hist[kMaxPasses][256] | counters[kMaxPasses] (+pad) | lookback[passes][parts][256]
constexpr size_t kHistBytes = sizeof(uint32_t) * kMaxPasses * kRadix;
constexpr size_t kCounterBytes = 256;

size_t n_parts(size_t n) { return (n + kPart - 1) / kPart; }

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Exclusive scan of one value per thread across a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_tmp) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) s_tmp[warp] = incl;
  __syncthreads();
  uint32_t before = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) before += (w < warp) ? s_tmp[w] : 0u;
  __syncthreads();
  return before + incl - v;
}

__global__ void __launch_bounds__(kThreads)
histogram_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ d_count,
                 int passes, uint32_t *__restrict__ hist) {
  __shared__ uint32_t s_hist[kMaxPasses][kRadix];
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += kThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t n = *d_count;
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * kThreads;
  for (uint32_t base = blockIdx.x * kThreads; base < n; base += stride) {
    const uint32_t i = base + threadIdx.x;
    const bool valid = i < n;
    const uint64_t k = valid ? keys[i] : 0ull;
    const unsigned active = __ballot_sync(0xffffffffu, valid);
    for (int p = 0; p < passes; ++p) {
      const uint32_t d = (uint32_t)(k >> (8 * p)) & 0xffu;
      if (valid) {
        // one shared-memory atomic per distinct digit of the warp
        const unsigned peers = __match_any_sync(active, d);
        if (lane == 31 - __clz(peers)) atomicAdd(&s_hist[p][d], (uint32_t)__popc(peers));
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += kThreads) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(hist + i, v);
  }
}

__global__ void __launch_bounds__(kThreads, 3)
onesweep_kernel(const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                uint64_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                const uint32_t *__restrict__ d_count, const uint32_t *__restrict__ hist,
                uint32_t *__restrict__ part_counter, uint32_t *__restrict__ lookback, int shift,
                uint32_t *__restrict__ status) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint64_t *s_keys = reinterpret_cast<uint64_t *>(s_dyn);
  uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_dyn + sizeof(uint64_t) * kPart);
  __shared__ uint32_t s_whist[kWarps][kRadix];
  __shared__ uint32_t s_local_excl[kRadix];
  __shared__ uint32_t s_gbase[kRadix];
  __shared__ uint32_t s_tmp[kWarps];
  __shared__ uint32_t s_part;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_part = atomicAdd(part_counter, 1u);
  for (int i = t; i < kWarps * kRadix; i += kThreads) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t part = s_part;
  const uint32_t n = *d_count;
  const uint32_t base = part * kPart;
  if (base >= n) return;

  // load: warp w owns keys [base + w*32*kKPT, ...), item k of lane l at k*32 + l
  uint64_t key[kKPT];
  uint32_t val[kKPT];
  uint32_t dr[kKPT];   // digit (9 bits, 256 = invalid) << 16 | rank in warp
  const uint32_t wbase = base + warp * 32 * kKPT + lane;
#pragma unroll
  for (int k = 0; k < kKPT; ++k) {
    const uint32_t i = wbase + k * 32;
    const bool valid = i < n;
    key[k] = valid ? keys_in[i] : 0ull;
    val[k] = valid ? vals_in[i] : 0u;
    dr[k] = valid ? ((uint32_t)(key[k] >> shift) & 0xffu) : 256u;
  }
  // warp-level multisplit ranking, in original order
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kKPT; ++k) {
    const uint32_t d = dr[k];
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = 0;
    uint32_t cnt = 0;
    if (d < 256u) {
      cnt = s_whist[warp][d];
      rank = cnt + __popc(peers & lt_mask);
    }
    __syncwarp();
    if (d < 256u && lane == 31 - __clz(peers)) s_whist[warp][d] = cnt + __popc(peers);
    __syncwarp();
    dr[k] = (d << 16) | rank;
  }
  __syncthreads();

  // per digit (thread t owns digit t): exclusive offsets across warps, CTA total
  const uint32_t d = t;
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = s_whist[w][d];
    s_whist[w][d] = total;
    total += c;
  }
  uint32_t *my_lb = lookback + (size_t)part * kRadix + d;
  st_relaxed(my_lb, (part == 0 ? kFlagPrefix : kFlagAgg) | total);
  const uint32_t local_excl = block_excl_scan(total, s_tmp);
  const uint32_t global_excl = block_excl_scan(hist[d], s_tmp);
  uint32_t excl = 0;
  if (part > 0) {
    int j = (int)part - 1;
    uint32_t spins = 0;
    while (true) {
      const uint32_t v = ld_relaxed(lookback + (size_t)j * kRadix + d);
      const uint32_t flag = v & ~kValMask;
      if (flag == 0u) {
        if (++spins > kSpinLimit) {
          atomicOr(status, kStatusTimeout);
          break;
        }
        continue;
      }
      excl += v & kValMask;
      if (flag == kFlagPrefix || j == 0) break;
      --j;
    }
    st_relaxed(my_lb, kFlagPrefix | ((excl + total) & kValMask));
  }
  s_local_excl[d] = local_excl;
  s_gbase[d] = global_excl + excl - local_excl;
  __syncthreads();

  // scatter into shared memory in digit order
#pragma unroll
  for (int k = 0; k < kKPT; ++k) {
    const uint32_t dk = dr[k] >> 16;
    if (dk < 256u) {
      const uint32_t pos = s_local_excl[dk] + s_whist[warp][dk] + (dr[k] & 0xffffu);
      s_keys[pos] = key[k];
      s_vals[pos] = val[k];
    }
  }
  __syncthreads();
  const uint32_t n_valid = min((uint32_t)kPart, n - base);
  for (uint32_t i = t; i < n_valid; i += kThreads) {
    const uint64_t k = s_keys[i];
    const uint32_t o = s_gbase[(uint32_t)(k >> shift) & 0xffu] + i;
    if (o < n) {   // always true unless a look-back wait gave up (status already set)
      keys_out[o] = k;
      vals_out[o] = s_vals[i];
    }
  }
}

int sm_count() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

size_t sort_workspace_bytes(size_t capacity) {
  return kHistBytes + kCounterBytes + sizeof(uint32_t) * kMaxPasses * kRadix * n_parts(capacity);
}

cudaError_t launch_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                        const uint32_t *d_count, size_t capacity, int key_bits, void *workspace,
                        uint32_t *status, bool *result_in_alt, cudaStream_t s) {
  *result_in_alt = false;
  if (capacity == 0 || key_bits <= 0) return cudaSuccess;
  const int passes = (key_bits + 7) / 8;
  const size_t parts = n_parts(capacity);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *hist = reinterpret_cast<uint32_t *>(ws);
  uint32_t *counters = reinterpret_cast<uint32_t *>(ws + kHistBytes);
  uint32_t *lookback = reinterpret_cast<uint32_t *>(ws + kHistBytes + kCounterBytes);
  const size_t lb_pass = (size_t)kRadix * parts;
  cudaError_t e = cudaMemsetAsync(
      ws, 0, kHistBytes + kCounterBytes + sizeof(uint32_t) * lb_pass * passes, s);
  if (e != cudaSuccess) return e;

  static bool attr_set = false;
  const size_t dyn = (sizeof(uint64_t) + sizeof(uint32_t)) * kPart;
  if (!attr_set) {
    e = cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int sms = sm_count();
  const size_t hb = (capacity + kThreads * 16 - 1) / (kThreads * 16);
  const int hist_blocks = (int)(hb < (size_t)sms * 4 ? hb : (size_t)sms * 4);
  histogram_kernel<<<hist_blocks > 0 ? hist_blocks : 1, kThreads, 0, s>>>(keys, d_count, passes,
                                                                         hist);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  uint64_t *kin = keys, *kout = keys_alt;
  uint32_t *vin = vals, *vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    onesweep_kernel<<<(unsigned)parts, kThreads, dyn, s>>>(
        kin, vin, kout, vout, d_count, hist + p * kRadix, counters + p, lookback + lb_pass * p,
        8 * p, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint64_t *tk = kin; kin = kout; kout = tk;
    uint32_t *tv = vin; vin = vout; vout = tv;
  }
  *result_in_alt = (passes % 2) == 1;
  return cudaSuccess;
}

}  // namespace a3fr
