// sort.cu -- stable LSD radix sort of (key, 32-bit value) pairs, the depth sort of 3DGS
// (Sec. 2.3, "Sorting").  The renderer uses it twice per frame: once on the Gaussians by
// depth (32-bit keys) and once on the depth-ordered instances by tile index (16-bit or
// narrower keys); a stable sort by tile of depth-ordered instances is the order of the
// (tile << 32 | depth) keys.  The public a3fr_sort_pairs sorts 64-bit keys directly.
//
// Algorithm: onesweep (Adinets & Merrill, "Onesweep: A Faster Least Significant Digit
// Radix Sort for GPUs", 2022).  A histogram kernel (or the producer of the keys) counts
// the digits of all passes at once; then each pass is ONE kernel that
//   1. takes a partition index from an atomic counter (so partitions start in order),
//   2. ranks its keys stably inside the CTA with warp-level multisplit
//      (the peers of a digit from one ballot per digit bit + per-warp digit counters),
//   3. publishes its per-digit counts and resolves the exclusive prefix of every digit by
//      decoupled look-back over earlier partitions (flag + 30-bit count in one word),
//      reading a window of 8 predecessors per step so a single wave of partitions does
//      not serialise on one L2 round trip per predecessor,
//   4. stages the pairs in shared memory in digit order and writes them out in runs.
// Every look-back wait is bounded: after kSpinLimit polls the CTA records
// kStatusTimeout in the status word and carries on (its writes stay in bounds), so a
// scheduling anomaly can corrupt a result but never hang the GPU.  Partitions beyond the
// device-resident count exit at once, so grids are sized for a capacity without a host
// synchronisation.
#include "common.cuh"

namespace a3fr {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRadix = 256;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr uint32_t kSpinLimit = 1u << 22;   // polls 256 ns apart: about a second
constexpr int kWin = 8;   // look-back window (predecessor partitions read at once)

template <typename K> struct Part;
template <> struct Part<uint64_t> { static constexpr int kKPT = 12; };
template <> struct Part<uint32_t> { static constexpr int kKPT = 16; };

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

// Digit histograms of every pass in one read of the keys.  Each thread walks a contiguous
// run of keys and, per pass, adds to shared memory only when the digit changes (so the
// few-valued high digits of depths cost one atomic per run instead of one per key); each
// warp owns a private copy of the counters, summed at the end.
constexpr int kHistKeysPerThread = 8;

template <typename K, bool kRebase>
__global__ void __launch_bounds__(kThreads)
histogram_kernel(K *__restrict__ keys, const uint32_t *__restrict__ d_count, SortPlan plan,
                 uint32_t *__restrict__ hist, const uint32_t *__restrict__ range) {
  pdl_begin();
  __shared__ uint32_t s_hist[kWarps][4][kRadix];   // per warp, up to 4 passes per launch
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t n = *d_count;
  for (int p0 = 0; p0 < plan.passes; p0 += 4) {
    const int np = min(4, plan.passes - p0);
    for (int i = t; i < kWarps * 4 * kRadix; i += kThreads) (&s_hist[0][0][0])[i] = 0;
    __syncthreads();
    const uint32_t per_block = kThreads * kHistKeysPerThread;
    // a thread's 8 consecutive 32-bit keys as two 16-byte loads (and stores, when rebased)
    constexpr bool kVec = sizeof(K) == 4 && kHistKeysPerThread == 8;
    const bool vec_ok = kVec && (reinterpret_cast<uintptr_t>(keys) & 15u) == 0u;
    for (uint32_t base = blockIdx.x * per_block; base < n; base += gridDim.x * per_block) {
      const uint32_t i0 = base + t * kHistKeysPerThread;
      const uint32_t i1 = min(n, i0 + kHistKeysPerThread);
      const bool vec = vec_ok && i1 == i0 + kHistKeysPerThread;
      K kv[kHistKeysPerThread];
      if constexpr (kVec) {
        if (vec) {
          const uint4 a = reinterpret_cast<const uint4 *>(keys + i0)[0];
          const uint4 b = reinterpret_cast<const uint4 *>(keys + i0)[1];
          kv[0] = a.x; kv[1] = a.y; kv[2] = a.z; kv[3] = a.w;
          kv[4] = b.x; kv[5] = b.y; kv[6] = b.z; kv[7] = b.w;
        }
      }
      bool rebased = false;
      uint32_t cur[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
      uint32_t run[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int j = 0; j < kHistKeysPerThread; ++j) {
        const uint32_t i = i0 + (uint32_t)j;
        if (i >= i1) break;
        K k = vec ? kv[j] : keys[i];
        if (kRebase && p0 == 0) {
          // visible keys are <= max; a range under 2^24 leaves the top digit zero
          const uint32_t kmin = ~range[0], kmax = range[2];
          if (kmax >= kmin && kmax - kmin < (1u << 24)) {
            k = (K)((uint32_t)k <= kmax ? (uint32_t)k - kmin : 0xffffffu);
            if (vec) {
              kv[j] = k;
              rebased = true;
            } else {
              keys[i] = k;
            }
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (q < np) {
            const uint32_t d = (uint32_t)(k >> plan.shift[p0 + q]) & plan.mask;
            if (d != cur[q]) {
              if (run[q]) atomicAdd(&s_hist[warp][q][cur[q]], run[q]);
              cur[q] = d;
              run[q] = 0;
            }
            ++run[q];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < np && run[q]) atomicAdd(&s_hist[warp][q][cur[q]], run[q]);
      if constexpr (kVec) {
        if (rebased) {
          reinterpret_cast<uint4 *>(keys + i0)[0] = make_uint4(kv[0], kv[1], kv[2], kv[3]);
          reinterpret_cast<uint4 *>(keys + i0)[1] = make_uint4(kv[4], kv[5], kv[6], kv[7]);
        }
      }
    }
    __syncthreads();
    for (int i = t; i < np * kRadix; i += kThreads) {
      const int q = i / kRadix, d = i - q * kRadix;
      uint32_t v = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) v += s_hist[w][q][d];
      if (v) atomicAdd(hist + (p0 + q) * kRadix + d, v);
    }
    __syncthreads();
  }
}

// Where a pass's pairs come from.  MemSource reads them from memory (the value may be the
// input position); a pass whose digit is the same for every key may copy them through.
template <typename K>
struct MemSource {
  const K *keys;
  const uint32_t *vals;   // null: the value is the input position
  static constexpr bool kCopyable = true;
  // item k of lane l of warp w: position base + w*32*KPT + k*32 + l
  template <int KPT>
  __device__ __forceinline__ void load(uint32_t base, uint32_t n, K (&key)[KPT], uint32_t (&val)[KPT],
                                       unsigned char *) const {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t wbase = base + warp * 32 * KPT + lane;
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const uint32_t i = wbase + k * 32;
      const bool valid = i < n;
      key[k] = valid ? keys[i] : K(0);
      val[k] = valid ? (vals ? vals[i] : i) : 0u;
    }
  }
  __device__ __forceinline__ void copy(uint32_t i, K *keys_out, uint32_t *vals_out) const {
    if (keys_out) keys_out[i] = keys[i];
    vals_out[i] = vals ? vals[i] : i;
  }
};

// The tile instances of the depth-ordered entries, generated in place of being read: slot q of
// the instance array is instance q - off[j] of the entry j with off[j] <= q < off[j + 1]
// (exclusive instance offsets); instance r of an entry whose tile rectangle is w tiles wide is
// tile (x0 + r mod w, y0 + r div w), so the slots list every entry's tiles row-major, entries
// in depth order -- the array an emit of the instances would write, here never stored.  Per
// partition: its first and last entries (pstart); the entries between them staged in shared
// memory as (offset, first tile, width, Gaussian), one thread per entry, each entry with
// instances marking its first slot; the marks spread over the slots by a running maximum (no
// per-slot search); then each slot reads its entry's record.
static_assert(kGenPart == kThreads * 16, "a generated partition is one 32-bit-key partition");
constexpr int kGenWin = 2048;   // entries per window: a partition's whenever its entries average
                                // two or more instances (else several windows)
constexpr size_t kGenSmem = (size_t)kGenWin * 16 + (size_t)kGenPart * 2;

struct GenSource {
  EmitSource e;
  static constexpr bool kCopyable = false;

  // offset of entry j relative to slot base, at most kGenPart (past the entries: the total)
  __device__ __forceinline__ int rel_off(uint32_t j, uint32_t base, unsigned long long total) const {
    const unsigned long long o = j < (uint32_t)e.n_entries ? (unsigned long long)e.off[j] : total;
    const long long d = (long long)o - (long long)base;
    return (int)(d < kGenPart ? d : kGenPart);
  }

  template <int KPT>
  __device__ __forceinline__ void load(uint32_t base, uint32_t n, uint32_t (&key)[KPT],
                                       uint32_t (&val)[KPT], unsigned char *smem) const {
    static_assert(kThreads * KPT == kGenPart, "one slot per item");
    uint4 *s_rec = reinterpret_cast<uint4 *>(smem);                      // per window entry
    uint16_t *s_ent = reinterpret_cast<uint16_t *>(smem + 16 * kGenWin);  // slot -> window entry
    __shared__ uint32_t s_wmax[kWarps];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // every item below n is generated by exactly one window; the others stay unset (the pass
    // marks them invalid and never reads them)
    const uint32_t *__restrict__ entries = e.entries.get();
    const unsigned long long total = *e.total;
    const uint32_t part = base / kGenPart;
    // the entries holding this partition's first slot and the next partition's first slot
    // (or the last entry): every slot of the partition lies between them
    uint32_t jw = e.pstart[part];
    const uint32_t j_last = (unsigned long long)base + kGenPart < total && part + 1 < (uint32_t)e.n_parts
                                ? e.pstart[part + 1] : (uint32_t)e.n_entries - 1u;
    const int q_end = (int)min(n - base, (uint32_t)kGenPart);   // this partition's slots
    int win_lo = 0;
    for (;;) {
      const uint32_t cnt = min((uint32_t)kGenWin, j_last + 1u - jw);   // entries of this window
      for (int i = t; i < kGenPart / 8; i += kThreads) reinterpret_cast<uint4 *>(s_ent)[i] = make_uint4(0u, 0u, 0u, 0u);
      __syncthreads();
      for (uint32_t i = t; i < cnt; i += kThreads) {
        const uint32_t j = jw + i;
        const uint32_t v = entries[j];
        const int o = rel_off(j, base, total), o1 = rel_off(j + 1, base, total);
        const ushort4 rc = e.rect[v];
        const uint32_t eye = v >= (uint32_t)e.n ? 1u : 0u;
        s_rec[i] = make_uint4((uint32_t)o, eye * (uint32_t)e.n_tiles + (uint32_t)rc.y * (uint32_t)e.tiles_x + rc.x,
                              (uint32_t)(rc.z - rc.x), v - eye * (uint32_t)e.n);
        // every entry with instances marks its first slot (those offsets strictly increase)
        if (o >= 0 && o < kGenPart && o1 > o) s_ent[o] = (uint16_t)i;
      }
      const int next = rel_off(jw + cnt, base, total);   // the first offset past the window
      __syncthreads();
      // running maximum over the slots (thread t: slots 16t .. 16t + 15): each slot's entry is
      // the last one marked at or before it; unmarked leading slots keep entry 0
      {
        uint4 *p = reinterpret_cast<uint4 *>(s_ent) + 2 * t;
        const uint4 a = p[0], c = p[1];
        uint32_t w[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
        uint32_t run = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) run = max(run, max(w[i] & 0xffffu, w[i] >> 16));
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl = max(incl, v);
        }
        if (lane == 31) s_wmax[warp] = incl;
        uint32_t prev = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) prev = 0;
        __syncthreads();
        for (int ww = 0; ww < warp; ++ww) prev = max(prev, s_wmax[ww]);
        run = prev;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint32_t lo16 = max(run, w[i] & 0xffffu);
          const uint32_t hi16 = max(lo16, w[i] >> 16);
          w[i] = lo16 | (hi16 << 16);
          run = hi16;
        }
        p[0] = make_uint4(w[0], w[1], w[2], w[3]);
        p[1] = make_uint4(w[4], w[5], w[6], w[7]);
      }
      __syncthreads();
      const bool last = jw + cnt > j_last;
      const int win_hi = last ? kGenPart : next;
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        const int q = warp * 32 * KPT + k * 32 + lane;
        if (q < q_end && q >= win_lo && q < win_hi) {
          const uint4 rec = s_rec[s_ent[q]];   // (offset, first tile, width, Gaussian)
          const uint32_t r = (uint32_t)(q - (int)rec.x);   // < 2^16 instances per entry
          const uint32_t dy = div_small(r, rec.z), dx = r - dy * rec.z;
          key[k] = rec.y + dy * (uint32_t)e.tiles_x + dx;
          val[k] = rec.w;
        }
      }
      if (last || next >= q_end) break;
      __syncthreads();   // the next window reuses the staging
      win_lo = next;
      jw += cnt;
    }
  }
  __device__ __forceinline__ void copy(uint32_t, uint32_t *, uint32_t *) const {}
};

template <typename K, int KPT, class Src>
__global__ void __launch_bounds__(kThreads, 3)
onesweep_kernel(Src src, K *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                const uint32_t *__restrict__ d_count, const uint32_t *__restrict__ hist,
                uint32_t *__restrict__ part_counter, uint32_t *__restrict__ lookback, int shift,
                uint32_t mask, uint32_t *__restrict__ status, uint32_t *__restrict__ skip_flag) {
  pdl_begin();
  constexpr int PART = kThreads * KPT;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  K *s_keys = reinterpret_cast<K *>(s_dyn);
  uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_dyn + sizeof(K) * PART);
  __shared__ uint32_t s_whist[kWarps][kRadix];
  __shared__ uint32_t s_local_excl[kRadix];
  __shared__ uint32_t s_gbase[kRadix];
  __shared__ uint32_t s_tmp[kWarps];
  __shared__ uint32_t s_part;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_part = atomicAdd(part_counter, 1u);
  for (int i = t; i < kWarps * kRadix; i += kThreads) (&s_whist[0][0])[i] = 0;
  const uint32_t n = *d_count;
  // a pass whose digit is the same for every key is the identity permutation (the sort is
  // stable): each partition just copies itself
  const bool trivial = __syncthreads_or(n > 0 && hist[t] == n) != 0 && Src::kCopyable;
  const uint32_t part = s_part;
  const uint32_t base = part * PART;
  if (base >= n) return;
  if (trivial && skip_flag) {
    // the caller reads the result from this pass's input instead (the pass is the identity)
    if (t == 0) *skip_flag = 1u;
    return;
  }
  if (trivial) {
    const uint32_t end = min(n, base + (uint32_t)PART);
    for (uint32_t i = base + t; i < end; i += kThreads) src.copy(i, keys_out, vals_out);
    return;
  }

  // load: warp w owns [base + w*32*KPT, ...), item k of lane l at k*32 + l
  K key[KPT];
  uint32_t val[KPT];
  uint32_t dr[KPT];   // digit (9 bits, 256 = invalid) << 16 | rank in warp
  src.template load<KPT>(base, n, key, val, s_dyn);
  const uint32_t wbase = base + warp * 32 * KPT + lane;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const uint32_t i = wbase + k * 32;
    dr[k] = i < n ? ((uint32_t)(key[k] >> shift) & mask) : 256u;
  }
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const uint32_t d = dr[k];
    // the lanes holding the same digit: one ballot per digit bit (the digits have at most 8),
    // restricted to the lanes with a key
    unsigned peers = __ballot_sync(0xffffffffu, d < 256u);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const bool bit = (d >> b) & 1u;
      const unsigned v = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? v : ~v;
    }
    uint32_t rank = 0, cnt = 0;
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

  // thread t owns digit t: exclusive offsets across warps and the CTA total
  const uint32_t d = t;
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = s_whist[w][d];
    s_whist[w][d] = total;
    total += c;
  }
  uint32_t *my_lb = lookback + (size_t)part * kRadix + d;
  // a digit with no key anywhere (narrow digits leave most of the 256 empty) needs no
  // look-back: every partition skips it alike, so nobody reads its entries either
  const bool used = hist[d] != 0u;
  if (used) st_relaxed(my_lb, (part == 0 ? kFlagPrefix : kFlagAgg) | total);
  const uint32_t local_excl = block_excl_scan(total, s_tmp);
  const uint32_t global_excl = block_excl_scan(hist[d], s_tmp);
  uint32_t excl = 0;
  if (part > 0 && used) {
    // windowed look-back: kWin predecessors are read at once (independent loads), summed
    // nearest first up to the first inclusive prefix; an unpublished one is polled again
    int j = (int)part - 1;
    uint32_t spins = 0;
    while (true) {
      uint32_t w[kWin];
#pragma unroll
      for (int k = 0; k < kWin; ++k)
        w[k] = (j - k >= 0) ? ld_relaxed(lookback + (size_t)(j - k) * kRadix + d) : kFlagPrefix;
      bool done = false;
      int k = 0;
      for (; k < kWin; ++k) {
        const uint32_t flag = w[k] & ~kValMask;
        if (flag == 0u) break;
        excl += w[k] & kValMask;
        if (flag == kFlagPrefix) {
          done = true;
          break;
        }
      }
      if (done) break;
      j -= k;
      if (k < kWin) {   // an unpublished predecessor: back off before polling it again
        if (++spins > kSpinLimit) {
          atomicOr(status, kStatusTimeout);
          break;
        }
        __nanosleep(spins < 3 ? 32u << spins : 256u);
      }
    }
    st_relaxed(my_lb, kFlagPrefix | ((excl + total) & kValMask));
  }
  s_local_excl[d] = local_excl;
  s_gbase[d] = global_excl + excl - local_excl;
  __syncthreads();

#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const uint32_t dk = dr[k] >> 16;
    if (dk < 256u) {
      const uint32_t pos = s_local_excl[dk] + s_whist[warp][dk] + (dr[k] & 0xffffu);
      s_keys[pos] = key[k];
      s_vals[pos] = val[k];
    }
  }
  __syncthreads();
  const uint32_t n_valid = min((uint32_t)PART, n - base);
  for (uint32_t i = t; i < n_valid; i += kThreads) {
    const K k = s_keys[i];
    const uint32_t o = s_gbase[(uint32_t)(k >> shift) & mask] + i;
    if (o < n) {   // always true unless a look-back wait gave up (status already set)
      if (keys_out) keys_out[o] = k;   // null: the caller reads only the values
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

template <typename K, int KPT, class Src>
constexpr size_t onesweep_smem() {
  constexpr size_t staging = (sizeof(K) + sizeof(uint32_t)) * kThreads * KPT;
  return Src::kCopyable ? staging : (staging > kGenSmem ? staging : kGenSmem);
}

template <typename K, int KPT, class Src>
cudaError_t set_smem_attr() {
  // per device: the attribute lives in each device's context
  constexpr int kMaxDev = 64;
  static bool done[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDev && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(onesweep_kernel<K, KPT, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)onesweep_smem<K, KPT, Src>());
  if (e == cudaSuccess && dev >= 0 && dev < kMaxDev) done[dev] = true;
  return e;
}

}  // namespace

SortPlan sort_plan(int key_bits, int digit_bits_max) {
  SortPlan p{};
  if (key_bits < 1) key_bits = 1;
  p.passes = (key_bits + digit_bits_max - 1) / digit_bits_max;
  const int db = (key_bits + p.passes - 1) / p.passes;
  p.mask = (1u << db) - 1u;
  for (int i = 0; i < p.passes; ++i) p.shift[i] = i * db;
  return p;
}

size_t onesweep_part_size(bool wide_keys, bool small_parts) {
  return (size_t)kThreads * (wide_keys ? Part<uint64_t>::kKPT : (small_parts ? 8 : Part<uint32_t>::kKPT));
}

size_t onesweep_lookback_bytes(size_t capacity, int passes, bool wide_keys, bool small_parts) {
  const size_t part = onesweep_part_size(wide_keys, small_parts);
  return sizeof(uint32_t) * kRadix * (size_t)passes * ((capacity + part - 1) / part);
}

int histogram_blocks(size_t capacity) {
  const int sms = sm_count();
  const size_t per_block = (size_t)kThreads * kHistKeysPerThread;
  const size_t hb = (capacity + per_block - 1) / per_block;
  return (int)(hb < (size_t)sms * 8 ? (hb > 0 ? hb : 1) : (size_t)sms * 8);
}

template <typename K>
cudaError_t launch_histogram(const K *keys, const uint32_t *d_count, size_t capacity,
                             const SortPlan &plan, uint32_t *hist, cudaStream_t s) {
  {
    const cudaError_t e_ = launch_pdl(histogram_kernel<K, false>, histogram_blocks(capacity), kThreads, 0, s,
                                      const_cast<K *>(keys), d_count, plan, hist, nullptr);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

cudaError_t launch_depth_histogram(uint32_t *keys, const uint32_t *d_count, const uint32_t *range,
                                   size_t capacity, const SortPlan &plan, uint32_t *hist,
                                   cudaStream_t s) {
  {
    const cudaError_t e_ = launch_pdl(histogram_kernel<uint32_t, true>, histogram_blocks(capacity), kThreads,
                                      0, s, keys, d_count, plan, hist, range);
    if (e_ != cudaSuccess) return e_;
  }
  return cudaGetLastError();
}

// Passes first .. plan.passes - 1 over (kin, vin) -> (kout, vout), ping-ponging.
template <typename K, int KPT>
cudaError_t run_passes(int first, K *kin, uint32_t *vin, K *kout, uint32_t *vout, bool implicit_vals,
                       const uint32_t *d_count, size_t parts, const SortPlan &plan, const uint32_t *hist,
                       uint32_t *counters, uint32_t *lookback, uint32_t *status, cudaStream_t s,
                       bool drop_final_keys, uint32_t *final_skip) {
  cudaError_t e = set_smem_attr<K, KPT, MemSource<K>>();
  if (e != cudaSuccess) return e;
  constexpr size_t dyn = onesweep_smem<K, KPT, MemSource<K>>();
  for (int p = first; p < plan.passes; ++p) {
    // the first pass may take the values to be the input positions (vals unread)
    const MemSource<K> src{kin, (p == 0 && implicit_vals) ? nullptr : vin};
    K *kdst = (drop_final_keys && p == plan.passes - 1) ? nullptr : kout;
    {
      const cudaError_t e_ = launch_pdl(onesweep_kernel<K, KPT, MemSource<K>>, (unsigned)parts, kThreads, dyn,
                                        s, src, kdst, vout, d_count, hist + p * kRadix, counters + p,
                                        lookback + (size_t)kRadix * parts * p, plan.shift[p], plan.mask,
                                        status, p == plan.passes - 1 ? final_skip : nullptr);
      if (e_ != cudaSuccess) return e_;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    K *tk = kin; kin = kout; kout = tk;
    uint32_t *tv = vin; vin = vout; vout = tv;
  }
  return cudaSuccess;
}

template <typename K, int KPT>
cudaError_t launch_onesweep_kpt(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt,
                                bool implicit_vals, const uint32_t *d_count, size_t capacity,
                                const SortPlan &plan, const uint32_t *hist, uint32_t *counters,
                                uint32_t *lookback, uint32_t *status, bool *result_in_alt,
                                cudaStream_t s, bool drop_final_keys, uint32_t *final_skip) {
  *result_in_alt = false;
  if (capacity == 0) return cudaSuccess;
  constexpr int PART = kThreads * KPT;
  const size_t parts = (capacity + PART - 1) / PART;
  cudaError_t e = run_passes<K, KPT>(0, keys, vals, keys_alt, vals_alt, implicit_vals, d_count, parts, plan,
                                     hist, counters, lookback, status, s, drop_final_keys, final_skip);
  if (e != cudaSuccess) return e;
  *result_in_alt = (plan.passes % 2) == 1;
  return cudaSuccess;
}

template <typename K>
cudaError_t launch_onesweep(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt,
                            bool implicit_vals, const uint32_t *d_count, size_t capacity,
                            const SortPlan &plan, const uint32_t *hist, uint32_t *counters,
                            uint32_t *lookback, uint32_t *status, bool *result_in_alt,
                            cudaStream_t s, bool small_parts, bool drop_final_keys,
                            uint32_t *final_skip) {
  if (sizeof(K) == 4 && small_parts)
    return launch_onesweep_kpt<K, 8>(keys, vals, keys_alt, vals_alt, implicit_vals, d_count, capacity,
                                     plan, hist, counters, lookback, status, result_in_alt, s,
                                     drop_final_keys, final_skip);
  return launch_onesweep_kpt<K, Part<K>::kKPT>(keys, vals, keys_alt, vals_alt, implicit_vals, d_count,
                                               capacity, plan, hist, counters, lookback, status,
                                               result_in_alt, s, drop_final_keys, final_skip);
}

template cudaError_t launch_histogram<uint32_t>(const uint32_t *, const uint32_t *, size_t,
                                                const SortPlan &, uint32_t *, cudaStream_t);
template cudaError_t launch_onesweep<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *,
                                               bool, const uint32_t *, size_t, const SortPlan &,
                                               const uint32_t *, uint32_t *, uint32_t *,
                                               uint32_t *, bool *, cudaStream_t, bool, bool,
                                               uint32_t *);

cudaError_t launch_emit_onesweep(const EmitSource &src, uint32_t *keys, uint32_t *vals, uint32_t *keys_alt,
                                 uint32_t *vals_alt, const uint32_t *d_count, size_t capacity,
                                 const SortPlan &plan, const uint32_t *hist, uint32_t *counters,
                                 uint32_t *lookback, uint32_t *status, bool *result_in_alt,
                                 cudaStream_t s, bool drop_final_keys) {
  *result_in_alt = false;
  if (capacity == 0 || plan.passes < 1) return cudaSuccess;
  constexpr int KPT = Part<uint32_t>::kKPT;
  const size_t parts = (capacity + kGenPart - 1) / kGenPart;
  cudaError_t e = set_smem_attr<uint32_t, KPT, GenSource>();
  if (e != cudaSuccess) return e;
  // pass 0 generates its pairs and writes the alternate buffers
  {
    const cudaError_t e_ = launch_pdl(onesweep_kernel<uint32_t, KPT, GenSource>, (unsigned)parts, kThreads,
                                      onesweep_smem<uint32_t, KPT, GenSource>(), s, GenSource{src},
                                      (drop_final_keys && plan.passes == 1) ? nullptr : keys_alt, vals_alt,
                                      d_count, hist, counters, lookback, plan.shift[0], plan.mask, status,
                                      nullptr);
    if (e_ != cudaSuccess) return e_;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = run_passes<uint32_t, KPT>(1, keys_alt, vals_alt, keys, vals, false, d_count, parts, plan, hist, counters,
                                lookback, status, s, drop_final_keys, nullptr);
  if (e != cudaSuccess) return e;
  *result_in_alt = (plan.passes % 2) == 1;
  return cudaSuccess;
}

// ---- the 64-bit pair sort of the public API (8-bit digits) ----
constexpr size_t kHistBytes = sizeof(uint32_t) * kMaxSortPasses * kRadix;
constexpr size_t kCounterBytes = 256;

size_t sort_workspace_bytes(size_t capacity) {
  return kHistBytes + kCounterBytes + onesweep_lookback_bytes(capacity, kMaxSortPasses, true, false);
}

cudaError_t launch_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                        const uint32_t *d_count, size_t capacity, int key_bits, void *workspace,
                        uint32_t *status, bool *result_in_alt, cudaStream_t s) {
  *result_in_alt = false;
  if (capacity == 0 || key_bits <= 0) return cudaSuccess;
  const SortPlan plan = sort_plan(key_bits, 8);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *hist = reinterpret_cast<uint32_t *>(ws);
  uint32_t *counters = reinterpret_cast<uint32_t *>(ws + kHistBytes);
  uint32_t *lookback = reinterpret_cast<uint32_t *>(ws + kHistBytes + kCounterBytes);
  cudaError_t e = cudaMemsetAsync(
      ws, 0, kHistBytes + kCounterBytes + onesweep_lookback_bytes(capacity, plan.passes, true, false), s);
  if (e != cudaSuccess) return e;
  e = launch_histogram<uint64_t>(keys, d_count, capacity, plan, hist, s);
  if (e != cudaSuccess) return e;
  return launch_onesweep<uint64_t>(keys, vals, keys_alt, vals_alt, false, d_count, capacity,
                                   plan, hist, counters, lookback, status, result_in_alt, s, false);
}

}  // namespace a3fr
