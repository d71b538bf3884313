// Standalone row-wise k-selection (section 2 "k-selection" and section 4's goal: one
// pass over the input at memory bandwidth).
//
// One thread block per (row, segment).  Threads stream the segment with 16-byte
// loads (cache-streaming, eight in flight per thread), compare each value once against
// the block threshold and append the rare survivors to a shared buffer (select_core.cuh).  Long rows are cut
// into segments when there are too few rows to fill the GPU; each segment leaves its
// k best composites in scratch and a merge kernel selects across segments - the
// paper's two-pass k-selection (section 5.3, "Multi-pass kernels").  k = 1 is a plain
// argmin/argmax reduction (section 6.2 notes that k = 1 needs no selection structure).
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kselect.cuh"
#include "select_core.cuh"
#include "sm100.cuh"

namespace gbk {

namespace {

// v[b] for a per-lane index b without indexing the register array (which would move it to
// local memory): a binary tree of selects on the bits of b (PT - 1 selects).
template <int PT>
__device__ __forceinline__ float select_reg(const float (&v)[PT], int b) {
  static_assert(PT == 16 || PT == 32, "16 or 32 values per thread");
  float t[16];
  if constexpr (PT == 32) {
#pragma unroll
    for (int i = 0; i < 16; i++) t[i] = (b & 16) ? v[i + 16] : v[i];
  } else {
#pragma unroll
    for (int i = 0; i < 16; i++) t[i] = v[i];
  }
#pragma unroll
  for (int i = 0; i < 8; i++) t[i] = (b & 8) ? t[i + 8] : t[i];
#pragma unroll
  for (int i = 0; i < 4; i++) t[i] = (b & 4) ? t[i + 4] : t[i];
#pragma unroll
  for (int i = 0; i < 2; i++) t[i] = (b & 2) ? t[i + 2] : t[i];
  return (b & 1) ? t[1] : t[0];
}

template <int THREADS, int KP, int UNROLL, bool LARGEST>
struct KselCfg {
  static constexpr int PT = UNROLL * 4;          // floats per thread per iteration
  static constexpr int CHUNK = THREADS * PT;     // floats per block iteration
  // candidate buffer (a larger one for large k costs more occupancy than the compactions
  // it saves)
  static constexpr int CAP = 2048;
  static_assert(PT <= 32, "one 32-bit mask per thread");
  using Sel = BlockSelect<THREADS, KP, CAP>;
  static constexpr size_t SMEM = 16 + sizeof(typename Sel::Smem);
};

// One block per work unit (a row, or a segment of one).  Every thread keeps UNROLL 16-byte
// loads in flight per iteration (16 KB per 128-thread block, ~128 KB per SM at eight), filters
// them against the block threshold and appends survivors with one reservation per warp.
// A reservation that does not fit the buffer is not written; that warp keeps its values in
// registers and offers them again after the block compacts (block-uniform offer rounds),
// so the buffer never needs room for a worst-case iteration.
template <int THREADS, int KP, int UNROLL, bool LARGEST>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    kselect_rows_kernel(const float* __restrict__ vals, int64_t len, int k, int segs,
                        int64_t seg_len, float* __restrict__ outD, int64_t* __restrict__ outI,
                        uint64_t* __restrict__ part) {
  using C = KselCfg<THREADS, KP, UNROLL, LARGEST>;
  using Sel = typename C::Sel;
  constexpr bool PIPE = (UNROLL == 4);  // 4: double-buffered loads; 8: one fat buffer
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* overflow = reinterpret_cast<int*>(smem_raw);
  int* n_ok = overflow + 1;
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(smem_raw + 16);
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t unit = blockIdx.x;
  const int64_t row = unit / segs;
  const int seg = (int)(unit % segs);
  const int64_t s0 = (int64_t)seg * seg_len;
  const int64_t n = (len < s0 + seg_len ? len : s0 + seg_len) - s0;
  const float* rowp = vals + row * len;
  const float* p = rowp + s0;
  const int64_t he = (int64_t)(((16u - ((uintptr_t)p & 15u)) & 15u) / 4);
  const int head = (int)(n < he ? n : he);
  const int64_t n4 = (n - head) / 4;
  const int tail = (int)(n - head - n4 * 4);
  int* sure = overflow + 2;  // a compaction to k happened under the provisional threshold
  // Provisional threshold (k > 32 on long rows): from the first iteration's sample, the
  // r-th smallest of four group minima per thread, r ~ 1.25 k sample/n + 8; exact as soon
  // as k values at or below it are found (checked at the end, else the row is redone with
  // the plain threshold).
  const int64_t sample = (n4 < (int64_t)C::CHUNK / 4 ? n4 : (int64_t)C::CHUNK / 4) * 4;
  constexpr int GROUPS = 4;  // minima per thread (groups of PT / 4 values)
  const int64_t r64 = n > 0 ? (5 * (int64_t)k * sample) / (4 * n) + 8 : 0;
  // (the rank-th minimum is found by a compaction to `rank`, so rank may not exceed the
  // kept set's capacity KP: on short rows 1.25 k sample/n + 8 can, e.g. k = 125, n = 2606)
  const bool use_guess = k > 32 && r64 < (int64_t)(GROUPS * THREADS / 2) && r64 <= KP &&
                         sample >= 4 * (int64_t)THREADS;
  const int rank = (int)r64;
  float ht_v = 0.f;  // this thread's head / tail element, offered after the guess
  int64_t ht_e = -1;
  if (tid < head) ht_e = tid;
  else if (tid >= 32 && tid < 32 + tail) ht_e = head + n4 * 4 + (tid - 32);
  if (ht_e >= 0) ht_v = p[ht_e];
  const float4* p4 = reinterpret_cast<const float4*>(p + head);
  const uint32_t idx0 = (uint32_t)(s0 + head);
  ValueFilter f;
  for (int attempt = 0; attempt < 2; attempt++) {
  const bool guess = use_guess && attempt == 0;
  Sel::init(s);
  if (tid == 0) {
    *overflow = 0;
    *sure = 0;
  }
  __syncthreads();
  f.set(NAN_KEY, LARGEST);
  if (!guess) {
    uint64_t c[1];
    uint32_t mask = 0;
    if (ht_e >= 0 && f.pass(ht_v)) {
      c[0] = composite(ordered_key(ht_v, LARGEST), (uint32_t)(s0 + ht_e));
      mask = 1u;
    }
    Sel::template push<1>(s, mask, c);
  }
  __syncthreads();
  if (tid == 0) *n_ok = s.n_buf;
  // PIPE: the next iteration's loads are issued before this one is filtered, so the
  // block's capacity barrier never leaves the SM without loads in flight.
  float4 nxt[PIPE ? UNROLL : 1];
  if (PIPE) {
#pragma unroll
    for (int u = 0; u < UNROLL; u++) {
      const int64_t i = (int64_t)u * THREADS + tid;
      nxt[u] = i < n4 ? __ldcs(p4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  for (int64_t base = 0; base < n4; base += (int64_t)THREADS * UNROLL) {
    float v[C::PT];
#pragma unroll
    for (int u = 0; u < UNROLL; u++) {
      const int64_t i = base + u * THREADS + tid;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (PIPE) {
        x = nxt[u];
        const int64_t inext = i + (int64_t)THREADS * UNROLL;
        if (inext < n4) nxt[u] = __ldcs(p4 + inext);
      } else if (i < n4) {
        x = __ldcs(p4 + i);
      }
      v[u * 4 + 0] = x.x;
      v[u * 4 + 1] = x.y;
      v[u * 4 + 2] = x.z;
      v[u * 4 + 3] = x.w;
    }
    uint32_t skip = 0u;  // slots already offered as this thread's minima
    if (base == 0 && guess) {
      // GROUPS group minima of every thread; their rank-th smallest, g, has at least
      // rank sample values at or below it
      uint64_t mn[GROUPS];
      uint32_t gm = 0;
#pragma unroll
      for (int gi = 0; gi < GROUPS; gi++) mn[gi] = ~0ull;
#pragma unroll
      for (int u = 0; u < UNROLL; u++) {
        if (u * THREADS + tid < n4) {
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const int slot = u * 4 + j, gi = slot / (C::PT / GROUPS);
            const uint64_t c = composite(ordered_key(v[slot], LARGEST),
                                         idx0 + (uint32_t)((u * THREADS + tid) * 4 + j));
            if (c < mn[gi]) mn[gi] = c;
            gm |= 1u << gi;
          }
        }
      }
      Sel::template push<GROUPS>(s, gm, mn);
      __syncthreads();
      const bool have = s.n_buf > rank;  // uniform
      if (have) Sel::compact(s, rank);
      const uint32_t gkey = (uint32_t)(s.thr >> 32);
      __syncthreads();
      // the minima only located g: start the selection afresh with g as a provisional
      // value threshold, so every value <= g (ties included) is offered below
      if (tid == 0) {
        s.n_top = 0;
        s.n_buf = 0;
        s.thr = ~0ull;
      }
      __syncthreads();
      if (have) f.set(gkey, LARGEST);
      {
        uint64_t c[1];
        uint32_t mask = 0;
        if (ht_e >= 0 && f.pass(ht_v)) {
          c[0] = composite(ordered_key(ht_v, LARGEST), (uint32_t)(s0 + ht_e));
          mask = 1u;
        }
        Sel::template push<1>(s, mask, c);
      }
      __syncthreads();
      if (tid == 0) *n_ok = s.n_buf;
      __syncthreads();
    } else if (base == 0 && k <= THREADS) {
      // Seed the threshold: every thread offers the smallest of its first values; the
      // k-th smallest of these distinct elements bounds the row's k-th from above and is
      // about as tight as the k-th of the whole first iteration, at 1/PT of the work.
      uint64_t mn = ~0ull;
      int ms = -1;
#pragma unroll
      for (int u = 0; u < UNROLL; u++) {
        if (u * THREADS + tid < n4) {
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const uint64_t c = composite(ordered_key(v[u * 4 + j], LARGEST),
                                         idx0 + (uint32_t)((u * THREADS + tid) * 4 + j));
            if (c < mn) {
              mn = c;
              ms = u * 4 + j;
            }
          }
        }
      }
      uint64_t cm[1] = {mn};
      Sel::template push<1>(s, ms >= 0 ? 1u : 0u, cm);
      if (ms >= 0) skip = 1u << ms;
      __syncthreads();
      if (s.n_top + s.n_buf > k) {
        Sel::compact(s, k);
        f.set((uint32_t)(s.thr >> 32), LARGEST);
      }
      if (tid == 0) *n_ok = s.n_buf;
      __syncthreads();
    }
    bool pending = true;
    for (;;) {
      uint32_t mask = 0;
      if (pending) {
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
          if (base + u * THREADS + tid < n4) {
#pragma unroll
            for (int j = 0; j < 4; j++) mask |= (f.pass(v[u * 4 + j]) ? 1u : 0u) << (u * 4 + j);
          }
        }
        mask &= ~skip;
      }
      bool retry = false;
      if (__any_sync(FULL_MASK, mask != 0u)) {
        const int cnt = __popc(mask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(FULL_MASK, incl, o);
          if (lane >= o) incl += t;
        }
        int wbase = 0;
        if (lane == 31) wbase = atomicAdd(&s.n_buf, incl);
        wbase = __shfl_sync(FULL_MASK, wbase, 31);
        const int total = __shfl_sync(FULL_MASK, incl, 31);
        if (wbase + total <= C::CAP) {
          // survivors are rare: visit only the set bits (a lane's loop runs popc(mask) times)
          int pos = wbase + incl - cnt;
          const uint32_t ib = idx0 + (uint32_t)((base + tid) * 4);
          for (uint32_t m = mask; m; m &= m - 1) {
            const int b = __ffs(m) - 1;
            const float x = select_reg<C::PT>(v, b);
            s.buf[pos++] = composite(ordered_key(x, LARGEST),
                                     ib + (uint32_t)((b >> 2) * THREADS * 4 + (b & 3)));
          }
          if (lane == 31) atomicAdd(n_ok, total);
        } else {
          retry = true;
          if (lane == 31) *overflow = 1;
        }
      }
      pending = retry;
      __syncthreads();
      const bool ovf = *overflow != 0;
      if (!ovf) break;  // uniform: nobody writes the flag between the barriers
      __syncthreads();  // all have read the flag before it is reset
      if (tid == 0) {
        s.n_buf = *n_ok;  // successful reservations form a prefix of the buffer
        *overflow = 0;
        *sure = 1;        // more than CAP >= k candidates: the threshold is a true bound
      }
      __syncthreads();
      Sel::compact(s, k);
      f.set((uint32_t)(s.thr >> 32), LARGEST);
      if (tid == 0) *n_ok = s.n_buf;
      __syncthreads();
    }
  }
  __syncthreads();
  // a provisional threshold is exact once k candidates at or below it were found
  if (!guess || *sure != 0 || s.n_top + s.n_buf >= k) break;  // uniform (after a barrier)
  __syncthreads();  // all have read the state before the retry resets it
  }  // attempt
  Sel::finish(s, k);
  if (segs == 1) {
    for (int j = tid; j < k; j += THREADS) {
      const uint64_t e = s.top[j];
      const uint32_t idx = (uint32_t)e;
      if (idx < (uint32_t)len) {
        outD[row * k + j] = selected_value(e, LARGEST, rowp);
        outI[row * k + j] = (int64_t)idx;
      }
    }
  } else {
    uint64_t* dst = part + unit * k;
    for (int j = tid; j < k; j += THREADS) dst[j] = s.top[j];
  }
}

// The same selection with the row streamed through a shared-memory ring: one thread keeps
// RING_STAGES bulk copies (cp.async.bulk, 16 KB each) in flight ahead of the block, so HBM
// latency stays off the per-iteration path and no registers hold loads in flight.  Stage j
// holds float4s [j*STG4, (j+1)*STG4) of the 16-byte aligned body; every thread takes 4
// float4s of it.  A stage is refilled once every thread has read it (the barrier after the
// read).  Waits are bounded: a timeout sets the status word, the block stops at the next
// iteration boundary (agreed with a block-wide OR, so no barrier is ever skipped by a
// subset of threads) and waits, again with a limit, for its copies still in flight.
constexpr int RING_STAGES = 4;
template <int THREADS, int KP>
struct RingCfg {
  static constexpr int STG4 = THREADS * 4;  // float4 per stage
  static constexpr int PT = 16;             // floats per thread per stage
  static constexpr int CAP = 2048;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  static constexpr size_t RING_OFF = 128;   // after flags and barriers
  static constexpr size_t SEL_OFF = RING_OFF + (size_t)RING_STAGES * STG4 * 16;
  static constexpr size_t SMEM = SEL_OFF + sizeof(typename Sel::Smem);
};

template <int THREADS, int KP, bool LARGEST>
__global__ void __launch_bounds__(THREADS, 2)
    kselect_ring_kernel(const float* __restrict__ vals, int64_t len, int k, int segs,
                        int64_t seg_len, float* __restrict__ outD, int64_t* __restrict__ outI,
                        uint64_t* __restrict__ part, uint32_t* __restrict__ status) {
  using C = RingCfg<THREADS, KP>;
  using Sel = typename C::Sel;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int* overflow = reinterpret_cast<int*>(smem_raw);
  int* n_ok = overflow + 1;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(overflow + 2);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + 64);  // [RING_STAGES]
  float4* ring = reinterpret_cast<float4*>(smem_raw + C::RING_OFF);
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(smem_raw + C::SEL_OFF);
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t unit = blockIdx.x;
  const int64_t row = unit / segs;
  const int seg = (int)(unit % segs);
  const int64_t s0 = (int64_t)seg * seg_len;
  const int64_t n = (len < s0 + seg_len ? len : s0 + seg_len) - s0;
  const float* rowp = vals + row * len;
  const float* p = rowp + s0;
  const int64_t he = (int64_t)(((16u - ((uintptr_t)p & 15u)) & 15u) / 4);
  const int head = (int)(n < he ? n : he);
  const int64_t n4 = (n - head) / 4;
  const int tail = (int)(n - head - n4 * 4);
  const float4* p4 = reinterpret_cast<const float4*>(p + head);
  const int64_t nst = (n4 + C::STG4 - 1) / C::STG4;
  auto issue = [&](int64_t j) {  // thread 0: stage j into its slot
    const int slot = (int)(j % RING_STAGES);
    const int64_t rem = n4 - j * C::STG4;
    const int64_t c4 = rem < C::STG4 ? rem : (int64_t)C::STG4;
    sm100::fence_proxy_async_smem();
    sm100::mbar_arrive_expect_tx(&full[slot], (uint32_t)(c4 * 16));
    sm100::bulk_load(ring + (size_t)slot * C::STG4, p4 + j * C::STG4, (uint32_t)(c4 * 16),
                     &full[slot]);
  };
  Sel::init(s);
  if (tid == 0) {
    *overflow = 0;
    *abort_flag = 0;
    for (int i = 0; i < RING_STAGES; i++) sm100::mbar_init(&full[i], 1);
    sm100::fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int64_t j = 0; j < nst && j < RING_STAGES; j++) issue(j);
  ValueFilter f;
  f.set(NAN_KEY, LARGEST);
  {
    uint64_t c[1];
    uint32_t mask = 0;
    int64_t e = -1;
    if (tid < head) e = tid;
    else if (tid >= 32 && tid < 32 + tail) e = head + n4 * 4 + (tid - 32);
    if (e >= 0) {
      const float v = p[e];
      if (f.pass(v)) {
        c[0] = composite(ordered_key(v, LARGEST), (uint32_t)(s0 + e));
        mask = 1u;
      }
    }
    Sel::template push<1>(s, mask, c);
  }
  __syncthreads();
  if (tid == 0) *n_ok = s.n_buf;
  const uint32_t idx0 = (uint32_t)(s0 + head);
  int64_t waited = 0;  // stages [0, waited) have completed
  for (int64_t j = 0; j < nst; j++) {
    const int slot = (int)(j % RING_STAGES);
    const bool okw =
        sm100::mbar_wait(&full[slot], (uint32_t)((j / RING_STAGES) & 1), status, abort_flag);
    const int64_t base = j * C::STG4;
    float v[C::PT];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int64_t i = base + u * THREADS + tid;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (okw && i < n4) x = ring[(size_t)slot * C::STG4 + u * THREADS + tid];
      v[u * 4 + 0] = x.x;
      v[u * 4 + 1] = x.y;
      v[u * 4 + 2] = x.z;
      v[u * 4 + 3] = x.w;
    }
    if (__syncthreads_or(okw ? 0 : 1)) break;  // uniform: some wait gave up
    waited = j + 1;
    if (tid == 0 && j + RING_STAGES < nst) issue(j + RING_STAGES);  // the slot is free
    uint32_t skip = 0u;
    if (j == 0 && k <= THREADS) {
      // threshold seed: the k-th of the threads' minima (see kselect_rows_kernel)
      uint64_t mn = ~0ull;
      int ms = -1;
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (u * THREADS + tid < n4) {
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const uint64_t c = composite(ordered_key(v[u * 4 + q], LARGEST),
                                         idx0 + (uint32_t)((u * THREADS + tid) * 4 + q));
            if (c < mn) {
              mn = c;
              ms = u * 4 + q;
            }
          }
        }
      }
      uint64_t cm[1] = {mn};
      Sel::template push<1>(s, ms >= 0 ? 1u : 0u, cm);
      if (ms >= 0) skip = 1u << ms;
      __syncthreads();
      if (s.n_top + s.n_buf > k) {
        Sel::compact(s, k);
        f.set((uint32_t)(s.thr >> 32), LARGEST);
      }
      if (tid == 0) *n_ok = s.n_buf;
      __syncthreads();
    }
    bool pending = true;
    for (;;) {
      uint32_t mask = 0;
      if (pending) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if (base + u * THREADS + tid < n4) {
#pragma unroll
            for (int q = 0; q < 4; q++) mask |= (f.pass(v[u * 4 + q]) ? 1u : 0u) << (u * 4 + q);
          }
        }
        mask &= ~skip;
      }
      bool retry = false;
      if (__any_sync(FULL_MASK, mask != 0u)) {
        const int cnt = __popc(mask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(FULL_MASK, incl, o);
          if (lane >= o) incl += t;
        }
        int wbase = 0;
        if (lane == 31) wbase = atomicAdd(&s.n_buf, incl);
        wbase = __shfl_sync(FULL_MASK, wbase, 31);
        const int total = __shfl_sync(FULL_MASK, incl, 31);
        if (wbase + total <= C::CAP) {
          int pos = wbase + incl - cnt;
          const uint32_t ib = idx0 + (uint32_t)((base + tid) * 4);
          for (uint32_t m = mask; m; m &= m - 1) {
            const int b = __ffs(m) - 1;
            const float x = select_reg<C::PT>(v, b);
            s.buf[pos++] = composite(ordered_key(x, LARGEST),
                                     ib + (uint32_t)((b >> 2) * THREADS * 4 + (b & 3)));
          }
          if (lane == 31) atomicAdd(n_ok, total);
        } else {
          retry = true;
          if (lane == 31) *overflow = 1;
        }
      }
      pending = retry;
      __syncthreads();
      const bool ovf = *overflow != 0;
      if (!ovf) break;  // uniform: nobody writes the flag between the barriers
      __syncthreads();
      if (tid == 0) {
        s.n_buf = *n_ok;
        *overflow = 0;
      }
      __syncthreads();
      Sel::compact(s, k);
      f.set((uint32_t)(s.thr >> 32), LARGEST);
      if (tid == 0) *n_ok = s.n_buf;
      __syncthreads();
    }
  }
  if (waited < nst) {
    // gave up: let the copies still in flight land (bounded) before the block exits
    if (tid == 0) {
      const int64_t hi = nst < waited + RING_STAGES ? nst : waited + RING_STAGES;
      for (int64_t j = waited; j < hi; j++) {
        const int slot = (int)(j % RING_STAGES);
        const uint64_t t0 = sm100::globaltimer();
        while (!sm100::mbar_try_wait(&full[slot], (uint32_t)((j / RING_STAGES) & 1)) &&
               sm100::globaltimer() - t0 < sm100::WAIT_LIMIT_NS) {
        }
      }
    }
    __syncthreads();
    return;
  }
  Sel::finish(s, k);
  if (segs == 1) {
    for (int j = tid; j < k; j += THREADS) {
      const uint64_t e = s.top[j];
      const uint32_t idx = (uint32_t)e;
      if (idx < (uint32_t)len) {
        outD[row * k + j] = selected_value(e, LARGEST, rowp);
        outI[row * k + j] = (int64_t)idx;
      }
    }
  } else {
    uint64_t* dst = part + unit * k;
    for (int j = tid; j < k; j += THREADS) dst[j] = s.top[j];
  }
}

// k = 1: every thread keeps its best (key, index) - indices grow along a thread's walk,
// so a strict compare keeps the lowest index among equal keys - then a block reduction.
template <int THREADS, bool LARGEST>
__global__ void __launch_bounds__(THREADS)
    kselect_k1_kernel(const float* __restrict__ vals, int64_t len, int segs, int64_t seg_len,
                      float* __restrict__ outD, int64_t* __restrict__ outI,
                      uint64_t* __restrict__ part) {
  __shared__ uint64_t red[THREADS / 32];
  const int tid = threadIdx.x;
  const int64_t row = blockIdx.x / segs;
  const int seg = blockIdx.x % segs;
  const float* rowp = vals + row * len;
  const int64_t s0 = (int64_t)seg * seg_len;
  const int64_t s1 = min(len, s0 + seg_len);
  const int64_t n = s1 - s0;
  const float* p = rowp + s0;
  const int64_t head_e = (int64_t)(((16u - ((uintptr_t)p & 15u)) & 15u) / 4);
  const int head = (int)(n < head_e ? n : head_e);
  const int64_t n4 = (n - head) / 4;
  const int tail = (int)(n - head - n4 * 4);
  uint64_t best = ~0ull;
  if (tid < head) best = composite(ordered_key(p[tid], LARGEST), (uint32_t)(s0 + tid));
  if (tid >= 32 && tid < 32 + tail) {
    const int64_t e = head + n4 * 4 + (tid - 32);
    best = min(best, composite(ordered_key(p[e], LARGEST), (uint32_t)(s0 + e)));
  }
  uint32_t bk = (uint32_t)(best >> 32), bi = (uint32_t)best;
  const float4* p4 = reinterpret_cast<const float4*>(p + head);
  const uint32_t idx0 = (uint32_t)(s0 + head);
  constexpr int UNROLL = 4;
  for (int64_t base = 0; base < n4; base += (int64_t)THREADS * UNROLL) {
    float4 v[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; u++) {
      const int64_t i = base + u * THREADS + tid;
      if (i < n4) v[u] = __ldcs(p4 + i);
    }
#pragma unroll
    for (int u = 0; u < UNROLL; u++) {
      const int64_t i = base + u * THREADS + tid;
      if (i < n4) {
        const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const uint32_t key = ordered_key(x[j], LARGEST);
          const uint32_t idx = idx0 + (uint32_t)(i * 4 + j);
          // head/tail elements may carry larger indices than body ones: full compare
          if (key < bk || (key == bk && idx < bi)) {
            bk = key;
            bi = idx;
          }
        }
      }
    }
  }
  best = composite(bk, bi);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(FULL_MASK, best, o));
  if ((tid & 31) == 0) red[tid >> 5] = best;
  __syncthreads();
  if (tid < 32) {
    best = tid < THREADS / 32 ? red[tid] : ~0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(FULL_MASK, best, o));
    if (tid == 0) {
      if (segs == 1) {
        const uint32_t idx = (uint32_t)best;
        outD[row] = selected_value(best, LARGEST, rowp);
        outI[row] = (int64_t)idx;
      } else {
        part[row * segs + seg] = best;
      }
    }
  }
}

// Selection across the segments' partial results (already composites).
template <int THREADS, int KP>
__global__ void __launch_bounds__(THREADS)
    kselect_merge_kernel(const uint64_t* __restrict__ part, int64_t nper, int k,
                         const float* __restrict__ vals, int64_t len, int largest,
                         float* __restrict__ outD, int64_t* __restrict__ outI) {
  constexpr int CAP = 4096;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(smem_raw);
  const int64_t row = blockIdx.x;
  const uint64_t* src = part + row * nper;
  Sel::init(s);
  __syncthreads();
  uint64_t thr = ~0ull;
  for (int64_t base = 0; base < nper; base += THREADS) {
    const int64_t i = base + threadIdx.x;
    uint64_t c[1];
    uint32_t mask = 0;
    if (i < nper) {
      c[0] = src[i];
      mask = (c[0] != ~0ull && c[0] <= thr) ? 1u : 0u;
    }
    Sel::template push<1>(s, mask, c);
    __syncthreads();
    if (s.n_buf > CAP - THREADS) {
      Sel::compact(s, k);
      thr = s.thr;
    }
  }
  Sel::finish(s, k);
  const float* rowp = vals + row * len;
  for (int j = threadIdx.x; j < k; j += THREADS) {
    const uint64_t e = s.top[j];
    const uint32_t idx = (uint32_t)e;
    outD[row * k + j] = selected_value(e, largest != 0, rowp);
    outI[row * k + j] = (int64_t)idx;
  }
}

template <int KP, int UNROLL, bool LARGEST>
gbk_status launch_rows(const float* vals, int64_t rows, int64_t len, int k, int segs,
                       int64_t seg_len, float* D, int64_t* I, uint64_t* part, cudaStream_t stream) {
  // 4-warp blocks, 8 per SM: the per-iteration barriers synchronise fewer warps, and a
  // block's stall leaves the SM 7 others (measured 1.19-1.22x over 8-warp blocks at
  // k = 32..1024 on 10,000 x 65,536 rows)
  constexpr int THREADS = 128;
  using C = KselCfg<THREADS, KP, UNROLL, LARGEST>;
  auto kern = kselect_rows_kernel<THREADS, KP, UNROLL, LARGEST>;
  GBK_TRY(set_smem_limit(kern, C::SMEM, true));
  kern<<<(unsigned)(rows * segs), THREADS, C::SMEM, stream>>>(vals, len, k, segs, seg_len, D, I,
                                                                part);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

template <int KP, bool LARGEST>
gbk_status launch_ring(const float* vals, int64_t rows, int64_t len, int k, int segs,
                       int64_t seg_len, float* D, int64_t* I, uint64_t* part, cudaStream_t stream) {
  constexpr int THREADS = 256;
  using C = RingCfg<THREADS, KP>;
  auto kern = kselect_ring_kernel<THREADS, KP, LARGEST>;
  GBK_TRY(set_smem_limit(kern, C::SMEM));
  uint32_t* status = device_status();
  if (!status) return set_error(GBK_ECUDA, "device status word unavailable");
  kern<<<(unsigned)(rows * segs), THREADS, C::SMEM, stream>>>(vals, len, k, segs, seg_len, D, I,
                                                                part, status);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

template <bool LARGEST>
gbk_status dispatch_rows(const float* vals, int64_t rows, int64_t len, int k, int segs,
                         int64_t seg_len, float* D, int64_t* I, uint64_t* part,
                         cudaStream_t st, const KselectTuning& tu) {
  if (tu.unroll == 1) {
#define GBK_RING(KP) return launch_ring<KP, LARGEST>(vals, rows, len, k, segs, seg_len, D, I, part, st)
    if (k <= 32) GBK_RING(32);
    if (k <= 64) GBK_RING(64);
    if (k <= 128) GBK_RING(128);
    if (k <= 256) GBK_RING(256);
    if (k <= 512) GBK_RING(512);
    GBK_RING(1024);
#undef GBK_RING
  }
  const bool wide = tu.unroll >= 8;
#define GBK_ROWS(KP)                                                                         \
  return wide ? launch_rows<KP, 8, LARGEST>(vals, rows, len, k, segs, seg_len, D, I, part, st) \
              : launch_rows<KP, 4, LARGEST>(vals, rows, len, k, segs, seg_len, D, I, part, st)
  if (k <= 32) GBK_ROWS(32);
  if (k <= 64) GBK_ROWS(64);
  if (k <= 128) GBK_ROWS(128);
  if (k <= 256) GBK_ROWS(256);
  if (k <= 512) GBK_ROWS(512);
  GBK_ROWS(1024);
#undef GBK_ROWS
}

template <int KP>
gbk_status launch_merge(const uint64_t* part, int64_t rows, int64_t nper, int k,
                        const float* vals, int64_t len, bool largest, float* D, int64_t* I,
                        cudaStream_t stream) {
  constexpr int THREADS = 256;
  using Sel = BlockSelect<THREADS, KP, 4096>;
  auto kern = kselect_merge_kernel<THREADS, KP>;
  GBK_TRY(set_smem_limit(kern, sizeof(typename Sel::Smem)));
  kern<<<(unsigned)rows, THREADS, sizeof(typename Sel::Smem), stream>>>(part, nper, k, vals, len,
                                                                         largest ? 1 : 0, D, I);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status dispatch_merge(const uint64_t* part, int64_t rows, int64_t nper, int k,
                          const float* vals, int64_t len, bool largest, float* D, int64_t* I,
                          cudaStream_t st) {
  if (k <= 32) return launch_merge<32>(part, rows, nper, k, vals, len, largest, D, I, st);
  if (k <= 64) return launch_merge<64>(part, rows, nper, k, vals, len, largest, D, I, st);
  if (k <= 128) return launch_merge<128>(part, rows, nper, k, vals, len, largest, D, I, st);
  if (k <= 256) return launch_merge<256>(part, rows, nper, k, vals, len, largest, D, I, st);
  if (k <= 512) return launch_merge<512>(part, rows, nper, k, vals, len, largest, D, I, st);
  return launch_merge<1024>(part, rows, nper, k, vals, len, largest, D, I, st);
}

}  // namespace

KselectTuning kselect_default_tuning(int64_t rows, int64_t len, int k) {
  KselectTuning t;
  const int sms = device_info().sm_count;
  t.unroll = 8;
  // enough blocks to fill the GPU several times over; segments no shorter than 8K
  const int64_t target = 8ll * sms;
  int64_t segs = 1;
  if (rows < target) {
    const int64_t min_seg = std::max<int64_t>(8192, 8ll * k);
    segs = std::min<int64_t>((target + rows - 1) / rows, std::max<int64_t>(1, len / min_seg));
    segs = std::max<int64_t>(1, std::min<int64_t>(segs, 4096));
  }
  t.segs = (int)segs;
  return t;
}

namespace {

// Segment length (a multiple of 4 floats) and the resulting segment count for a request.
void plan_segments(int64_t len, int want, int64_t* segs_out, int64_t* seg_len_out) {
  int64_t segs = std::max(1, want);
  int64_t seg_len = (len + segs - 1) / segs;
  seg_len = (seg_len + 3) & ~int64_t(3);
  *seg_len_out = seg_len;
  *segs_out = (len + seg_len - 1) / seg_len;
}

// Launches for a plan; `part` must hold rows * segs * k composites when segs > 1.
gbk_status kselect_launch(const float* vals, int64_t rows, int64_t len, int k, bool largest,
                          float* D, int64_t* I, cudaStream_t st, const KselectTuning& tu,
                          int64_t segs, int64_t seg_len, uint64_t* pp) {
  gbk_status r;
  ProfScope prof(k == 1 ? "kselect_k1" : "kselect_rows", st);
  if (k == 1) {
    if (largest)
      kselect_k1_kernel<256, true><<<(unsigned)(rows * segs), 256, 0, st>>>(vals, len, (int)segs,
                                                                           seg_len, D, I, pp);
    else
      kselect_k1_kernel<256, false><<<(unsigned)(rows * segs), 256, 0, st>>>(vals, len, (int)segs,
                                                                            seg_len, D, I, pp);
    GBK_LAUNCH_CHECK();
    r = GBK_OK;
  } else {
    r = largest ? dispatch_rows<true>(vals, rows, len, k, (int)segs, seg_len, D, I, pp, st, tu)
                : dispatch_rows<false>(vals, rows, len, k, (int)segs, seg_len, D, I, pp, st, tu);
  }
  if (r != GBK_OK || segs == 1) return r;
  const int64_t nper = segs * (k == 1 ? 1 : k);
  return dispatch_merge(pp, rows, nper, k, vals, len, largest, D, I, st);
}

}  // namespace

gbk_status kselect_run(const float* vals, int64_t rows, int64_t len, int k, bool largest,
                       float* D, int64_t* I, cudaStream_t st, const KselectTuning* tuning) {
  if (rows == 0) return GBK_OK;
  KselectTuning tu = tuning ? *tuning : kselect_default_tuning(rows, len, k);
  int64_t segs, seg_len;
  plan_segments(len, tu.segs, &segs, &seg_len);
  Scratch part;
  if (segs > 1) {
    gbk_status r = part.alloc(sizeof(uint64_t) * (size_t)(rows * segs * k), st);
    if (r != GBK_OK) return r;
  }
  return kselect_launch(vals, rows, len, k, largest, D, I, st, tu, segs, seg_len,
                        part.as<uint64_t>());
}

// ------------------------------------------------------------------ no-allocation variant
//
// Some callers cannot allocate device memory at call time: code running while a CUDA graph
// is being captured with a memory pool they do not own, real-time paths that forbid any
// allocator call after start-up, and hosts whose only allocator is their own (a tensor
// framework's caching allocator the library is not wired to).  For them the segmented
// two-pass k-selection keeps its per-segment partial results in this fixed array instead
// of scratch memory.  The array is part of the library image: every GPU that loads the
// library holds it (16 MiB) until the process exits.  All calls share it and it keeps the
// contents of the last call; each call fully writes the partials it then reads, so nothing
// needs clearing, but calls whose executions overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
constexpr int64_t STATIC_PART_ELEMS = (int64_t)2 << 20;  // composites (16 MiB)
static __device__ __align__(256) uint64_t g_static_part[STATIC_PART_ELEMS];

namespace {
// Device address of g_static_part, looked up once per device with that device current
// (in host code the symbol's name is only a host-side stand-in).
uint64_t* static_part_address(gbk_status* st) {
  static std::mutex mu;
  static uint64_t* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *st = set_error(GBK_ECUDA, "gbk_kselect_static: no current device");
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_part);
    if (e != cudaSuccess) {
      *st = set_error(GBK_ECUDA, "gbk_kselect_static: cudaGetSymbolAddress: %s",
                      cudaGetErrorString(e));
      return nullptr;
    }
    addr[dev] = static_cast<uint64_t*>(p);
  }
  return addr[dev];
}
}  // namespace

gbk_status kselect_static_run(const float* vals, int64_t rows, int64_t len, int k, bool largest,
                              int segments, float* D, int64_t* I, cudaStream_t st) {
  if (rows == 0) return GBK_OK;
  KselectTuning tu = kselect_default_tuning(rows, len, k);
  if (segments > 0) tu.segs = segments;
  int64_t segs, seg_len;
  plan_segments(len, tu.segs, &segs, &seg_len);
  if (segs > 1 && rows * segs * (int64_t)k > STATIC_PART_ELEMS)
    return set_error(GBK_EINVAL,
                     "gbk_kselect_static: rows*segments*k = %lld exceeds the fixed capacity of "
                     "%lld partial results",
                     (long long)(rows * segs * (int64_t)k), (long long)STATIC_PART_ELEMS);
  gbk_status r = GBK_OK;
  uint64_t* pp = segs > 1 ? static_part_address(&r) : nullptr;
  if (segs > 1 && !pp) return r;
  return kselect_launch(vals, rows, len, k, largest, D, I, st, tu, segs, seg_len, pp);
}

}  // namespace gbk
