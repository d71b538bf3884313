// Block-wide streaming k-selection used by every selecting kernel of the library.
//
// Definition followed: section 2 "k-selection" of the paper (the k lowest values of an
// array, sorted, with their indices).  The kernels never keep a sorted order while
// streaming.  Instead:
//   * every candidate is a 64-bit composite  (ordered 32-bit key << 32) | 32-bit index,
//     where the ordered key maps float order to unsigned order (NaN worst, -0 == +0).
//     Composite order is then the library's total order: value first, lower index on
//     ties, so one unsigned compare settles everything and all composites are distinct;
//   * threads filter incoming values against the block's threshold (the value of the
//     k-th best composite seen so far) held in a register, and append survivors to a
//     shared-memory buffer with one atomic per warp;
//   * when the buffer nears capacity the block computes the exact k best of
//     (kept set U buffer) with an MSB-first radix select over the composites and keeps
//     only those; the threshold drops to their maximum.
// The paper's own design (WarpSelect: per-lane register queues merged with odd-size
// bitonic networks, section 4) is prior art for Maxwell; this one spends shared memory
// instead of registers, which sm_103a has in abundance (228 KB per SM), and touches each
// input element with one compare.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbk {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr uint32_t NAN_KEY = 0xffffffffu;

// Map a float to an unsigned key whose order is the selection order.  `largest`
// selects the highest values: the key of v is then the key of -v.
__device__ __forceinline__ uint32_t ordered_key(float v, bool largest) {
  if (largest) v = -v;
  uint32_t b = __float_as_uint(v);
  if (v != v) return NAN_KEY;
  if (b == 0x80000000u) b = 0u;  // -0 ranks with +0
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Inverse of ordered_key for non-NaN keys (returns the value in the original sense).
__device__ __forceinline__ float key_value(uint32_t k, bool largest) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  float v = __uint_as_float(b);
  return largest ? -v : v;
}

// The input value of a selected composite e (index in its low word into `row`).  The key
// is a bijection of the float's bits except that -0 and +0 share a key and every NaN maps
// to NAN_KEY: only those are read back from the input (the sign of a zero, a NaN's
// payload); every other value is rebuilt from the key, which saves a scattered read per
// selected element.
__device__ __forceinline__ float selected_value(uint64_t e, bool largest, const float* row) {
  const uint32_t key = (uint32_t)(e >> 32);
  if (key == NAN_KEY || key == 0x80000000u) return row[(uint32_t)e];
  return key_value(key, largest);
}

__device__ __forceinline__ uint64_t composite(uint32_t key, uint32_t idx) {
  return ((uint64_t)key << 32) | (uint64_t)idx;
}

__device__ __forceinline__ uint64_t shr64(uint64_t x, int s) { return s >= 64 ? 0ull : (x >> s); }

// Threshold filter in value space: pass(v) is true for every v whose key is <= the
// threshold key (ties pass and are settled exactly at compaction).
struct ValueFilter {
  float thr;
  bool nan_ok;
  bool largest;
  __device__ __forceinline__ void set(uint32_t thr_key, bool lg) {
    largest = lg;
    if (thr_key == NAN_KEY) {
      nan_ok = true;
      thr = lg ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000);
    } else {
      nan_ok = false;
      thr = key_value(thr_key, lg);
    }
  }
  __device__ __forceinline__ bool pass(float v) const {
    return (largest ? (v >= thr) : (v <= thr)) || nan_ok;
  }
};

// One shared atomic per warp: returns this lane's slot among the lanes with `want`.
__device__ __forceinline__ int warp_reserve(int& counter, bool want) {
  const int lane = threadIdx.x & 31;
  const unsigned b = __ballot_sync(FULL_MASK, want);
  int base = 0;
  if (b && lane == __ffs(b) - 1) base = atomicAdd(&counter, __popc(b));
  base = __shfl_sync(FULL_MASK, base, b ? __ffs(b) - 1 : 0);
  return base + __popc(b & ((1u << lane) - 1u));
}

template <int THREADS, int KP, int CAP>
struct BlockSelect {
  static_assert(THREADS % 32 == 0, "whole warps");
  static_assert((KP & (KP - 1)) == 0 && KP >= 32, "KP power of two >= 32");
  struct Smem {
    uint64_t top[KP];   // kept set (unordered until finish)
    uint64_t buf[CAP];  // candidates appended since the last compaction
    uint32_t hist[256];
    uint64_t thr;       // max kept composite once n_top == k, else ~0 (everything passes)
    uint64_t diff, tmax, P;
    int n_top, n_buf, need, shift, done, cnt;
  };

  __device__ static void init(Smem& s) {
    if (threadIdx.x == 0) {
      s.n_top = 0;
      s.n_buf = 0;
      s.thr = ~0ull;
    }
  }

  // Warp-aggregated append.  Every lane of the warp must call it; lane l offers the
  // composites c[j] for which bit j of `mask` is set.
  template <int NV>
  __device__ __forceinline__ static void push(Smem& s, uint32_t mask, const uint64_t (&c)[NV]) {
    const int lane = threadIdx.x & 31;
    if (!__any_sync(FULL_MASK, mask != 0u)) return;
    int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(FULL_MASK, incl, o);
      if (lane >= o) incl += t;
    }
    int base = 0;
    if (lane == 31) base = atomicAdd(&s.n_buf, incl);
    base = __shfl_sync(FULL_MASK, base, 31);
    int pos = base + incl - cnt;
#pragma unroll
    for (int j = 0; j < NV; j++) {
      if (mask & (1u << j)) s.buf[pos++] = c[j];
    }
  }

  // Exact k best of top U buf; all threads call it after a __syncthreads().  Kept out of
  // line: it is the rare path and must not inflate the streaming loop's registers.
  __device__ __noinline__ static void compact(Smem& s, int k) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int n_top = s.n_top, n_buf = s.n_buf;
    const int total = n_top + n_buf;
    if (total <= k) {
      for (int i = tid; i < n_buf; i += THREADS) s.top[n_top + i] = s.buf[i];
      __syncthreads();
      if (tid == 0) {
        s.n_top = total;
        s.n_buf = 0;
        s.tmax = 0ull;
      }
      __syncthreads();
      if (total == k) {
        uint64_t m = 0ull;
        for (int i = tid; i < total; i += THREADS) m = max(m, s.top[i]);
        atomicMax((unsigned long long*)&s.tmax, (unsigned long long)m);
        __syncthreads();
        if (tid == 0) s.thr = s.tmax;
      }
      __syncthreads();
      return;
    }
    // 1. bits shared by every element
    const uint64_t x0 = n_top > 0 ? s.top[0] : s.buf[0];
    if (tid == 0) s.diff = 0ull;
    __syncthreads();
    uint64_t dacc = 0ull;
    for (int i = tid; i < total; i += THREADS) {
      uint64_t e = i < n_top ? s.top[i] : s.buf[i - n_top];
      dacc |= e ^ x0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dacc |= __shfl_xor_sync(FULL_MASK, dacc, o);
    if (lane == 0 && dacc) atomicOr((unsigned long long*)&s.diff, (unsigned long long)dacc);
    __syncthreads();
    int shift = 64 - __clzll((long long)s.diff);  // distinct composites -> diff != 0
    uint64_t P = shr64(x0, shift);
    int need = k;
    // 2. MSB-first radix select of the need-th smallest composite.  Digits never straddle
    //    the 32-bit word boundary, so every test below is a 32-bit operation.
    for (;;) {
      const int w = shift > 32 ? min(8, shift - 32) : min(8, shift);
      const int nshift = shift - w;
      const uint32_t dmask = (1u << w) - 1u;
      // prefix test (e >> shift) == P split into words
      const bool hi_only = shift >= 32;
      const uint32_t ph = hi_only ? (uint32_t)P : (uint32_t)(P >> (32 - shift));
      const int sh_h = hi_only ? shift - 32 : 0;
      const uint32_t pl = hi_only ? 0u : (shift == 32 ? 0u : (uint32_t)P & (uint32_t)((1ull << (32 - shift)) - 1ull));
      const bool dig_hi = nshift >= 32;
      const int dsh = dig_hi ? nshift - 32 : nshift;
      for (int i = tid; i < 256; i += THREADS) s.hist[i] = 0u;
      __syncthreads();
      // warp-aggregated: one shared atomic per distinct digit per warp (the digits of
      // surviving candidates are highly skewed, plain atomics would serialise)
      for (int i0 = 0; i0 < total; i0 += THREADS) {
        const int i = i0 + tid;
        uint32_t bin = 0xffffffffu;
        if (i < total) {
          const uint64_t e = i < n_top ? s.top[i] : s.buf[i - n_top];
          const uint32_t eh = (uint32_t)(e >> 32), el = (uint32_t)e;
          const bool match = hi_only ? (sh_h >= 32 ? true : (eh >> sh_h) == ph)
                                     : (eh == ph && (shift == 32 ? true : (el >> shift) == pl));
          if (match) bin = ((dig_hi ? eh : el) >> dsh) & dmask;
        }
        const unsigned grp = __match_any_sync(FULL_MASK, bin);
        if (bin != 0xffffffffu && lane == __ffs(grp) - 1) atomicAdd(&s.hist[bin], (uint32_t)__popc(grp));
      }
      __syncthreads();
      if (tid < 32) {
        // lane owns bins [8*lane, 8*lane+8)
        uint32_t h[8];
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
          h[j] = s.hist[lane * 8 + j];
          sum += h[j];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t t = __shfl_up_sync(FULL_MASK, incl, o);
          if (lane >= o) incl += t;
        }
        uint32_t excl = incl - sum;
        if (excl < (uint32_t)need && (uint32_t)need <= incl) {
          uint32_t cum = excl;
#pragma unroll
          for (int j = 0; j < 8; j++) {
            if (cum < (uint32_t)need && (uint32_t)need <= cum + h[j]) {
              const int nneed = need - (int)cum;
              s.need = nneed;
              s.P = (P << w) | (uint64_t)(lane * 8 + j);
              s.shift = nshift;
              s.done = (h[j] == (uint32_t)nneed) || nshift == 0;
            }
            cum += h[j];
          }
        }
      }
      __syncthreads();
      need = s.need;
      P = s.P;
      shift = s.shift;
      const int done = s.done;
      __syncthreads();
      if (done) break;
    }
    // 3. keep e iff (e >> shift) <= P : exactly k elements
    constexpr int TPT = (KP + THREADS - 1) / THREADS;
    uint64_t mine[TPT];
#pragma unroll
    for (int j = 0; j < TPT; j++) {
      int i = tid + j * THREADS;
      mine[j] = i < n_top ? s.top[i] : ~0ull;
    }
    if (tid == 0) {
      s.cnt = 0;
      s.tmax = 0ull;
    }
    __syncthreads();
    // (e >> shift) <= P  <=>  e <= (P << shift) | (2^shift - 1)
    const uint64_t lim = shift >= 64 ? ~0ull : ((P << shift) | ((1ull << shift) - 1ull));
    uint64_t m = 0ull;
#pragma unroll
    for (int j = 0; j < TPT; j++) {
      const int i = tid + j * THREADS;
      const bool keep = i < n_top && mine[j] <= lim;
      const int pos = warp_reserve(s.cnt, keep);
      if (keep) {
        s.top[pos] = mine[j];
        m = max(m, mine[j]);
      }
    }
    for (int i0 = 0; i0 < n_buf; i0 += THREADS) {
      const int i = i0 + tid;
      uint64_t e = i < n_buf ? s.buf[i] : ~0ull;
      const bool keep = i < n_buf && e <= lim;
      const int pos = warp_reserve(s.cnt, keep);
      if (keep) {
        s.top[pos] = e;
        m = max(m, e);
      }
    }
    atomicMax((unsigned long long*)&s.tmax, (unsigned long long)m);
    __syncthreads();
    if (tid == 0) {
      s.n_top = s.cnt;
      s.n_buf = 0;
      s.thr = s.tmax;
    }
    __syncthreads();
  }

  // Final compaction and ascending sort of the kept set into top[0..KP); padding ~0.
  __device__ __noinline__ static void finish(Smem& s, int k) {
    __syncthreads();
    compact(s, k);
    const int n = s.n_top;
    for (int i = n + threadIdx.x; i < KP; i += THREADS) s.top[i] = ~0ull;
    __syncthreads();
    constexpr int E = KP / THREADS;  // elements per thread in the register sort
    if constexpr ((THREADS & (THREADS - 1)) == 0 && E >= 2 && E <= 16) {
      sort_registers(s);
    } else {
    for (int size = 2; size <= KP; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = threadIdx.x; t < KP / 2; t += THREADS) {
          int lo = 2 * t - (t & (stride - 1));
          int hi = lo + stride;
          bool asc = (lo & size) == 0;
          uint64_t a = s.top[lo], b = s.top[hi];
          if ((a > b) == asc) {
            s.top[lo] = b;
            s.top[hi] = a;
          }
        }
        __syncthreads();
      }
    }
    }
  }

  // The same bitonic network with thread t holding elements t*E .. t*E+E-1 in registers:
  // strides below E compare within a thread, strides below 32 E between the lanes of a
  // warp (shuffles), only the longer ones go through shared memory with block barriers
  // (3 of the 55 stages at KP = 1024 with 128 threads).
  __device__ static void sort_registers(Smem& s) {
    constexpr int E = KP / THREADS;
    const int t = threadIdx.x;
    uint64_t v[E];
#pragma unroll
    for (int r = 0; r < E; r++) v[r] = s.top[t * E + r];
    for (int size = 2; size <= KP; size <<= 1) {
      int stride = size >> 1;
      if (stride >= 32 * E) {  // partners in other warps
#pragma unroll
        for (int r = 0; r < E; r++) s.top[t * E + r] = v[r];
        __syncthreads();
        for (; stride >= 32 * E; stride >>= 1) {
          for (int p = t; p < KP / 2; p += THREADS) {
            const int lo = 2 * p - (p & (stride - 1));
            const int hi = lo + stride;
            const bool asc = (lo & size) == 0;
            const uint64_t a = s.top[lo], b = s.top[hi];
            if ((a > b) == asc) {
              s.top[lo] = b;
              s.top[hi] = a;
            }
          }
          __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < E; r++) v[r] = s.top[t * E + r];
        __syncthreads();  // every thread has read before the next write-back
      }
      for (; stride >= E; stride >>= 1) {  // partner lane t ^ (stride / E), same slot
        const int tm = stride / E;
        const bool lower = (t & tm) == 0;
#pragma unroll
        for (int r = 0; r < E; r++) {
          const uint64_t o = __shfl_xor_sync(FULL_MASK, v[r], tm);
          const bool asc = ((t * E + r) & size) == 0;
          v[r] = (lower == asc) ? min(v[r], o) : max(v[r], o);
        }
      }
#pragma unroll
      for (int st = E / 2; st >= 1; st >>= 1) {  // within the thread
        if (st < size) {
#pragma unroll
          for (int r = 0; r < E; r++) {
            if ((r & st) == 0) {
              const bool asc = ((t * E + r) & size) == 0;
              const uint64_t a = v[r], b = v[r + st];
              if ((a > b) == asc) {
                v[r] = b;
                v[r + st] = a;
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < E; r++) s.top[t * E + r] = v[r];
    __syncthreads();
  }
};

}  // namespace gbk
