// List-scan kernels of the IVFADC search (section 5.3, Algorithm 4): the per-query
// table scan and the direct-table scan with their fused k-selection, and the launch
// templates.  Each ivf_scan_m<M>.cu instantiates them for one code size M; the layout
// of tables and codes is described in ivf_scan.cu.
#pragma once
#include <algorithm>

#include "common.cuh"
#include "ivf.cuh"
#include "select_core.cuh"

namespace gbk {

// --------------------------------------------------------------------- scan

template <int M>
__device__ __forceinline__ void load_code(const uint8_t* codes, int64_t i, uint32_t (&w)[M / 4]) {
  if constexpr (M == 4) {
    w[0] = __ldg(reinterpret_cast<const uint32_t*>(codes) + i);
  } else if constexpr (M == 8) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(codes) + i);
    w[0] = v.x;
    w[1] = v.y;
  } else if constexpr (M == 16) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(codes) + i);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  } else if constexpr (M % 16 == 0) {  // 32, 48, 64 bytes: 16-byte loads
#pragma unroll
    for (int h = 0; h < M / 16; h++) {
      const uint4 a = __ldg(reinterpret_cast<const uint4*>(codes) + (M / 16) * i + h);
      w[4 * h + 0] = a.x;
      w[4 * h + 1] = a.y;
      w[4 * h + 2] = a.z;
      w[4 * h + 3] = a.w;
    }
  } else if constexpr (M % 8 == 0) {  // 24, 40, 56 bytes: 8-byte loads
#pragma unroll
    for (int h = 0; h < M / 8; h++) {
      const uint2 a = __ldg(reinterpret_cast<const uint2*>(codes) + (M / 8) * i + h);
      w[2 * h + 0] = a.x;
      w[2 * h + 1] = a.y;
    }
  } else {  // other multiples of 4 bytes: 4-byte loads
#pragma unroll
    for (int h = 0; h < M / 4; h++)
      w[h] = __ldg(reinterpret_cast<const uint32_t*>(codes) + (M / 4) * i + h);
  }
}

// Pairwise sum of N values in place (t[j] += t[j + h] for h = P/2, ..., 1 with P the
// power of two >= N; for a power-of-two N the usual halving tree).
template <int N>
__device__ __forceinline__ float pair_sum(float (&t)[N]) {
  constexpr int P = N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : N <= 32 ? 32 : 64;
#pragma unroll
  for (int h = P / 2; h >= 1; h >>= 1)
#pragma unroll
    for (int j = 0; j < h; j++)
      if (j + h < N) t[j] += t[j + h];
  return t[0];
}

// Code sizes other than 4, 8, 16, 32 bytes get one light launch shape (256 threads, two
// codes per thread) to keep the number of instantiated kernels small.
template <int M>
constexpr bool light_shape() {
  return (M & (M - 1)) != 0 || M > 32;
}

struct ScanArgs {
  int64_t nq;
  int nprobe, k;
  const int64_t* cl_I;   // [nq][nprobe] probed lists, nearest first (-1 = none)
  const float* cl_D;     // [nq][nprobe] term 2 = ||x - c_L||^2
  const float* s1;       // table mode: [ntotal] term 1 summed over each stored code
  const float* t3;       // table mode: [nq][256][M] term 3
  const float* xq;       // direct tables: queries
  const float* coarse;   // direct tables: coarse centroids
  const float* pq;       // direct tables: codebooks [M][256][dsub]
  int d;
  int direct;            // 1: LUT[m][c] = ||(x - c_L)^m - C_m[c]||^2 computed per list
  const int64_t* list_off;
  const uint8_t* codes;  // list order, rotated by list position (see the file comment)
  const int64_t* ids;    // null: list positions out instead of ids
  float* D;
  int64_t* I;
  // mixed batches (all optional): per-query k and nprobe (<= k, nprobe above), output
  // offsets (results of query q at D/I + out_off[q]); persistent mode takes queries from
  // `order` through the atomic `counter`.
  const int32_t* kq;
  const int32_t* npq;
  const int64_t* out_off;
  const int64_t* order;
  unsigned long long* counter;
};

// Next query of a block: static (block b serves queries b, b + grid, ...) or from the
// persistent work queue.  Uniform across the block; -1 when none is left.
__device__ __forceinline__ int64_t next_query(const ScanArgs& a, int64_t it, int64_t* q_sh) {
  if (!a.counter) return it < a.nq ? it : -1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long w = atomicAdd(a.counter, 1ull);
    *q_sh = w < (unsigned long long)a.nq ? a.order[w] : -1;
  }
  __syncthreads();
  return *q_sh;
}

// Sorted k best of a query (after the scan) to D/I at offset ob; ids of the winners only
// (section 5.3), (+inf, -1) padding.
template <class Sel>
__device__ __forceinline__ void write_results(const ScanArgs& a, typename Sel::Smem& s, int kq,
                                              int64_t ob) {
  Sel::finish(s, kq);
  for (int j = threadIdx.x; j < kq; j += (int)blockDim.x) {
    const uint64_t e = s.top[j];
    if (e == ~0ull) {
      a.D[ob + j] = __int_as_float(0x7f800000);
      a.I[ob + j] = -1;
    } else {
      a.D[ob + j] = key_value((uint32_t)(e >> 32), false);
      a.I[ob + j] = a.ids ? a.ids[(uint32_t)e] : (int64_t)(uint32_t)e;
    }
  }
}

// Table mode.  Block per query.  Its term-3 table sits in shared memory as 256 rows of 64
// words: word s of row c holds Q_x[s mod M][c] (s < 31 + M used), so lane l at step s reads
// word l + s: bank (l + s) mod 32, distinct across the warp.  The probed lists are laid end
// to end in a virtual range, each padded to a multiple of 32 positions, and the block walks
// that range STEP = THREADS U positions at a time: every warp-chunk of 32 positions lies in
// one list (lane = list position mod 32) and no step is left short by a list's end.  Each
// thread keeps the record of the list its positions are in (virtual start and end, offset
// to the stored position, term 2) in registers and reads the next one only at a list
// boundary.  Codes and term-1 sums of the next step are loaded (into the other of two
// register buffers) while the current step is scored; the k best are kept by the block
// selection (a single pass, section 4) and ids looked up for the winners only (5.3).
template <int M, int U>
struct TableStep {
  uint32_t w[U][M / 4];  // codes
  uint32_t pos[U];       // stored positions (0xffffffff: padding)
  float s1[U];           // term-1 sums (added when scored: the load is not waited for here)
  float base[U];         // term 2 of the list
};

// Words per row of the table kernel's term-3 table: lane l reads word l + s at step s < M.
template <int M>
constexpr int table_row_words() {
  return M <= 32 ? 64 : 128;
}

// Byte offset of the table kernel's list records in dynamic shared memory: after the
// term-3 table and the selection state, rounded up to 16 bytes for the 16-byte records.
template <int M, int KP>
constexpr size_t table_rec_offset() {
  return (sizeof(float) * 256 * table_row_words<M>() +
          sizeof(typename BlockSelect<256, KP, 4096>::Smem) + 15) /
         16 * 16;
}

template <int M, int KP, int U, int THREADS>
__global__ void __launch_bounds__(THREADS, 2)
    ivf_scan_table_kernel(const ScanArgs a) {
  constexpr int CAP = 4096, LW = table_row_words<M>();
  constexpr int STEP = THREADS * U;
  constexpr uint32_t NONE = 0xffffffffu;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* lut = reinterpret_cast<float*>(smem_raw);  // [256][LW]
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(lut + 256 * LW);
  // per probed list p: {virtual start, stored position - virtual position, virtual end,
  // term 2}; record npq holds {virtual total, ...}
  uint4* rec = reinterpret_cast<uint4*>(smem_raw + table_rec_offset<M, KP>());  // [nprobe + 1]
  __shared__ int64_t q_sh;
  __shared__ uint32_t wsum[THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lane4 = (uint32_t)lane * 4u;
  for (int64_t it = blockIdx.x;; it += gridDim.x) {
    const int64_t q = next_query(a, it, &q_sh);
    if (q < 0) break;
    const int kq = a.kq ? a.kq[q] : a.k;
    const int npq = a.npq ? min(a.npq[q], a.nprobe) : a.nprobe;
    const int64_t ob = a.out_off ? a.out_off[q] : q * (int64_t)a.k;
    __syncthreads();  // the previous query's tables are no longer read
    {
      const float4* t3q = reinterpret_cast<const float4*>(a.t3 + q * M * 256);
      float4* l4 = reinterpret_cast<float4*>(lut);
      for (int e = tid; e < 256 * LW / 4; e += THREADS) {
        const int c = e / (LW / 4), w4 = e % (LW / 4);  // words 4 w4 .. 4 w4 + 3 of row c
        const float4 t = __ldg(t3q + (c * M + (4 * w4) % M) / 4);  // M % 4 == 0: no wrap
        l4[e] = make_float4(-2.f * t.x, -2.f * t.y, -2.f * t.z, -2.f * t.w);
      }
    }
    {  // list records: lengths rounded up to 32 laid end to end (block-wide exclusive scan)
      const int ppt = (npq + THREADS - 1) / THREADS;
      uint32_t loc = 0;
      for (int j = 0; j < ppt; j++) {
        const int p = tid * ppt + j;
        if (p < npq) {
          const int64_t L = a.cl_I[q * a.nprobe + p];
          uint32_t st = 0, sz = 0, b = 0;
          if (L >= 0) {
            const int64_t o0 = a.list_off[L];
            st = (uint32_t)o0;
            sz = (uint32_t)(a.list_off[L + 1] - o0);
            b = __float_as_uint(a.cl_D[q * a.nprobe + p]);
          }
          rec[p] = make_uint4(sz, st, 0u, b);
          loc += (sz + 31u) & ~31u;
        }
      }
      uint32_t inc = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane == 31) wsum[warp] = inc;
      __syncthreads();
      uint32_t run = inc - loc;
      for (int w2 = 0; w2 < warp; w2++) run += wsum[w2];
      for (int j = 0; j < ppt; j++) {
        const int p = tid * ppt + j;
        if (p < npq) {
          const uint4 r0 = rec[p];  // {length, first stored position, -, term 2}
          rec[p] = make_uint4(run, r0.y - run, run + r0.x, r0.w);
          run += (r0.x + 31u) & ~31u;
        }
      }
      if (tid == THREADS - 1) rec[npq] = make_uint4(run, 0u, 0u, 0u);
    }
    Sel::init(s);
    __syncthreads();
    const uint32_t total = rec[npq].x;
    float thr = __int_as_float(0x7f800000);  // filter: pass unless above (NaN always passes)
    // this thread's list: record fields in registers; n_start = start of the next list
    int pw = -1;
    uint32_t c_off = 0, c_end = 0, c_base = 0, n_start = 0;
    auto fetch = [&](TableStep<M, U>& b, uint32_t v0) {
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint32_t v = v0 + (uint32_t)(u * THREADS + tid);
        b.pos[u] = NONE;
        if (v < total) {
          while (v >= n_start) {  // list boundary (rare): the next non-empty list's record
            pw++;
            const uint4 r = rec[pw];
            c_off = r.y;
            c_end = r.z;
            c_base = r.w;
            n_start = rec[pw + 1].x;
          }
          if (v < c_end) {
            const uint32_t i = v + c_off;
            b.pos[u] = i;
            load_code<M>(a.codes, i, b.w[u]);
            b.s1[u] = __ldg(a.s1 + i);
            b.base[u] = __uint_as_float(c_base);
          }
        }
      }
    };
    auto score = [&](const TableStep<M, U>& b) {
      uint32_t mask = 0;
      uint64_t cc[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        cc[u] = ~0ull;
        if (b.pos[u] != NONE) {
          // all look-ups first, then a pairwise sum: the loads overlap instead of each
          // waiting on the previous add (codes over 32 bytes: groups of 16, 8 or 4 look-ups,
          // each summed pairwise, then the group sums pairwise, to bound the registers)
          constexpr int G = M <= 32 ? M : M % 16 == 0 ? 16 : M % 8 == 0 ? 8 : 4;
          float gs[M / G];
#pragma unroll
          for (int gi = 0; gi < M / G; gi++) {
            float t[G];
#pragma unroll
            for (int j = 0; j < G; j++) {
              const int st = gi * G + j;
              uint32_t addr;
              if constexpr (LW == 64) {
                // (code byte st) * 256 + 4 lane: row of the code, word lane (+ st below)
                addr = __byte_perm(b.w[u][st >> 2], lane4, 0x6504u | ((st & 3) << 4));
              } else {
                addr = ((b.w[u][st >> 2] >> (8 * (st & 3))) & 255u) * (LW * 4u) + lane4;
              }
              t[j] = *reinterpret_cast<const float*>(smem_raw + addr + st * 4);
            }
            gs[gi] = pair_sum<G>(t);
          }
          const float dist = b.base[u] + (b.s1[u] + pair_sum<M / G>(gs));
          if (!(dist > thr)) {  // exact order is settled at compaction
            mask |= 1u << u;
            cc[u] = composite(ordered_key(dist, false), b.pos[u]);
          }
        }
      }
      Sel::template push<U>(s, mask, cc);
      __syncthreads();
      // compact when the buffer fills, and once early, as soon as a step's worth of
      // candidates is there while fewer than k are kept: the k-th of them becomes the
      // threshold, so later steps push a fraction of their codes instead of all of them
      // (uniform: both counts are read after the barrier)
      if (s.n_buf > CAP - STEP || (s.n_top < kq && s.n_buf >= STEP)) {
        Sel::compact(s, kq);
        const uint32_t tk = (uint32_t)(s.thr >> 32);
        thr = tk == NAN_KEY ? __int_as_float(0x7f800000) : key_value(tk, false);
      }
    };
    TableStep<M, U> A, B;
    if (total > 0) fetch(A, 0);
    for (uint32_t v0 = 0; v0 < total; v0 += 2 * STEP) {  // ping-pong between A and B
      if (v0 + STEP < total) fetch(B, v0 + STEP);
      score(A);
      if (v0 + STEP >= total) break;
      if (v0 + 2 * STEP < total) fetch(A, v0 + 2 * STEP);
      score(B);
    }
    write_results<Sel>(a, s, kq, ob);
  }
}

// Direct mode (no precomputed tables).  Block per query; for each probed list the LUT
// [256][DW] (DW = M ceil(32 / M): 32 for M dividing 32, M above 32) holds LUT[m][c] =
// ||(x - c_L)^m - C_m[c]||^2 at word c*DW + h*M + m for every copy h < DW/M, and lane l
// (copy h = l / M) reads sub-table (s + l) mod M at step s: 32 distinct words of a row (32
// distinct banks when M divides 32 or is 64).  Codes are streamed U per thread
// per step from the list's start, so lane l always holds a position r = l (mod 32) of the
// list.
template <int M, int KP, int U>
__global__ void __launch_bounds__(256)
    ivf_scan_direct_kernel(const ScanArgs a) {
  constexpr int THREADS = 256, CAP = 4096, STEP = THREADS * U, DW = (32 + M - 1) / M * M;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* lut = reinterpret_cast<float*>(smem_raw);  // [256][DW]
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(lut + 256 * DW);
  __shared__ int64_t q_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rot = lane % M, h = lane / M;
  const int dsub = a.d / M;
  for (int64_t it = blockIdx.x;; it += gridDim.x) {
    const int64_t q = next_query(a, it, &q_sh);
    if (q < 0) break;
    const int kq = a.kq ? a.kq[q] : a.k;
    const int npq = a.npq ? min(a.npq[q], a.nprobe) : a.nprobe;
    const int64_t ob = a.out_off ? a.out_off[q] : q * (int64_t)a.k;
    __syncthreads();
    Sel::init(s);
    __syncthreads();
    ValueFilter f;
    f.set(NAN_KEY, false);
    for (int p = 0; p < npq; p++) {
      const int64_t L = a.cl_I[q * a.nprobe + p];
      if (L < 0) continue;  // uniform across the block
      const int64_t o0 = a.list_off[L], o1 = a.list_off[L + 1];
      __syncthreads();  // the previous list's look-ups are done
      // warp w fills rows c of its 32; lane l computes the entries w = l, l + 32, ... < DW
      // of row c (entry w: sub-quantizer w mod M, copy w / M)
      for (int i = 0; i < 32; i++) {
        const int c = warp * 32 + i;
#pragma unroll
        for (int wd = lane; wd < DW; wd += 32) {
          const int m = wd % M;
          const float* C = a.pq + ((int64_t)m * 256 + c) * dsub;
          float v = 0.f;
          for (int t = 0; t < dsub; t++) {
            const float r = a.xq[q * a.d + m * dsub + t] - a.coarse[L * a.d + m * dsub + t];
            const float e2 = r - C[t];
            v = fmaf(e2, e2, v);
          }
          lut[c * DW + wd] = v;
        }
      }
      __syncthreads();
      for (int64_t b0 = o0; b0 < o1; b0 += STEP) {
        uint32_t mask = 0;
        uint64_t cc[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int64_t i = b0 + u * THREADS + tid;
          cc[u] = ~0ull;
          if (i < o1) {
            uint32_t w[M / 4];
            load_code<M>(a.codes, i, w);
            float acc = 0.f;
#pragma unroll
            for (int st = 0; st < M; st++) {
              const uint32_t c = (w[st >> 2] >> ((st & 3) * 8)) & 255u;
              int m;
              if constexpr ((M & (M - 1)) == 0) {
                m = (st + rot) & (M - 1);
              } else {
                m = st + rot;  // < 2M
                m -= m >= M ? M : 0;
              }
              acc += lut[c * DW + h * M + m];
            }
            if (f.pass(acc)) {
              mask |= 1u << u;
              cc[u] = composite(ordered_key(acc, false), (uint32_t)i);
            }
          }
        }
        Sel::template push<U>(s, mask, cc);
        __syncthreads();
        if (s.n_buf > CAP - STEP || (s.n_top < kq && s.n_buf >= STEP)) {  // as above
          Sel::compact(s, kq);
          f.set((uint32_t)(s.thr >> 32), false);
        }
      }
    }
    write_results<Sel>(a, s, kq, ob);
  }
}

template <int M, int KP, int U>
static gbk_status launch_scan(const ScanArgs& a, const ScanTuning& tun, cudaStream_t st) {
  using Sel = BlockSelect<256, KP, 4096>;
  size_t smem;
  void (*kern)(const ScanArgs);
  int threads = 256;
  // the light shape: two codes per thread (up to 16 code words each in registers)
  constexpr int UC = light_shape<M>() ? 2 : U;
  if (a.direct) {
    kern = ivf_scan_direct_kernel<M, KP, UC>;
    smem = sizeof(float) * 256 * ((32 + M - 1) / M * M) + sizeof(typename Sel::Smem);
  } else if constexpr (light_shape<M>()) {
    // (above 32 bytes a 128 KB table: one block per SM)
    kern = ivf_scan_table_kernel<M, KP, UC, 256>;
    smem = table_rec_offset<M, KP>() + sizeof(uint4) * ((size_t)a.nprobe + 1);
  } else {
    // the selection's shared state does not depend on the block size
    static_assert(sizeof(typename BlockSelect<512, KP, 4096>::Smem) == sizeof(typename Sel::Smem),
                  "selection state independent of the block size");
    // two resident blocks per SM bound the registers: 128 (256 threads, any U), 85 (384
    // threads, U <= 4), 64 (512 threads, U = 2)
    if (tun.threads == 512 && U == 2) {
      kern = ivf_scan_table_kernel<M, KP, 2, 512>;
      threads = 512;
    } else if (tun.threads == 384 && U <= 4) {
      kern = ivf_scan_table_kernel<M, KP, (U <= 4 ? U : 4), 384>;
      threads = 384;
    } else {
      kern = ivf_scan_table_kernel<M, KP, U, 256>;
    }
    smem = table_rec_offset<M, KP>() + sizeof(uint4) * ((size_t)a.nprobe + 1);
  }
  GBK_TRY(set_smem_limit(kern, smem));
  // persistent mode: blocks_per_sm resident blocks per SM pull queries from the counter
  const int64_t grid =
      a.counter ? std::min<int64_t>(a.nq, (int64_t)tun.blocks_per_sm * device_info().sm_count)
                : a.nq;
  kern<<<(unsigned)grid, threads, smem, st>>>(a);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

template <int M, int KP>
static gbk_status scan_u(const ScanArgs& a, const ScanTuning& tun, cudaStream_t st) {
  switch (tun.codes_per_thread) {
    case 2: return launch_scan<M, KP, 2>(a, tun, st);
    case 4: return launch_scan<M, KP, 4>(a, tun, st);
    case 8: return launch_scan<M, KP, 8>(a, tun, st);
    default: return set_error(GBK_EINVAL, "scan tuning: codes per thread must be 2, 4 or 8");
  }
}

template <int M>
gbk_status scan_k(const ScanArgs& a, const ScanTuning& tun, cudaStream_t st) {
  if (a.k <= 32) return scan_u<M, 32>(a, tun, st);  // a.k = largest k
  if (a.k <= 128) return scan_u<M, 128>(a, tun, st);
  if (a.k <= 256) return scan_u<M, 256>(a, tun, st);
  return scan_u<M, 1024>(a, tun, st);
}

// instantiations: one translation unit per power-of-two code size (ivf_scan_m4.cu ...
// ivf_scan_m64.cu), the other multiples of 4 bytes grouped (ivf_scan_m12_28.cu, ...)
#define GBK_SCAN_SIZE(M) \
  extern template gbk_status scan_k<M>(const ScanArgs&, const ScanTuning&, cudaStream_t);
GBK_SCAN_SIZE(4) GBK_SCAN_SIZE(8) GBK_SCAN_SIZE(12) GBK_SCAN_SIZE(16) GBK_SCAN_SIZE(20)
GBK_SCAN_SIZE(24) GBK_SCAN_SIZE(28) GBK_SCAN_SIZE(32) GBK_SCAN_SIZE(36) GBK_SCAN_SIZE(40)
GBK_SCAN_SIZE(44) GBK_SCAN_SIZE(48) GBK_SCAN_SIZE(52) GBK_SCAN_SIZE(56) GBK_SCAN_SIZE(60)
GBK_SCAN_SIZE(64)
#undef GBK_SCAN_SIZE

}  // namespace gbk
