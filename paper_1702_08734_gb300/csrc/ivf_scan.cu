// IVFADC kernels: product-quantizer encoding, the precomputed term-1 table, term 3, and
// the fused list scan + k-selection (section 5.2 / 5.3, Algorithm 4).
//
// Distance of query x to database vector y in list L (Eq. 11):
//   ||x - q(y)||^2 = sum_m T[L][m][code_m]  +  ||x - c_L||^2  -  2 sum_m <x^m, C_m[code_m]>
// with T[L][m][c] = ||C_m[c]||^2 + 2 <c_L^m, C_m[c]> (term 1, query independent), term 2
// the coarse distance, term 3 computed once per query.  The scan builds, per (query, list),
// LUT[m][c] = T[L][m][c] - 2 term3[m][c] in shared memory and sums b look-ups per code.
//
// Shared-memory LUT layout: entry (c, m) is stored at c*32 + h*M + m for every copy
// h < 32/M, and lane l of a warp reads sub-table m = (s + l) mod M at step s from copy
// h = l / M.  The 32 lanes of a warp then always hit 32 distinct banks (conflict-free),
// instead of the ~3.5-way conflicts of random look-ups into LUT[m][c].  Each lane rotates
// its 16-byte code by (l mod M) bytes once so that step s reads byte s.
#include <algorithm>

#include "common.cuh"
#include "ivf.cuh"
#include "knn.cuh"
#include "select_core.cuh"
#include "sm100.cuh"

namespace gbk {

// --------------------------------------------------------------------- encoding

// Residual sub-vector (float32) of each (vector, sub-quantizer) and the nearest of its 256
// centroids by direct float32 distance, summed over the dsub coordinates in order (ties to
// the lowest), written to codes.  Persistent blocks hold all codebooks in shared memory as
// [c][t][m] (consecutive lanes = consecutive sub-quantizers: conflict-free) and loop over
// the vectors; each thread serves V vectors of one sub-quantizer, so every codebook read
// feeds V distance updates.
template <int DS, int V>
__global__ void __launch_bounds__(512)
    pq_encode_kernel(const float* __restrict__ x, int64_t n, int d, int M,
                     const float* __restrict__ coarse, const int32_t* __restrict__ lists,
                     const float* __restrict__ pq, uint8_t* __restrict__ codes) {
  extern __shared__ float cb[];  // [256][dsub][M]
  const int dsub = d / M;
  for (int i = threadIdx.x; i < 256 * d; i += blockDim.x) {
    const int m = i / (256 * dsub), rem = i % (256 * dsub), c = rem / dsub, t = rem % dsub;
    cb[(c * dsub + t) * M + m] = pq[i];
  }
  __syncthreads();
  const int G = (int)blockDim.x / M;  // vector groups per block
  const int m = (int)threadIdx.x % M, g = (int)threadIdx.x / M;
  if (g >= G) return;
  for (int64_t v0 = ((int64_t)blockIdx.x * G + g) * V; v0 < n; v0 += (int64_t)gridDim.x * G * V) {
    float r[V][DS];
#pragma unroll
    for (int vv = 0; vv < V; vv++) {
      const int64_t v = v0 + vv;
      const int64_t L = v < n ? lists[v] : 0;
#pragma unroll
      for (int t = 0; t < DS; t++)
        r[vv][t] = (v < n && t < dsub) ? x[v * d + m * dsub + t] - coarse[L * d + m * dsub + t]
                                       : 0.f;
    }
    float best[V];
    int bc[V];
#pragma unroll
    for (int vv = 0; vv < V; vv++) {
      best[vv] = __int_as_float(0x7f800000);
      bc[vv] = 0;
    }
    for (int c = 0; c < 256; c++) {
      float sum[V];
#pragma unroll
      for (int vv = 0; vv < V; vv++) sum[vv] = 0.f;
#pragma unroll
      for (int t = 0; t < DS; t++) {
        if (t < dsub) {
          const float cv = cb[(c * dsub + t) * M + m];
#pragma unroll
          for (int vv = 0; vv < V; vv++) {
            const float e = r[vv][t] - cv;
            sum[vv] = fmaf(e, e, sum[vv]);
          }
        }
      }
#pragma unroll
      for (int vv = 0; vv < V; vv++)
        if (sum[vv] < best[vv]) {
          best[vv] = sum[vv];
          bc[vv] = c;
        }
    }
#pragma unroll
    for (int vv = 0; vv < V; vv++)
      if (v0 + vv < n) codes[(v0 + vv) * M + m] = (uint8_t)bc[vv];
  }
}

// T[L][c][m] = ||C_m[c]||^2 + 2 <c_L^m, C_m[c]>  (block per list, thread per (c, m)); the
// c-major layout makes one list's table a contiguous block whose rows the scan reads whole.
__global__ void term1_kernel(const float* __restrict__ coarse, const float* __restrict__ pq, int d,
                             int M, float* __restrict__ T) {
  const int L = blockIdx.x;
  const int dsub = d / M;
  for (int e = threadIdx.x; e < M * 256; e += blockDim.x) {  // e = c * M + m
    const int m = e % M, c = e / M;
    const float* C = pq + ((int64_t)m * 256 + c) * dsub;
    const float* cl = coarse + (int64_t)L * d + m * dsub;
    float nn = 0.f, ip = 0.f;
    for (int t = 0; t < dsub; t++) {
      nn = fmaf(C[t], C[t], nn);
      ip = fmaf(cl[t], C[t], ip);
    }
    T[(int64_t)L * M * 256 + e] = fmaf(2.f, ip, nn);
  }
}

// term3[q][c][m] = <x^m, C_m[c]> (Eq. 11's third term) is one GEMM: against the
// block-diagonal codebook matrix E [256 M][d] whose row c M + m holds C_m[c] in the
// columns of sub-vector m (zeros elsewhere), x E^T is exactly term3 in its [c][m] layout.
// The zeros cost M times the useful multiply-adds, which the tensor cores absorb.
__global__ void expand_codebooks_kernel(const float* __restrict__ pq, int d, int M,
                                        float* __restrict__ E) {
  const int dsub = d / M;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)256 * M * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / d), t = (int)(e % d);
    const int c = row / M, m = row % M;
    E[e] = (t / dsub == m) ? pq[((int64_t)m * 256 + c) * dsub + (t % dsub)] : 0.f;
  }
}

// --------------------------------------------------------------------- scan

template <int M>
struct CodeWords {
  static constexpr int NW = M / 4;
};

// Rotate the M-byte code right by `rot` bytes (byte s of the result = byte (s+rot) mod M).
template <int M>
__device__ __forceinline__ void rotate_code(uint32_t (&w)[M / 4], int rot) {
  constexpr int NW = M / 4;
  const int q = rot >> 2, r8 = (rot & 3) * 8;
  uint32_t t[NW];
#pragma unroll
  for (int b = 1; b < NW; b <<= 1) {
    if (q & b) {
#pragma unroll
      for (int j = 0; j < NW; j++) t[j] = w[(j + b) % NW];
#pragma unroll
      for (int j = 0; j < NW; j++) w[j] = t[j];
    }
  }
#pragma unroll
  for (int j = 0; j < NW; j++) t[j] = __funnelshift_r(w[j], w[(j + 1) % NW], r8);
#pragma unroll
  for (int j = 0; j < NW; j++) w[j] = t[j];
}

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
  } else {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(codes) + 2 * i);
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(codes) + 2 * i + 1);
    w[0] = a.x;
    w[1] = a.y;
    w[2] = a.z;
    w[3] = a.w;
    w[4] = b.x;
    w[5] = b.y;
    w[6] = b.z;
    w[7] = b.w;
  }
}

struct ScanArgs {
  int64_t nq;
  int nprobe, k;
  const int64_t* cl_I;   // [nq][nprobe] probed lists, nearest first (-1 = none)
  const float* cl_D;     // [nq][nprobe] term 2 = ||x - c_L||^2
  const float* T;        // [nlist][256][M] term 1 (precomputed tables)
  const float* t3;       // [nq][256][M] term 3
  const float* xq;       // direct tables: queries
  const float* coarse;   // direct tables: coarse centroids
  const float* pq;       // direct tables: codebooks [M][256][dsub]
  int d;
  int direct;            // 1: LUT[m][c] = ||(x - c_L)^m - C_m[c]||^2 computed in place
  const int64_t* list_off;
  const uint8_t* codes;
  const int64_t* ids;    // null: list positions out instead of ids
  float* D;
  int64_t* I;
  // mixed batches (all optional): per-query k and nprobe (<= k, nprobe above), output
  // offsets (results of query q at D/I + out_off[q]); persistent mode takes queries from
  // `order` (longest first) through the atomic `counter`.
  const int32_t* kq;
  const int32_t* npq;
  const int64_t* out_off;
  const int64_t* order;
  unsigned long long* counter;
  uint32_t* status;      // device status word (bounded waits record a timeout here)
};

// Block per query: for each probed list, build the LUT, stream the codes (U 16-byte codes
// per thread per step), form the distance and keep the k best (block selection, section 4
// goal of a single pass); ids are looked up only for the winners (section 5.3).
template <int M, int KP, int U>
__global__ void __launch_bounds__(256)
    ivf_scan_kernel(const ScanArgs a) {
  constexpr int THREADS = 256, CAP = 4096;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* lut = reinterpret_cast<float*>(smem_raw);                  // [256][32]
  float* t3s = lut + 256 * 32;                                       // [256][M]
  float* tst = t3s + M * 256;                                        // [256][M] term 1 of a list
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(tst + M * 256);
  __shared__ int64_t q_sh;
  __shared__ uint64_t t_bar;  // completion of the term-1 bulk copy
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rot = lane % M, h = lane / M;
  constexpr uint32_t TBYTES = M * 256 * sizeof(float);
  uint32_t t_phase = 0;
  if (tid == 0) {
    sm100::mbar_init(&t_bar, 1);
    abort_flag = 0;
    sm100::fence_mbar_init();
  }
  __syncthreads();
  // one thread starts the copy of list L's term-1 table into tst
  auto copy_T = [&](int64_t L) {
    if (tid == 0) {
      sm100::fence_proxy_async_smem();
      sm100::mbar_arrive_expect_tx(&t_bar, TBYTES);
      sm100::bulk_load(tst, a.T + L * M * 256, TBYTES, &t_bar);
    }
  };
  for (int64_t it = blockIdx.x;; it += gridDim.x) {
    // next query: static (one block per query) or from the persistent work queue
    if (a.counter) {
      __syncthreads();
      if (tid == 0) {
        const unsigned long long w = atomicAdd(a.counter, 1ull);
        q_sh = w < (unsigned long long)a.nq ? a.order[w] : -1;
      }
      __syncthreads();
    }
    const int64_t q = a.counter ? q_sh : (it < a.nq ? it : -1);
    if (q < 0) break;
    const int kq = a.kq ? a.kq[q] : a.k;
    const int npq = a.npq ? min(a.npq[q], a.nprobe) : a.nprobe;
    const int64_t ob = a.out_off ? a.out_off[q] : q * (int64_t)a.k;
    __syncthreads();
    if (!a.direct)
      for (int e = tid; e < M * 256; e += THREADS) t3s[e] = a.t3[q * M * 256 + e];
    Sel::init(s);
    __syncthreads();
    ValueFilter f;
    f.set(NAN_KEY, false);
    // Software pipeline across the probed lists: the term-1 table of list p+1 is copied
    // into shared memory (bulk copy) and the first codes of each list are loaded into
    // registers while earlier work proceeds, so no global-memory latency is exposed once
    // per list.
    int64_t Lc = -1, o0c = 0, o1c = 0;  // current list
    auto fetch_list = [&](int p, int64_t& L, int64_t& o0, int64_t& o1) {
      L = p < npq ? a.cl_I[q * a.nprobe + p] : -1;
      if (L >= 0) {
        o0 = a.list_off[L];
        o1 = a.list_off[L + 1];
      } else {
        o0 = o1 = 0;
      }
    };
    constexpr int STEP = THREADS * U;
    uint32_t wn[U][M / 4];               // codes of the next step, in flight
    auto fetch_codes = [&](int64_t b0, int64_t o1) {
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int64_t i = b0 + u * THREADS + tid;
        if (i < o1) load_code<M>(a.codes, i, wn[u]);
      }
    };
    fetch_list(0, Lc, o0c, o1c);
    if (Lc >= 0 && !a.direct) copy_T(Lc);
    bool ok = true;
    for (int p = 0; p < npq && ok; p++) {
      const int64_t L = Lc, o0 = o0c, o1 = o1c;
      if (L >= 0) fetch_codes(o0, o1);
      __syncthreads();  // previous list's look-ups are done
      if (L >= 0) {
        // LUT[c][h*M + m] = T[L][c][m] - 2 term3[c][m]: warp w fills rows c of its 32; lane l
        // writes word c*32 + l (copy h = l / M of sub-table m = l % M): conflict-free.
        if (!a.direct) {
          ok = sm100::mbar_wait(&t_bar, t_phase, a.status, (volatile int*)&abort_flag);
          t_phase ^= 1u;
          if (ok) {
#pragma unroll 4
            for (int i = 0; i < 32; i++) {
              const int c = warp * 32 + i;
              const int e = c * M + rot;
              lut[c * 32 + lane] = fmaf(-2.f, t3s[e], tst[e]);
            }
          }
        } else {
          const int dsub = a.d / M;
          for (int i = 0; i < 32; i++) {
            const int c = warp * 32 + i, m = rot;
            const float* C = a.pq + ((int64_t)m * 256 + c) * dsub;
            float v = 0.f;
            for (int t = 0; t < dsub; t++) {
              const float r = a.xq[q * a.d + m * dsub + t] - a.coarse[L * a.d + m * dsub + t];
              const float e2 = r - C[t];
              v = fmaf(e2, e2, v);
            }
            lut[c * 32 + lane] = v;
          }
        }
      }
      const float term2 = L >= 0 ? a.cl_D[q * a.nprobe + p] : 0.f;
      fetch_list(p + 1, Lc, o0c, o1c);  // next list's extent
      __syncthreads();                   // LUT complete, tst consumed
      if (Lc >= 0 && !a.direct && ok) copy_T(Lc);
      if (L < 0 || !ok) continue;        // uniform across the block
      const float base = a.direct ? 0.f : term2;
      for (int64_t b0 = o0; b0 < o1; b0 += STEP) {
        uint32_t w[U][M / 4];
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
          for (int j = 0; j < M / 4; j++) w[u][j] = wn[u][j];
        if (b0 + STEP < o1) fetch_codes(b0 + STEP, o1);
        uint32_t mask = 0;
        uint64_t cc[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int64_t i = b0 + u * THREADS + tid;
          cc[u] = ~0ull;
          if (i < o1) {
            rotate_code<M>(w[u], rot);
            float acc = 0.f;
#pragma unroll
            for (int st = 0; st < M; st++) {
              const uint32_t c = (w[u][st >> 2] >> ((st & 3) * 8)) & 255u;
              const int m = (st + rot) & (M - 1);
              acc += lut[c * 32 + h * M + m];
            }
            const float dist = base + acc;
            if (f.pass(dist)) {
              mask |= 1u << u;
              cc[u] = composite(ordered_key(dist, false), (uint32_t)i);
            }
          }
        }
        Sel::template push<U>(s, mask, cc);
        __syncthreads();
        if (s.n_buf > CAP - STEP) {
          Sel::compact(s, kq);
          f.set((uint32_t)(s.thr >> 32), false);
        }
      }
    }
    Sel::finish(s, kq);
    for (int j = tid; j < kq; j += THREADS) {
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
}

template <int M, int KP, int U>
static gbk_status launch_scan(const ScanArgs& a, const ScanTuning& tun, cudaStream_t st) {
  using Sel = BlockSelect<256, KP, 4096>;
  const size_t smem = sizeof(float) * (256 * 32 + 2 * M * 256) + sizeof(typename Sel::Smem);
  auto kern = ivf_scan_kernel<M, KP, U>;
  static bool attr = false;
  if (!attr) {
    GBK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr = true;
  }
  // persistent mode: blocks_per_sm resident blocks per SM pull queries from the counter
  const int64_t grid =
      a.counter ? std::min<int64_t>(a.nq, (int64_t)tun.blocks_per_sm * device_info().sm_count)
                : a.nq;
  kern<<<(unsigned)grid, 256, smem, st>>>(a);
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
static gbk_status scan_k(const ScanArgs& a, const ScanTuning& tun, cudaStream_t st) {
  if (a.k <= 32) return scan_u<M, 32>(a, tun, st);  // a.k = largest k
  if (a.k <= 128) return scan_u<M, 128>(a, tun, st);
  if (a.k <= 256) return scan_u<M, 256>(a, tun, st);
  return scan_u<M, 1024>(a, tun, st);
}

gbk_status ivf_scan_run(int M, int64_t nq, int nprobe, int k, const int64_t* cl_I,
                        const float* cl_D, const float* T, const float* t3, const float* xq,
                        const float* coarse, const float* pq, int d, bool direct,
                        const int64_t* list_off, const uint8_t* codes, const int64_t* ids,
                        float* D, int64_t* I, cudaStream_t st, const int32_t* kq,
                        const int32_t* npq, const int64_t* out_off, const int64_t* order,
                        unsigned long long* counter, ScanTuning tun) {
  if (nq == 0) return GBK_OK;
  if (tun.blocks_per_sm < 1 || tun.blocks_per_sm > 8)
    return set_error(GBK_EINVAL, "scan tuning: blocks per SM must be in [1, 8]");
  ScanArgs a{nq, nprobe, k, cl_I, cl_D, T, t3, xq, coarse, pq, d, direct ? 1 : 0, list_off,
             codes, ids, D, I, kq, npq, out_off, order, counter, device_status()};
  if (!a.status) return set_error(GBK_ECUDA, "device status word unavailable");
  ProfScope prof("ivf_scan", st);
  if (M == 4) return scan_k<4>(a, tun, st);
  if (M == 8) return scan_k<8>(a, tun, st);
  if (M == 16) return scan_k<16>(a, tun, st);
  if (M == 32) return scan_k<32>(a, tun, st);
  return set_error(GBK_EUNSUPPORTED, "IVFPQ scan supports M in {4, 8, 16, 32}");
}

// Work of each query (codes scanned) for longest-first scheduling: key = 31 - log2(work)
// so that a stable bucketing by key lists the heaviest queries first.
__global__ void scan_cost_kernel(const int64_t* __restrict__ cl_I, int64_t nq, int nprobe,
                                 const int32_t* __restrict__ npq, const int64_t* __restrict__ off,
                                 int32_t* __restrict__ key) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int np = npq ? min(npq[q], nprobe) : nprobe;
  long long w = 1;
  for (int p = 0; p < np; p++) {
    const int64_t L = cl_I[q * nprobe + p];
    if (L >= 0) w += off[L + 1] - off[L] + 64;
  }
  key[q] = 63 - __clzll(w) > 31 ? 0 : 31 - (63 - __clzll(w));
}

gbk_status scan_cost_run(const int64_t* cl_I, int64_t nq, int nprobe, const int32_t* npq,
                         const int64_t* off, int32_t* key, cudaStream_t st) {
  scan_cost_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(cl_I, nq, nprobe, npq, off, key);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status pq_encode_run(const float* x, int64_t n, int d, int M, const float* coarse,
                         const int32_t* lists, const float* pq, uint8_t* codes, cudaStream_t st) {
  if (n == 0) return GBK_OK;
  if (d / M > 32) return set_error(GBK_EUNSUPPORTED, "PQ sub-vectors longer than 32");
  ProfScope prof("pq_encode", st);
  const size_t smem = sizeof(float) * 256 * (size_t)d;
  const DeviceInfo& di = device_info();
  if (smem > di.smem_optin)
    return set_error(GBK_EUNSUPPORTED, "PQ codebooks do not fit in shared memory (d too large)");
  const int dsub = d / M;
  const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, di.smem_optin / smem));
  const unsigned grid = (unsigned)(di.sm_count * per_sm);
  auto go = [&](auto kern) -> gbk_status {
    GBK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)di.smem_optin));
    kern<<<grid, 512, smem, st>>>(x, n, d, M, coarse, lists, pq, codes);
    GBK_LAUNCH_CHECK();
    return GBK_OK;
  };
  if (dsub <= 8) return go(pq_encode_kernel<8, 4>);
  if (dsub <= 16) return go(pq_encode_kernel<16, 2>);
  return go(pq_encode_kernel<32, 1>);
}

gbk_status term1_run(const float* coarse, const float* pq, int nlist, int d, int M, float* T,
                     cudaStream_t st) {
  ProfScope prof("term1_table", st);
  term1_kernel<<<nlist, 256, 0, st>>>(coarse, pq, d, M, T);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status term3_run(const float* xq, int64_t nq, const float* pq, int d, int M, float* t3,
                     cudaStream_t st) {
  if (nq == 0) return GBK_OK;
  ProfScope prof("term3", st);
  gbk_status r;
  const int64_t ne = (int64_t)256 * M;
  Scratch E;
  if ((r = E.alloc(sizeof(float) * (size_t)ne * d, st)) != GBK_OK) return r;
  expand_codebooks_kernel<<<(unsigned)std::min<int64_t>((ne * d + 255) / 256, 4096), 256, 0, st>>>(
      pq, d, M, E.as<float>());
  GBK_LAUNCH_CHECK();
  PreparedOperand Q, B;
  if ((r = prepare_operand(xq, nq, d, GBK_PREC_FP32, nq, 0.f, &Q, st)) != GBK_OK) return r;
  if ((r = prepare_operand(E.as<float>(), ne, d, GBK_PREC_FP32, (ne + 127) / 128 * 128, 0.f, &B,
                           st)) != GBK_OK)
    return r;
  return pairwise_run(Q, B, true, t3, ne, st);
}

}  // namespace gbk
