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
#include "select_core.cuh"

namespace gbk {

// --------------------------------------------------------------------- encoding

// One thread per (vector, sub-quantizer): residual sub-vector (float32), nearest of the 256
// centroids by direct float32 distance (ties to the lowest), byte written to codes.
// Shared memory holds all codebooks as [c][t][m] (broadcast across the M lanes of a vector).
__global__ void __launch_bounds__(256)
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
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * M) return;
  const int64_t v = p / M;
  const int m = (int)(p % M);
  const int64_t L = lists[v];
  float r[32];
#pragma unroll
  for (int t = 0; t < 32; t++)
    r[t] = t < dsub ? x[v * d + m * dsub + t] - coarse[L * d + m * dsub + t] : 0.f;
  float best = __int_as_float(0x7f800000);
  int bc = 0;
  for (int c = 0; c < 256; c++) {
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < 32; t++) {
      if (t < dsub) {
        const float e = r[t] - cb[(c * dsub + t) * M + m];
        s = fmaf(e, e, s);
      }
    }
    if (s < best) {
      best = s;
      bc = c;
    }
  }
  codes[v * M + m] = (uint8_t)bc;
}

// T[L][m][c] = ||C_m[c]||^2 + 2 <c_L^m, C_m[c]>  (block per list, thread per (m, c)).
__global__ void term1_kernel(const float* __restrict__ coarse, const float* __restrict__ pq, int d,
                             int M, float* __restrict__ T) {
  const int L = blockIdx.x;
  const int dsub = d / M;
  for (int e = threadIdx.x; e < M * 256; e += blockDim.x) {
    const int m = e / 256, c = e % 256;
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

// term3[q][m][c] = <x^m, C_m[c]>  (block per query).
__global__ void term3_kernel(const float* __restrict__ xq, const float* __restrict__ pq, int d,
                             int M, float* __restrict__ t3) {
  const int64_t q = blockIdx.x;
  const int dsub = d / M;
  __shared__ float xs[1024];
  for (int t = threadIdx.x; t < d; t += blockDim.x) xs[t] = xq[q * d + t];
  __syncthreads();
  for (int e = threadIdx.x; e < M * 256; e += blockDim.x) {
    const int m = e / 256, c = e % 256;
    const float* C = pq + ((int64_t)m * 256 + c) * dsub;
    float ip = 0.f;
    for (int t = 0; t < dsub; t++) ip = fmaf(xs[m * dsub + t], C[t], ip);
    t3[q * M * 256 + e] = ip;
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
  if constexpr (M == 8) {
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
  const float* T;        // [nlist][M][256] term 1 (precomputed tables)
  const float* t3;       // [nq][M][256] term 3
  const float* xq;       // direct tables: queries
  const float* coarse;   // direct tables: coarse centroids
  const float* pq;       // direct tables: codebooks [M][256][dsub]
  int d;
  int direct;            // 1: LUT[m][c] = ||(x - c_L)^m - C_m[c]||^2 computed in place
  const int64_t* list_off;
  const uint8_t* codes;
  const int64_t* ids;
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
};

// Block per query: for each probed list, build the LUT, stream the codes (one 16-byte code
// per thread), form the distance and keep the k best (block selection, section 4 goal of a
// single pass); ids are looked up only for the winners (section 5.3).
template <int M, int KP>
__global__ void __launch_bounds__(256)
    ivf_scan_kernel(const ScanArgs a) {
  constexpr int THREADS = 256, CAP = 4096;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* lut = reinterpret_cast<float*>(smem_raw);                  // [256][32]
  float* t3s = lut + 256 * 32;                                       // [M][256]
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(t3s + M * 256);
  __shared__ int64_t q_sh;
  const int tid = threadIdx.x, lane = tid & 31;
  const int rot = lane % M, h = lane / M;
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
    for (int p = 0; p < npq; p++) {
      const int64_t L = a.cl_I[q * a.nprobe + p];
      if (L < 0) continue;  // uniform across the block
      const float term2 = a.cl_D[q * a.nprobe + p];
      __syncthreads();  // previous list's look-ups are done
      if (!a.direct) {
        const float* TL = a.T + L * M * 256;
        for (int e = tid; e < M * 256; e += THREADS) {
          const int m = e >> 8, c = e & 255;
          const float v = fmaf(-2.f, t3s[e], __ldg(TL + e));
#pragma unroll
          for (int hh = 0; hh < 32 / M; hh++) lut[c * 32 + hh * M + m] = v;
        }
      } else {
        const int dsub = a.d / M;
        for (int e = tid; e < M * 256; e += THREADS) {
          const int m = e >> 8, c = e & 255;
          const float* C = a.pq + ((int64_t)m * 256 + c) * dsub;
          float v = 0.f;
          for (int t = 0; t < dsub; t++) {
            const float r = a.xq[q * a.d + m * dsub + t] - a.coarse[L * a.d + m * dsub + t];
            const float e2 = r - C[t];
            v = fmaf(e2, e2, v);
          }
#pragma unroll
          for (int hh = 0; hh < 32 / M; hh++) lut[c * 32 + hh * M + m] = v;
        }
      }
      __syncthreads();
      const int64_t o0 = a.list_off[L], o1 = a.list_off[L + 1];
      const float base = a.direct ? 0.f : term2;
      for (int64_t b0 = o0; b0 < o1; b0 += THREADS) {
        const int64_t i = b0 + tid;
        float dist = 0.f;
        bool valid = i < o1;
        if (valid) {
          uint32_t w[M / 4];
          load_code<M>(a.codes, i, w);
          rotate_code<M>(w, rot);
          float acc = 0.f;
#pragma unroll
          for (int st = 0; st < M; st++) {
            const uint32_t c = (w[st >> 2] >> ((st & 3) * 8)) & 255u;
            const int m = (st + rot) & (M - 1);
            acc += lut[c * 32 + h * M + m];
          }
          dist = base + acc;
        }
        const bool pass = valid && f.pass(dist);
        uint64_t cc[1];
        if (pass) cc[0] = composite(ordered_key(dist, false), (uint32_t)i);
        Sel::template push<1>(s, pass ? 1u : 0u, cc);
        __syncthreads();
        if (s.n_buf > CAP - THREADS) {
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
        a.I[ob + j] = a.ids[(uint32_t)e];
      }
    }
  }
}

template <int M, int KP>
static gbk_status launch_scan(const ScanArgs& a, cudaStream_t st) {
  using Sel = BlockSelect<256, KP, 4096>;
  const size_t smem = sizeof(float) * (256 * 32 + M * 256) + sizeof(typename Sel::Smem);
  auto kern = ivf_scan_kernel<M, KP>;
  static bool attr = false;
  if (!attr) {
    GBK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr = true;
  }
  const int64_t grid = a.counter ? std::min<int64_t>(a.nq, 2ll * device_info().sm_count) : a.nq;
  kern<<<(unsigned)grid, 256, smem, st>>>(a);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

template <int M>
static gbk_status scan_k(const ScanArgs& a, cudaStream_t st) {  // a.k = largest k
  if (a.k <= 32) return launch_scan<M, 32>(a, st);
  if (a.k <= 128) return launch_scan<M, 128>(a, st);
  if (a.k <= 256) return launch_scan<M, 256>(a, st);
  return launch_scan<M, 1024>(a, st);
}

gbk_status ivf_scan_run(int M, int64_t nq, int nprobe, int k, const int64_t* cl_I,
                        const float* cl_D, const float* T, const float* t3, const float* xq,
                        const float* coarse, const float* pq, int d, bool direct,
                        const int64_t* list_off, const uint8_t* codes, const int64_t* ids,
                        float* D, int64_t* I, cudaStream_t st, const int32_t* kq,
                        const int32_t* npq, const int64_t* out_off, const int64_t* order,
                        unsigned long long* counter) {
  if (nq == 0) return GBK_OK;
  ScanArgs a{nq, nprobe, k, cl_I, cl_D, T, t3, xq, coarse, pq, d, direct ? 1 : 0, list_off,
             codes, ids, D, I, kq, npq, out_off, order, counter};
  ProfScope prof("ivf_scan", st);
  if (M == 8) return scan_k<8>(a, st);
  if (M == 16) return scan_k<16>(a, st);
  if (M == 32) return scan_k<32>(a, st);
  return set_error(GBK_EUNSUPPORTED, "IVFPQ scan supports M in {8, 16, 32}");
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
  static bool attr = false;
  if (!attr) {
    GBK_CUDA_CHECK(cudaFuncSetAttribute(pq_encode_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)device_info().smem_optin));
    attr = true;
  }
  if (smem > device_info().smem_optin)
    return set_error(GBK_EUNSUPPORTED, "PQ codebooks do not fit in shared memory (d too large)");
  const int64_t pairs = n * M;
  pq_encode_kernel<<<(unsigned)((pairs + 255) / 256), 256, smem, st>>>(x, n, d, M, coarse, lists, pq,
                                                                       codes);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
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
  if (d > 1024) return set_error(GBK_EUNSUPPORTED, "term 3 supports d <= 1024");
  ProfScope prof("term3", st);
  term3_kernel<<<(unsigned)nq, 256, 0, st>>>(xq, pq, d, M, t3);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace gbk
