// IVFADC kernels: product-quantizer encoding, the precomputed term-1 table, term 3, and
// the fused list scan + k-selection (section 5.2 / 5.3, Algorithm 4).
//
// Distance of query x to database vector y in list L (Eq. 11):
//   ||x - q(y)||^2 = sum_m T[L][m][code_m]  +  ||x - c_L||^2  -  2 sum_m <x^m, C_m[code_m]>
// with T[L][m][c] = ||C_m[c]||^2 + 2 <c_L^m, C_m[c]> (term 1, query independent), term 2
// the coarse distance, term 3 computed once per query.  Term 1 depends on the stored vector
// only, so its sum over the code, s1[j] = sum_m T[L][m][code_jm], is formed once per vector
// when the lists are built; the scan then adds, per code, M look-ups into the query's
// term-3 table Q_x[m][c] = -2 <x^m, C_m[c]>, which is built once per query (not once per
// (query, list) as the tables of section 5.3 are).  Without precomputed tables (the direct
// mode) the scan builds LUT[m][c] = ||(x - c_L)^m - C_m[c]||^2 per (query, list).
//
// Bank-conflict-free look-ups: the 32 lanes of a warp look up 32 different codes at once.
// Stored codes are rotated per list position: the code at position r of its list holds
// sub-quantizer (s + (r mod 32)) mod M in byte s.  A warp scans 32 consecutive positions of
// one list, so lane l (= r mod 32) reads sub-table (s + l) mod M at step s, and the tables
// are laid out so that those 32 reads fall in 32 different banks whatever the codes are.
#include <algorithm>

#include "common.cuh"
#include "ivf.cuh"
#include "ivf_scan_kernels.cuh"
#include "knn.cuh"
#include "select_core.cuh"

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

gbk_status ivf_scan_run(int M, int64_t nq, int nprobe, int k, const int64_t* cl_I,
                        const float* cl_D, const float* s1, const float* t3, const float* xq,
                        const float* coarse, const float* pq, int d, bool direct,
                        const int64_t* list_off, const uint8_t* codes, const int64_t* ids,
                        float* D, int64_t* I, cudaStream_t st, const int32_t* kq,
                        const int32_t* npq, const int64_t* out_off, const int64_t* order,
                        unsigned long long* counter, ScanTuning tun) {
  if (nq == 0) return GBK_OK;
  if (tun.blocks_per_sm < 1 || tun.blocks_per_sm > 8)
    return set_error(GBK_EINVAL, "scan tuning: blocks per SM must be in [1, 8]");
  ScanArgs a{nq,     nprobe, k,     cl_I, cl_D, s1,      t3,   xq,      coarse, pq, d,
             direct ? 1 : 0, list_off, codes, ids, D, I, kq, npq, out_off, order, counter};
  ProfScope prof("ivf_scan", st);
  switch (M) {
    case 4: return scan_k<4>(a, tun, st);
    case 8: return scan_k<8>(a, tun, st);
    case 12: return scan_k<12>(a, tun, st);
    case 16: return scan_k<16>(a, tun, st);
    case 20: return scan_k<20>(a, tun, st);
    case 24: return scan_k<24>(a, tun, st);
    case 28: return scan_k<28>(a, tun, st);
    case 32: return scan_k<32>(a, tun, st);
    case 36: return scan_k<36>(a, tun, st);
    case 40: return scan_k<40>(a, tun, st);
    case 44: return scan_k<44>(a, tun, st);
    case 48: return scan_k<48>(a, tun, st);
    case 52: return scan_k<52>(a, tun, st);
    case 56: return scan_k<56>(a, tun, st);
    case 60: return scan_k<60>(a, tun, st);
    case 64: return scan_k<64>(a, tun, st);
    default: return set_error(GBK_EUNSUPPORTED, "IVFPQ scan supports M a multiple of 4 up to 64");
  }
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
