// Host driver of the fused distance GEMM: operand preparation, work planning, TMA
// descriptors, the cross-chunk merge (the paper's two-pass k-selection, section 5.3)
// and the large-k path that tiles the distance matrix over queries (section 5.1).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "dist_gemm.cuh"
#include "dist_gemm_launch.cuh"
#include "dist_gemm_kernel.cuh"
#include "ivf.cuh"
#include "kselect.cuh"
#include "knn.cuh"

namespace gbk {

// ------------------------------------------------------------------ prep kernels

__global__ void prep_tf32x3_kernel(const float* __restrict__ x, int64_t n, int d, int dpad,
                                   float* __restrict__ hi, float* __restrict__ lo,
                                   float* __restrict__ norms, int64_t nrows_pad,
                                   float pad_norm) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= nrows_pad) return;
  if (row >= n) {
    if (lane == 0) norms[row] = pad_norm;
    return;
  }
  float s = 0.f;
  for (int t = lane; t < dpad; t += 32) {
    const float v = t < d ? x[row * d + t] : 0.f;
    const float h = tf32_rna(v);
    const float l = tf32_rna(v - h);
    hi[row * dpad + t] = h;
    lo[row * dpad + t] = l;
    s = fmaf(v, v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
  if (lane == 0) norms[row] = s;
}

__global__ void prep_bf16_kernel(const float* __restrict__ x, int64_t n, int d, int dpad,
                                 __nv_bfloat16* __restrict__ out, float* __restrict__ norms,
                                 int64_t nrows_pad, float pad_norm) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= nrows_pad) return;
  if (row >= n) {
    if (lane == 0) norms[row] = pad_norm;
    return;
  }
  float s = 0.f;
  for (int t = lane; t < dpad; t += 32) {
    const float v = t < d ? x[row * d + t] : 0.f;
    out[row * dpad + t] = __float2bfloat16_rn(v);
    s = fmaf(v, v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
  if (lane == 0) norms[row] = s;
}

// Rows per warp of prep_fp16x3_kernel: both rows' loads are issued before either is used,
// doubling the bytes in flight per SM (one row per warp reached 63% of HBM at d = 128).
constexpr int PREP16_ROWS = 2;

__global__ void prep_fp16x3_kernel(const float* __restrict__ x, int64_t n, int d, int dpad,
                                   __half* __restrict__ hi, __half* __restrict__ lo,
                                   float* __restrict__ scale, float* __restrict__ norms,
                                   int64_t nrows_pad, float pad_norm) {
  const int lane = threadIdx.x & 31;
  const int64_t row0 =
      ((int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * PREP16_ROWS;
  constexpr int MAXE = 8;  // elements per lane kept in registers (dpad <= 256)
  const bool in_regs = dpad <= 32 * MAXE;
  float v[PREP16_ROWS][MAXE];
  if (in_regs) {
#pragma unroll
    for (int r = 0; r < PREP16_ROWS; r++) {
      const int64_t row = row0 + r;
#pragma unroll
      for (int i = 0; i < MAXE; i++) {
        const int t = lane + 32 * i;
        v[r][i] = (row < n && t < d) ? x[row * d + t] : 0.f;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < PREP16_ROWS; r++) {
    const int64_t row = row0 + r;
    if (row >= nrows_pad) return;
    if (row >= n) {
      if (lane == 0) {
        norms[row] = pad_norm;
        scale[row] = 0.f;
      }
      continue;
    }
    // sum of squares in element order per lane, then across lanes (the same order for
    // every row length)
    float s = 0.f, amax = 0.f;
    if (in_regs) {
#pragma unroll
      for (int i = 0; i < MAXE; i++) {
        if (lane + 32 * i < dpad) {
          s = fmaf(v[r][i], v[r][i], s);
          amax = fmaxf(amax, fabsf(v[r][i]));
        }
      }
    } else {
      for (int t = lane; t < dpad; t += 32) {
        const float u = t < d ? x[row * d + t] : 0.f;
        s = fmaf(u, u, s);
        amax = fmaxf(amax, fabsf(u));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(FULL_MASK, s, o);
      amax = fmaxf(amax, __shfl_xor_sync(FULL_MASK, amax, o));
    }
    // s = 2^e with amax / s in [0.5, 1): the scaled row is exact and within FP16's range
    int e = 0;
    if (amax > 0.f) frexpf(amax, &e);
    if (in_regs) {
#pragma unroll
      for (int i = 0; i < MAXE; i++) {
        const int t = lane + 32 * i;
        if (t < dpad) {
          const float u = ldexpf(v[r][i], -e);
          const __half h = __float2half_rn(u);
          hi[row * dpad + t] = h;
          lo[row * dpad + t] = __float2half_rn(u - __half2float(h));
        }
      }
    } else {
      for (int t = lane; t < dpad; t += 32) {
        const float u = t < d ? ldexpf(x[row * d + t], -e) : 0.f;
        const __half h = __float2half_rn(u);
        hi[row * dpad + t] = h;
        lo[row * dpad + t] = __float2half_rn(u - __half2float(h));
      }
    }
    if (lane == 0) {
      norms[row] = s;
      scale[row] = ldexpf(1.f, e);
    }
  }
}

__global__ void prep_fp8_kernel(const float* __restrict__ x, int64_t n, int d, int dpad,
                                __nv_fp8_e4m3* __restrict__ out, float* __restrict__ scale,
                                float* __restrict__ norms, int64_t nrows_pad, float pad_norm) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= nrows_pad) return;
  if (row >= n) {
    if (lane == 0) {
      norms[row] = pad_norm;
      scale[row] = 0.f;
    }
    return;
  }
  float s = 0.f, amax = 0.f;
  for (int t = lane; t < d; t += 32) {
    const float v = x[row * d + t];
    s = fmaf(v, v, s);
    amax = fmaxf(amax, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(FULL_MASK, s, o);
    amax = fmaxf(amax, __shfl_xor_sync(FULL_MASK, amax, o));
  }
  const float sc = amax > 0.f ? amax / 448.f : 1.f;
  const float inv = 1.f / sc;
  for (int t = lane; t < dpad; t += 32) {
    const float v = t < d ? x[row * d + t] * inv : 0.f;
    out[row * dpad + t] = __nv_fp8_e4m3(v);
  }
  if (lane == 0) {
    norms[row] = s;
    scale[row] = sc;
  }
}

namespace {

// ------------------------------------------------------------------ cross-chunk merge

// D[q][j] <- max(0, D[q][j] + ||x_q||^2): the query norm added to selected L2 values.
__global__ void add_norm_clamp_kernel(float* __restrict__ D, int64_t nq, int k,
                                      const float* __restrict__ xnorm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nq * k) D[i] = fmaxf(D[i] + xnorm[i / k], 0.f);
}

template <int KP>
__global__ void __launch_bounds__(256)
    knn_merge_kernel(const uint64_t* __restrict__ part, int chunks, int kp, int k,
                     const float* __restrict__ xnorm, int largest, float* __restrict__ D,
                     int64_t* __restrict__ I) {
  constexpr int THREADS = 256, CAP = 4096;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(smem_raw);
  const int64_t q = blockIdx.x;
  const uint64_t* src = part + q * (int64_t)chunks * kp;
  Sel::init(s);
  uint64_t thr = ~0ull;
  if (KP <= 32) {
    __syncthreads();
    const int64_t nper = (int64_t)chunks * k;
    for (int64_t base = 0; base < nper; base += THREADS) {
      const int64_t i = base + threadIdx.x;
      uint64_t c[1];
      uint32_t mask = 0;
      if (i < nper) {
        const int64_t ch = i / k, j = i % k;
        c[0] = src[ch * kp + j];
        mask = (c[0] != ~0ull && c[0] <= thr) ? 1u : 0u;
      }
      Sel::template push<1>(s, mask, c);
      __syncthreads();
      if (s.n_buf > CAP - THREADS) {
        Sel::compact(s, k);
        thr = s.thr;
      }
    }
  } else {
    // Longer lists: rounds of 32 entries of every list still alive, one list per warp
    // per step (coalesced 256-byte reads).  The first k candidates in give the threshold
    // (an early compaction), and since each list is sorted, a list whose last entry of a
    // round misses the threshold has no later entry that passes: it is not read again.
    constexpr int NW = THREADS / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* alive = smem_raw + sizeof(typename Sel::Smem);
    for (int l = threadIdx.x; l < chunks; l += THREADS) alive[l] = 1;
    __syncthreads();
    for (int r = 0; r * 32 < k; r++) {
      for (int l0 = 0; l0 < chunks; l0 += NW) {
        const int l = l0 + warp;
        uint64_t c[1] = {~0ull};
        uint32_t mask = 0;
        if (l < chunks && alive[l]) {  // warp-uniform
          const int j = r * 32 + lane;
          if (j < k) c[0] = src[(int64_t)l * kp + j];
          mask = (c[0] != ~0ull && c[0] <= thr) ? 1u : 0u;
          const uint64_t last = __shfl_sync(FULL_MASK, c[0], 31);
          if (lane == 0 && (last == ~0ull || last > thr)) alive[l] = 0;
        }
        Sel::template push<1>(s, mask, c);
        __syncthreads();
        if (s.n_buf > CAP - THREADS || (s.n_top < k && s.n_top + s.n_buf >= k)) {
          Sel::compact(s, k);
          thr = s.thr;
        }
      }
    }
  }
  Sel::finish(s, k);
  const float xn = xnorm ? xnorm[q] : 0.f;
  for (int j = threadIdx.x; j < k; j += THREADS) {
    const uint64_t e = s.top[j];
    float dv;
    int64_t id;
    if (e == ~0ull) {
      dv = largest ? -INFINITY : INFINITY;
      id = -1;
    } else {
      dv = key_value((uint32_t)(e >> 32), largest != 0);
      if (!largest) dv = fmaxf(dv + xn, 0.f);
      id = (int64_t)(uint32_t)e;
    }
    D[q * k + j] = dv;
    I[q * k + j] = id;
  }
}

template <int KP>
gbk_status launch_knn_merge(const uint64_t* part, int64_t nq, int chunks, int kp, int k,
                            const float* xnorm, int largest, float* D, int64_t* I,
                            cudaStream_t st) {
  using Sel = BlockSelect<256, KP, 4096>;
  auto kern = knn_merge_kernel<KP>;
  const size_t smem = sizeof(typename Sel::Smem) + (KP > 32 ? (size_t)chunks : 0);  // + alive
  GBK_TRY(set_smem_limit(kern, smem));
  kern<<<(unsigned)nq, 256, smem, st>>>(part, chunks, kp, k, xnorm, largest, D, I);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

// k = 1: a thread per query takes the least composite over its chunks.
__global__ void knn_merge_k1_kernel(const uint64_t* __restrict__ part, int64_t nq, int chunks,
                                    int kp, const float* __restrict__ xnorm, int largest,
                                    float* __restrict__ D, int64_t* __restrict__ I) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  uint64_t best = ~0ull;
  for (int c = 0; c < chunks; c++) best = min(best, part[(q * chunks + c) * kp]);
  if (best == ~0ull) {
    D[q] = largest ? -INFINITY : INFINITY;
    I[q] = -1;
  } else {
    float dv = key_value((uint32_t)(best >> 32), largest != 0);
    if (!largest) dv = fmaxf(dv + xnorm[q], 0.f);
    D[q] = dv;
    I[q] = (int64_t)(uint32_t)best;
  }
}

gbk_status knn_merge(const uint64_t* part, int64_t nq, int chunks, int kp, int k,
                     const float* xnorm, int largest, float* D, int64_t* I, cudaStream_t st) {
  ProfScope prof("knn_merge", st);
  if (k == 1) {
    knn_merge_k1_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(part, nq, chunks, kp, xnorm,
                                                                      largest, D, I);
    GBK_LAUNCH_CHECK();
    return GBK_OK;
  }
  if (k <= 32) return launch_knn_merge<32>(part, nq, chunks, kp, k, xnorm, largest, D, I, st);
  if (k <= 64) return launch_knn_merge<64>(part, nq, chunks, kp, k, xnorm, largest, D, I, st);
  if (k <= 128) return launch_knn_merge<128>(part, nq, chunks, kp, k, xnorm, largest, D, I, st);
  if (k <= 256) return launch_knn_merge<256>(part, nq, chunks, kp, k, xnorm, largest, D, I, st);
  return launch_knn_merge<512>(part, nq, chunks, kp, k, xnorm, largest, D, I, st);
}

// ------------------------------------------------------------------ shard merge

// Top k of nparts sorted partial results per query (section 5.4: the extra k-selection
// after sharding).  Entries with a negative id are padding and skipped.
template <int KP>
__global__ void __launch_bounds__(256)
    merge_parts_kernel(const float* __restrict__ Dp, const int64_t* __restrict__ Ip, int nparts,
                       int64_t nq, int kin, int k, int largest, float* __restrict__ D,
                       int64_t* __restrict__ I) {
  constexpr int THREADS = 256, CAP = 4096;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename Sel::Smem& s = *reinterpret_cast<typename Sel::Smem*>(smem_raw);
  const int64_t q = blockIdx.x;
  const int64_t nper = (int64_t)nparts * kin;
  Sel::init(s);
  __syncthreads();
  uint64_t thr = ~0ull;
  for (int64_t base = 0; base < nper; base += THREADS) {
    const int64_t i = base + threadIdx.x;
    uint64_t c[1];
    uint32_t mask = 0;
    if (i < nper) {
      const int64_t p = i / kin, j = i % kin;
      const int64_t e = (p * nq + q) * kin + j;
      const int64_t id = Ip[e];
      if (id >= 0) {
        c[0] = composite(ordered_key(Dp[e], largest != 0), (uint32_t)id);
        mask = c[0] <= thr ? 1u : 0u;
      }
    }
    Sel::template push<1>(s, mask, c);
    __syncthreads();
    if (s.n_buf > CAP - THREADS) {
      Sel::compact(s, k);
      thr = s.thr;
    }
  }
  Sel::finish(s, k);
  for (int j = threadIdx.x; j < k; j += THREADS) {
    const uint64_t e = s.top[j];
    if (e == ~0ull) {
      D[q * k + j] = largest ? -INFINITY : INFINITY;
      I[q * k + j] = -1;
    } else {
      D[q * k + j] = key_value((uint32_t)(e >> 32), largest != 0);
      I[q * k + j] = (int64_t)(uint32_t)e;
    }
  }
}

template <int KP>
gbk_status launch_merge_parts(const float* Dp, const int64_t* Ip, int nparts, int64_t nq, int kin,
                              int k, bool largest, float* D, int64_t* I, cudaStream_t st) {
  using Sel = BlockSelect<256, KP, 4096>;
  auto kern = merge_parts_kernel<KP>;
  GBK_TRY(set_smem_limit(kern, sizeof(typename Sel::Smem)));
  kern<<<(unsigned)nq, 256, sizeof(typename Sel::Smem), st>>>(Dp, Ip, nparts, nq, kin, k,
                                                              largest ? 1 : 0, D, I);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace

gbk_status merge_parts_run(const float* Dp, const int64_t* Ip, int nparts, int64_t nq, int kin,
                           int k, bool largest, float* D, int64_t* I, cudaStream_t st) {
  if (nq == 0) return GBK_OK;
  ProfScope prof("merge_parts", st);
  if (k <= 32) return launch_merge_parts<32>(Dp, Ip, nparts, nq, kin, k, largest, D, I, st);
  if (k <= 64) return launch_merge_parts<64>(Dp, Ip, nparts, nq, kin, k, largest, D, I, st);
  if (k <= 128) return launch_merge_parts<128>(Dp, Ip, nparts, nq, kin, k, largest, D, I, st);
  if (k <= 256) return launch_merge_parts<256>(Dp, Ip, nparts, nq, kin, k, largest, D, I, st);
  if (k <= 512) return launch_merge_parts<512>(Dp, Ip, nparts, nq, kin, k, largest, D, I, st);
  return launch_merge_parts<1024>(Dp, Ip, nparts, nq, kin, k, largest, D, I, st);
}

namespace {

// ------------------------------------------------------------------ TMA descriptors

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn(gbk_status* st) {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  if (!fn) *st = set_error(GBK_ECUDA, "cuTensorMapEncodeTiled unavailable");
  return fn;
}

// Row-major [rows][cols] operand (cols already padded to a 128-byte multiple), boxes of
// 128 rows x 128 bytes with 128-byte swizzle; rows beyond `rows` read as zero.
gbk_status make_operand_map(CUtensorMap* m, const void* base, int64_t rows, int cols,
                            int elem_bytes) {
  gbk_status st = GBK_OK;
  EncodeTiledFn enc = encode_fn(&st);
  if (!enc) return st;
  const CUtensorMapDataType dt = elem_bytes == 4   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), 128u};
  cuuint32_t es[2] = {1u, 1u};
  CUresult r = enc(m, dt, 2, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(GBK_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return GBK_OK;
}

int elem_bytes_of(int prec) {
  const int kd = gemm_kind(prec);
  return kd == KIND_TF32X3 ? 4 : kd == KIND_FP8 ? 1 : 2;
}
int pieces_of(int prec) {
  const int kd = gemm_kind(prec);
  return kd == KIND_TF32X3 || kd == KIND_FP16X3 ? 2 : 1;
}
bool scaled_of(int prec) {
  const int kd = gemm_kind(prec);
  return kd == KIND_FP8 || kd == KIND_FP16X3;
}

}  // namespace

// ------------------------------------------------------------------ operand sets

gbk_status prepare_operand(const float* x, int64_t n, int d, int prec, int64_t nrows_pad,
                           float pad_norm, PreparedOperand* out, cudaStream_t st) {
  const int eb = elem_bytes_of(prec);
  const int dpad = (int)(((int64_t)d * eb + 127) / 128 * 128 / eb);
  out->prec = prec;
  out->n = n;
  out->d = d;
  out->dpad = dpad;
  out->nkb = dpad * eb / 128;
  const size_t piece = (size_t)std::max<int64_t>(n, 1) * dpad * eb;
  gbk_status r = out->data.alloc(piece * pieces_of(prec), st);
  if (r != GBK_OK) return r;
  r = out->norms.alloc(sizeof(float) * (size_t)nrows_pad, st);
  if (r != GBK_OK) return r;
  if (scaled_of(prec)) {
    r = out->scale.alloc(sizeof(float) * (size_t)nrows_pad, st);
    if (r != GBK_OK) return r;
  }
  unsigned char* base = out->data.as<unsigned char>();
  out->piece[0] = base;
  out->piece[1] = pieces_of(prec) > 1 ? base + piece : nullptr;
  const int warps = 8;
  const unsigned blocks = (unsigned)((nrows_pad + warps - 1) / warps);
  if (nrows_pad == 0) return GBK_OK;
  ProfScope prof("prep_operand", st);
  const int kind = gemm_kind(prec);
  if (kind == KIND_TF32X3)
    prep_tf32x3_kernel<<<blocks, warps * 32, 0, st>>>(
        x, n, d, dpad, (float*)out->piece[0], (float*)out->piece[1], out->norms.as<float>(),
        nrows_pad, pad_norm);
  else if (kind == KIND_BF16)
    prep_bf16_kernel<<<blocks, warps * 32, 0, st>>>(x, n, d, dpad, (__nv_bfloat16*)out->piece[0],
                                                   out->norms.as<float>(), nrows_pad, pad_norm);
  else if (kind == KIND_FP16X3)
    prep_fp16x3_kernel<<<(unsigned)((nrows_pad + warps * PREP16_ROWS - 1) / (warps * PREP16_ROWS)),
                         warps * 32, 0, st>>>(
        x, n, d, dpad, (__half*)out->piece[0], (__half*)out->piece[1], out->scale.as<float>(),
        out->norms.as<float>(), nrows_pad, pad_norm);
  else
    prep_fp8_kernel<<<blocks, warps * 32, 0, st>>>(x, n, d, dpad, (__nv_fp8_e4m3*)out->piece[0],
                                                  out->scale.as<float>(), out->norms.as<float>(),
                                                  nrows_pad, pad_norm);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

// Chunks whose candidate lists ([nq][chunks * epi][kp] composites) fit in 4 GiB.
static int list_chunk_cap(int64_t nq, int epi, int kp) {
  const int64_t per_chunk = std::max<int64_t>(1, nq * epi * kp * 8);
  return (int)std::max<int64_t>(1, std::min<int64_t>(512, ((int64_t)4 << 30) / per_chunk));
}

// Chunks S minimising waves x (tiles per chunk + per-item overhead); ties to fewer chunks.
// The overhead is a chunk's candidate lists learning their threshold again: measured at
// about 0.9 k tiles per (query tile, chunk) item for k = 16..128 (1e4 - 5e4 queries), none
// for k = 1 (callers pass a smaller k where a threshold pre-pass gives every list a
// near-final key from the start).  At most max_chunks (the candidate lists' memory, nq x chunks x lists, grows
// with S: with 10^8 queries a rounding gain of a few tiles would otherwise buy 100+
// chunks and 200 GB of lists).
int plan_chunks(int nqt, int ntiles, int grid_cap, int k, int max_chunks) {
  int best = 1;
  int64_t best_cost = INT64_MAX;
  const int64_t ovh = k <= 1 ? 0 : (9 * (int64_t)k + 9) / 10;
  for (int S = 1; S <= std::min(std::min(ntiles, 512), std::max(1, max_chunks)); S++) {
    const int64_t waves = ((int64_t)nqt * S + grid_cap - 1) / grid_cap;
    const int64_t tpc = (ntiles + S - 1) / S;
    const int64_t cost = waves * (tpc + ovh) * 64 + S;  // + small penalty per chunk (merge)
    if (cost < best_cost) {
      best_cost = cost;
      best = S;
    }
  }
  return best;
}

// Q rows [q0, q0 + qn) (all rows when qn < 0) against all of B.
gbk_status gemm_launch(int mode, int kpr, bool largest, const PreparedOperand& Q,
                       const PreparedOperand& B, GemmArgs a, cudaStream_t st, int64_t q0 = 0,
                       int64_t qn = -1) {
  const int prec = Q.prec;
  const int pieces = pieces_of(prec);
  const int eb = elem_bytes_of(prec);
  CUtensorMap maps[4];
  gbk_status r;
  if (qn < 0) qn = Q.n - q0;
  const size_t qoff = (size_t)q0 * Q.dpad * eb;  // a multiple of 128 bytes
  if ((r = make_operand_map(&maps[0], (const char*)Q.piece[0] + qoff, qn, Q.dpad, eb)) != GBK_OK)
    return r;
  if ((r = make_operand_map(&maps[2], B.piece[0], B.n, B.dpad, eb)) != GBK_OK) return r;
  if (pieces > 1) {
    if ((r = make_operand_map(&maps[1], (const char*)Q.piece[1] + qoff, qn, Q.dpad, eb)) !=
        GBK_OK)
      return r;
    if ((r = make_operand_map(&maps[3], B.piece[1], B.n, B.dpad, eb)) != GBK_OK) return r;
  } else {
    maps[1] = maps[0];
    maps[3] = maps[2];
  }
  const DeviceInfo& di = device_info();
  const bool queues = mode == MODE_SELECT && kpr > 0;
  const int epi = gemm_epi(prec);
  const GemmSmemLayout l0 = gemm_smem_layout(pieces, Q.nkb, 0, queues, epi);
  const int64_t avail = (int64_t)di.smem_optin - 1024 - l0.total;
  const int64_t stage_bytes = (int64_t)pieces * GEMM_TILE_BYTES + 16;
  int stages = (int)std::min<int64_t>(8, avail / stage_bytes);
  a.stream_a = 0;
  a.tmem_a = 0;
  a.nacc = GEMM_NACC;
  // A resident in shared memory leaves a ring shorter than two tiles: keep A in tensor
  // memory instead (its pieces x k-blocks x 32 columns beside two accumulator buffers)
  // when that makes room for a two-tile ring, so both MMA issuers can run; the remaining
  // columns hold 3 (d <= 128 for the FP16 split) or 2 accumulator buffers.  With only 2,
  // not for candidate lists longer than 32: their merges make the epilogue the bound and
  // it needs more slack (10^4 x 10^6 x 128, FP16 split, 2 buffers: k = 10 7.5 -> 6.4 ms,
  // k = 100 8.5 -> 9.1 ms)
  const int acols = pieces * Q.nkb * 32;  // tensor-memory columns of A
  const int nacc_t = std::min(GEMM_NACC, (512 - acols) / GEMM_BN);
  if (stages < 2 * Q.nkb && nacc_t >= 2 && (kpr <= 1 || nacc_t >= 3)) {
    const GemmSmemLayout lt = gemm_smem_layout(pieces, 1, 0, queues, epi);
    const int st_t = (int)std::min<int64_t>(8, ((int64_t)di.smem_optin - 1024 - lt.total) /
                                                   stage_bytes);
    if (st_t >= 2 * Q.nkb) {
      stages = st_t;
      a.tmem_a = 1;
      a.nacc = nacc_t;
    }
  }
  if (stages < 2) {
    // the query tile does not fit beside a 2-stage ring: stream its k-blocks with B's
    const GemmSmemLayout l1 = gemm_smem_layout(2 * pieces, 0, 0, queues, epi);
    const int64_t avail1 = (int64_t)di.smem_optin - 1024 - l1.total;
    stages = (int)std::min<int64_t>(8, avail1 / (2 * stage_bytes));
    if (stages < 2)
      return set_error(GBK_EUNSUPPORTED, "d=%d too large for the fused tensor-core kernel", Q.d);
    a.stream_a = 1;
  }
  a.stages = stages;
  a.nkb = Q.nkb;
  a.dual = stages >= 2 * Q.nkb ? 1 : 0;
  // at least half the SM's shared memory, so one CTA per SM owns the TMEM it allocates
  const GemmSmemLayout lf =
      a.stream_a ? gemm_smem_layout(2 * pieces, 0, stages, queues, epi)
                 : gemm_smem_layout(pieces, a.tmem_a ? 1 : Q.nkb, stages, queues, epi);
  const size_t smem = std::max<size_t>(lf.total + 1024, di.smem_optin / 2 + 1024);
  const int nitems = a.nqt * a.chunks;
  const int grid = std::min(nitems, di.sm_count);
  a.status = device_status();
  if (!a.status) return set_error(GBK_ECUDA, "device status word unavailable");
  const int kind = gemm_kind(prec);
  ProfScope prof(kind == KIND_TF32X3   ? "dist_gemm_tf32x3"
                 : kind == KIND_FP16X3 ? "dist_gemm_fp16x3"
                 : kind == KIND_BF16   ? "dist_gemm_bf16"
                                       : "dist_gemm_fp8",
                 st);
  if (kind == KIND_TF32X3)
    return launch_dist_gemm_tf32x3(mode, kpr, largest, maps, a, grid, smem, st);
  if (kind == KIND_FP16X3)
    return launch_dist_gemm_fp16x3(mode, kpr, largest, maps, a, grid, smem, st);
  if (kind == KIND_BF16)
    return launch_dist_gemm_bf16(mode, kpr, largest, maps, a, grid, smem, st);
  return launch_dist_gemm_fp8(mode, kpr, largest, maps, a, grid, smem, st);
}

// Distances of every (query, database) pair: max(0, ||x||^2 + ||y||^2 - 2<x,y>) for L2
// (||y||^2 - 2<x,y> without the query norm when add_xnorm is false), <x,y> for inner
// product.  Query rows [q0, q0 + qn) of Q (all when qn < 0); out row 0 is query q0.
gbk_status pairwise_run(const PreparedOperand& Q, const PreparedOperand& B, bool ip, float* out,
                        int64_t ldo, cudaStream_t st, int64_t q0, int64_t qn, bool add_xnorm) {
  if (qn < 0) qn = Q.n - q0;
  GemmArgs a = {};
  a.nq = (int)qn;
  a.nb = (int)B.n;
  a.nqt = (int)((qn + GEMM_BM - 1) / GEMM_BM);
  a.ntiles = (int)((B.n + GEMM_BN - 1) / GEMM_BN);
  a.chunks = plan_chunks(a.nqt, a.ntiles, device_info().sm_count, 1);
  a.tpc = (a.ntiles + a.chunks - 1) / a.chunks;
  a.chunks = (a.ntiles + a.tpc - 1) / a.tpc;
  a.ynorm = B.norms.as<float>();
  a.xnorm = ip || !add_xnorm ? nullptr : Q.norms.as<float>() + q0;
  a.qscale = Q.scale.p ? Q.scale.as<float>() + q0 : nullptr;
  a.bscale = B.scale.as<float>();
  a.out = out;
  a.ldo = ldo;
  return gemm_launch(MODE_STORE, 0, ip, Q, B, a, st, q0, qn);
}

// Row norms of the two pieces of a split operand, in the operand's units: hn = s ||hi||,
// ln = s ||lo|| (s the row scale, 1 without one), accumulated in float32 and rounded up by
// 2^-20 relative so they bound the exact norms.  One warp per row.  With `maxes` the
// rows' maxima go there (atomicMax on the bits of non-negative floats) instead of hn, ln.
template <typename E>
__global__ void split_norms_kernel(const E* __restrict__ p0, const E* __restrict__ p1,
                                   const float* __restrict__ scale, int64_t n, int dpad,
                                   float* __restrict__ hn, float* __restrict__ ln,
                                   float* __restrict__ maxes) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float mh = 0.f, ml = 0.f;
  for (int64_t r = w0; r < n; r += nw) {
    float sh = 0.f, sl = 0.f;
    for (int t = lane; t < dpad; t += 32) {
      const float h = (float)p0[r * dpad + t], l = (float)p1[r * dpad + t];
      sh = fmaf(h, h, sh);
      sl = fmaf(l, l, sl);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sh += __shfl_xor_sync(FULL_MASK, sh, o);
      sl += __shfl_xor_sync(FULL_MASK, sl, o);
    }
    const float sc = scale ? scale[r] : 1.f;
    const float h = sqrtf(sh) * sc * (1.f + 0x1p-20f), l = sqrtf(sl) * sc * (1.f + 0x1p-20f);
    if (maxes) {
      mh = fmaxf(mh, h);
      ml = fmaxf(ml, l);
    } else if (lane == 0) {
      hn[r] = h;
      ln[r] = l;
    }
  }
  if (maxes && lane == 0) {
    atomicMax(reinterpret_cast<unsigned int*>(&maxes[0]), __float_as_uint(mh));
    atomicMax(reinterpret_cast<unsigned int*>(&maxes[1]), __float_as_uint(ml));
  }
}

// thr[q] = ordered key of the k-th best value of row q of Dk [nq][k] (sorted best first).
// With xh (one-pass pre-pass over the high pieces, hi_only) the value is first widened by
// a bound on how far the one-pass value a of any row of the prefix can lie from the value
// v the full pass ranks (so the k rows behind the k-th best a have v within the key):
//   v - a = -2 (<xh, yl> + <xl, yh>) (L2; without the -2 for inner product) plus both
//   accumulations' rounding and the epilogue's;  |<xh, yl>| <= ||xh|| ||yl|| (Cauchy-
//   Schwarz) with the database side's maxima over the prefix (stats: max ||yh||, ||yl||),
//   the float32 accumulations (at most 4 dpad additions in all) within 4 dpad 2^-21
//   ||x|| ||y||, the epilogue's rounding within 2^-23 (||y||^2 + 2 ||x|| ||y||).
__global__ void kth_key_kernel(const float* __restrict__ Dk, int64_t nq, int k, bool largest,
                               const float* __restrict__ xh, const float* __restrict__ xl,
                               const float* __restrict__ stats, int dpad,
                               uint32_t* __restrict__ thr) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const float d = Dk[q * k + k - 1];
  if (!xh || !(fabsf(d) <= 3.0e38f)) {
    thr[q] = ordered_key(d, largest);
    return;
  }
  const double Xh = xh[q], Xl = xl[q], Yh = stats[0], Yl = stats[1];
  const double X = Xh + Xl, Y = Yh + Yl;
  const double cross = Xh * Yl + Xl * Yh;
  const double acc = 4.0 * dpad * 0x1p-21 * X * Y;
  const double eps = (largest ? cross + acc + 0x1p-23 * X * Y
                              : 2.0 * (cross + acc) + 0x1p-23 * (Y * Y + 2.0 * X * Y)) *
                         (1.0 + 0x1p-10) +
                     1e-30;
  const float t = largest ? __double2float_rd((double)d - eps) : __double2float_ru((double)d + eps);
  thr[q] = ordered_key(t, largest);
}

// Database tiles of the threshold pre-pass for a fused top-k over `ntiles` tiles (0: none).
// The pre-pass takes the best value of every (query, tile, column half) over a prefix of
// the database; the k-th best of those values is attained by k distinct rows, so it bounds
// the k-th nearest distance from the start and the fused selection queues far fewer
// candidates (a streamed threshold admits about k (1 + ln(n / k)) of n values, a threshold
// from a prefix of n / f rows about k (1 + ln f)).  prefilter: -1 off, 1 on for k > 1, 0 on
// for k >= 32 (k >= 64 with the TF32 split, whose slower GEMM makes the pre-pass dearer).
// The split kinds take the prefix in one MMA pass over their high pieces (the bound then
// widened, kth_key_kernel); the pass is bound by its epilogue, so the prefix is sized on
// measurements: a third of the database for k > 64, a quarter below (at least k values,
// at most half of it).  On 10^4 x 10^6 x 128, FP16 split, whole calls with a third / a
// quarter: k = 64 7.12 / 7.01 ms, k = 100 7.96 / 8.01, k = 256 12.9 / 14.7 (half: 22.1);
// k = 32 main pass 5.17 / 4.91 / 4.86 ms after 1/6, 1/4, 1/3; at k = 10 the pre-pass costs
// about what it saves and stays off.
static int prefilter_tiles(int prefilter, int k, int ntiles, int epi) {
  const int kmin = epi == 1 ? 64 : 32;
  if (prefilter < 0 || k <= 1 || (prefilter == 0 && k < kmin)) return 0;
  const int f = k > 64 ? 3 : 4;  // 1 / prefix fraction
  const int ts = std::max((ntiles + f - 1) / f, (k + epi - 1) / epi);
  return 2 * ts <= ntiles ? ts : 0;
}

// The threshold pre-pass (see prefilter_tiles) over the first tiles of B: per-(query, tile,
// half) best values, then their k-th best per query as its initial threshold key thr[q]
// (profiled as "*_bound").  Does nothing when prefilter_tiles gives none.
static gbk_status prefilter_run(const PreparedOperand& Q, const PreparedOperand& B, int64_t nq,
                                int64_t nb, int ntiles, int k, bool ip, int prefilter,
                                uint32_t* thr, cudaStream_t st) {
  const int epi = gemm_epi(Q.prec);
  const int ts = prefilter_tiles(prefilter, k, ntiles, epi);
  if (!ts) return GBK_OK;
  ProfSuffix tag("_bound");
  gbk_status r;
  const int nv = ts * epi;
  Scratch mins, Dk, Ik;
  if ((r = mins.alloc(sizeof(float) * (size_t)nq * nv, st)) != GBK_OK) return r;
  if ((r = Dk.alloc(sizeof(float) * (size_t)nq * k, st)) != GBK_OK) return r;
  if ((r = Ik.alloc(sizeof(int64_t) * (size_t)nq * k, st)) != GBK_OK) return r;
  GemmArgs p = {};
  p.nq = (int)nq;
  p.nb = (int)std::min<int64_t>(nb, (int64_t)ts * GEMM_BN);
  p.nqt = (int)((nq + GEMM_BM - 1) / GEMM_BM);
  p.ntiles = ts;
  p.chunks = plan_chunks(p.nqt, ts, device_info().sm_count, 1);
  p.tpc = (ts + p.chunks - 1) / p.chunks;
  p.chunks = (ts + p.tpc - 1) / p.tpc;
  p.k = 1;
  p.kp = 1;
  p.ynorm = B.norms.as<float>();
  p.qscale = Q.scale.as<float>();
  p.bscale = B.scale.as<float>();
  p.out = mins.as<float>();
  p.ldo = nv;
  p.tile_min = 1;
  // the split kinds bound with one pass over their high pieces, widened afterwards by the
  // bound on the two cross terms it leaves out (kth_key_kernel)
  const bool split = pieces_of(Q.prec) > 1;
  p.hi_only = split ? 1 : 0;
  if ((r = gemm_launch(MODE_SELECT, 0, ip, Q, B, p, st)) != GBK_OK) return r;
  Scratch xn, stats;
  if (split) {
    ProfScope prof("split_norms", st);
    if ((r = xn.alloc(sizeof(float) * 2 * (size_t)nq, st)) != GBK_OK) return r;
    if ((r = stats.alloc(2 * sizeof(float), st)) != GBK_OK) return r;
    GBK_CUDA_CHECK(cudaMemsetAsync(stats.p, 0, 2 * sizeof(float), st));
    const int64_t rows = p.nb;
    const unsigned gb = (unsigned)std::min<int64_t>((rows + 7) / 8, 8ll * device_info().sm_count);
    const unsigned gq = (unsigned)((nq + 7) / 8);
    const float* bsc = scaled_of(B.prec) ? B.scale.as<float>() : nullptr;
    const float* qsc = scaled_of(Q.prec) ? Q.scale.as<float>() : nullptr;
    float* xh = xn.as<float>();
    if (gemm_kind(Q.prec) == KIND_FP16X3) {
      split_norms_kernel<__half><<<gb, 256, 0, st>>>(
          (const __half*)B.piece[0], (const __half*)B.piece[1], bsc, rows, B.dpad, nullptr,
          nullptr, stats.as<float>());
      split_norms_kernel<__half><<<gq, 256, 0, st>>>(
          (const __half*)Q.piece[0], (const __half*)Q.piece[1], qsc, nq, Q.dpad, xh, xh + nq,
          nullptr);
    } else {
      split_norms_kernel<float><<<gb, 256, 0, st>>>(
          (const float*)B.piece[0], (const float*)B.piece[1], bsc, rows, B.dpad, nullptr,
          nullptr, stats.as<float>());
      split_norms_kernel<float><<<gq, 256, 0, st>>>(
          (const float*)Q.piece[0], (const float*)Q.piece[1], qsc, nq, Q.dpad, xh, xh + nq,
          nullptr);
    }
    GBK_LAUNCH_CHECK();
  }
  if ((r = kselect_run(mins.as<float>(), nq, nv, k, ip, Dk.as<float>(), Ik.as<int64_t>(), st,
                       nullptr)) != GBK_OK)
    return r;
  ProfScope prof("kth_key", st);
  kth_key_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(
      Dk.as<float>(), nq, k, ip, split ? xn.as<float>() : nullptr,
      split ? xn.as<float>() + nq : nullptr, split ? stats.as<float>() : nullptr, Q.dpad, thr);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

// Top-k (ascending distance / descending inner product) of prepared operands in their
// own precision, written as full distances D and database rows I.
static gbk_status select_run(const float* xq, const PreparedOperand& Q, const PreparedOperand& B,
                             int64_t nq, int64_t nb, int d, int k, bool ip, int chunks_opt,
                             int prefilter, float* D, int64_t* I, cudaStream_t st) {
  gbk_status r;
  const int ntiles = (int)((nb + GEMM_BN - 1) / GEMM_BN);
  if (k > 512 || (k > 1 && nb <= 65536)) {
    // Large k, or k > 1 against a short database (a coarse quantizer): distance blocks
    // of t_q queries x nb (section 5.1 tiling over queries), each followed by a row-wise
    // k-selection.  The blocks hold ||y||^2 - 2<x,y> (<x,y> for inner product), the values
    // the fused path ranks, so both routes select the same neighbours; the query norm is
    // added to the k winners afterwards.
    const int64_t budget = (int64_t)1 << 31;  // bytes of distance block
    int64_t tq = std::max<int64_t>(GEMM_BM, budget / (4 * nb) / GEMM_BM * GEMM_BM);
    tq = std::min(tq, nq);
    Scratch blk;
    if ((r = blk.alloc(sizeof(float) * (size_t)(tq * nb), st)) != GBK_OK) return r;
    for (int64_t q0 = 0; q0 < nq; q0 += tq) {
      const int64_t nqb = std::min(tq, nq - q0);
      if ((r = pairwise_run(Q, B, ip, blk.as<float>(), nb, st, q0, nqb, false)) != GBK_OK)
        return r;
      if ((r = kselect_run(blk.as<float>(), nqb, nb, k, ip, D + q0 * k, I + q0 * k, st,
                           nullptr)) != GBK_OK)
        return r;
    }
    if (!ip) {
      add_norm_clamp_kernel<<<(unsigned)((nq * k + 255) / 256), 256, 0, st>>>(
          D, nq, k, Q.norms.as<float>());
      GBK_LAUNCH_CHECK();
    }
    return GBK_OK;
  }
  GemmArgs a = {};
  a.nq = (int)nq;
  a.nb = (int)nb;
  a.nqt = (int)((nq + GEMM_BM - 1) / GEMM_BM);
  a.ntiles = ntiles;
  a.kp = k == 1 ? 1 : std::max(32, 1 << (32 - __builtin_clz((unsigned)(k - 1))));
  // With the threshold pre-pass every list starts from a near-final key, so a chunk's
  // lists relearn little: for k >= 64 the plan charges a tenth of the usual per-item
  // overhead (10^4 x 10^6 x 128: k = 64 / 100 / 256 6.98 -> 6.91, 8.00 -> 7.78,
  // 12.95 -> 11.91 ms; at k = 32 the usual charge stays, 6.19 against 6.24 ms)
  const int kplan =
      (k >= 64 && prefilter_tiles(prefilter, k, ntiles, gemm_epi(Q.prec))) ? (k + 8) / 9 : k;
  a.chunks = chunks_opt > 0 ? std::min(chunks_opt, ntiles)
                            : plan_chunks(a.nqt, ntiles, device_info().sm_count, kplan,
                                          list_chunk_cap(nq, gemm_epi(Q.prec), a.kp));
  a.tpc = (ntiles + a.chunks - 1) / a.chunks;
  a.chunks = (ntiles + a.tpc - 1) / a.tpc;
  a.k = k;
  a.ynorm = B.norms.as<float>();
  a.qscale = Q.scale.as<float>();
  a.bscale = B.scale.as<float>();
  const int lists = a.chunks * gemm_epi(Q.prec);  // candidate lists per query
  Scratch part, thr;
  if ((r = part.alloc(sizeof(uint64_t) * (size_t)nq * lists * a.kp, st)) != GBK_OK) return r;
  if ((r = thr.alloc(sizeof(uint32_t) * (size_t)nq, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemsetAsync(thr.p, 0xff, sizeof(uint32_t) * (size_t)nq, st));
  if ((r = prefilter_run(Q, B, nq, nb, ntiles, k, ip, prefilter, thr.as<uint32_t>(), st)) !=
      GBK_OK)
    return r;
  a.part = part.as<uint64_t>();
  a.thr_key = thr.as<uint32_t>();
  const int kpr = k == 1 ? 0 : a.kp / 32;
  if ((r = gemm_launch(MODE_SELECT, kpr, ip, Q, B, a, st)) != GBK_OK) return r;
  return knn_merge(a.part, nq, lists, a.kp, k, ip ? nullptr : Q.norms.as<float>(), ip, D, I, st);
}

// idx[0 .. *cnt) = the queries with certified[q] == 0 (in no particular order)
__global__ void uncertified_kernel(const int32_t* __restrict__ certified, int64_t nq,
                                   int64_t* __restrict__ idx, int32_t* __restrict__ cnt) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq && certified[q] == 0) idx[atomicAdd(cnt, 1)] = q;
}

// rows j of (Du, Iu) replace rows idx[j] of (D, I); certified[idx[j]] = 2
__global__ void scatter_rows_kernel(const float* __restrict__ Du, const int64_t* __restrict__ Iu,
                                    const int64_t* __restrict__ idx, int k, float* __restrict__ D,
                                    int64_t* __restrict__ I, int32_t* __restrict__ certified) {
  const int64_t j = blockIdx.x, q = idx[j];
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    D[q * k + t] = Du[j * k + t];
    I[q * k + t] = Iu[j * k + t];
  }
  if (threadIdx.x == 0) certified[q] = 2;
}

gbk_status prepare_database(const float* xb, int64_t nb, int d, int prec, PreparedOperand* B,
                            cudaStream_t st) {
  const int ntiles = (int)((nb + GEMM_BN - 1) / GEMM_BN);
  return prepare_operand(xb, nb, d, prec, (int64_t)ntiles * GEMM_BN, 0.f, B, st);
}

gbk_status knn_run(const float* xq, int64_t nq, const float* xb, int64_t nb, int d, int k,
                   int metric, float* D, int64_t* I, const KnnPlan& plan, cudaStream_t st) {
  if (nq == 0) return GBK_OK;
  PreparedOperand B;
  gbk_status r;
  if ((r = prepare_database(xb, nb, d, plan.prec, &B, st)) != GBK_OK) return r;
  return knn_run_prepared(xq, nq, xb, B, nb, d, k, metric, D, I, plan, st);
}

gbk_status knn_run_prepared(const float* xq, int64_t nq, const float* xb,
                            const PreparedOperand& B, int64_t nb, int d, int k, int metric,
                            float* D, int64_t* I, const KnnPlan& plan, cudaStream_t st) {
  if (nq == 0) return GBK_OK;
  const bool ip = metric == GBK_METRIC_IP;
  PreparedOperand Q;
  gbk_status r;
  if ((r = prepare_operand(xq, nq, d, plan.prec, nq, 0.f, &Q, st)) != GBK_OK) return r;
  if (plan.prec == GBK_PREC_FP32 || plan.prec == GBK_PREC_TF32X3)  // float32-accurate kinds
    return select_run(xq, Q, B, nq, nb, d, k, ip, plan.chunks, plan.prefilter, D, I, st);
  // low precision: over-fetch k' candidates, then the exact float32 re-rank + certificate.
  // Default k' = 4k for k <= 16 and k + k/4 above: longer candidate lists slow the fused
  // selection far more than the certificate gains (10^4 x 10^6 x 128, k = 100, BF16:
  // k' = 400 certifies every query but takes 100 ms, k' = 125 takes 14 ms and leaves the
  // queries to the float32 repair).  Not rounded up to the lists' power-of-two length: a
  // larger k' loosens the selection threshold and costs candidate pushes.
  int kp = plan.kprime > 0 ? plan.kprime : (k <= 16 ? 4 * k : k + k / 4);
  kp = std::min(kp, GBK_MAX_K);
  kp = (int)std::min<int64_t>(std::max(kp, k), nb);
  Scratch Dc, Ic, cert;
  if ((r = Dc.alloc(sizeof(float) * (size_t)nq * kp, st)) != GBK_OK) return r;
  if ((r = Ic.alloc(sizeof(int64_t) * (size_t)nq * kp, st)) != GBK_OK) return r;
  int32_t* cp = plan.certified;
  if (plan.exact && !cp) {
    if ((r = cert.alloc(sizeof(int32_t) * (size_t)nq, st)) != GBK_OK) return r;
    cp = cert.as<int32_t>();
  }
  if ((r = select_run(xq, Q, B, nq, nb, d, kp, ip, plan.chunks, plan.prefilter, Dc.as<float>(),
                      Ic.as<int64_t>(), st)) != GBK_OK)
    return r;
  if ((r = rerank_run(xq, xb, nq, nb, d, kp, k, ip, plan.prec, Q.norms.as<float>(),
                      Q.scale.as<float>(), B.norms.as<float>(), B.scale.as<float>(),
                      Ic.as<int64_t>(), Dc.as<float>(), D, I, cp, plan.error_bound, st)) != GBK_OK)
    return r;
  if (!plan.exact) return GBK_OK;
  // queries the certificate does not cover: searched again on the float32 path, whose
  // results replace theirs (certified = 2)
  Scratch cnt, idx;
  if ((r = cnt.alloc(sizeof(int32_t), st)) != GBK_OK) return r;
  if ((r = idx.alloc(sizeof(int64_t) * (size_t)nq, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t), st));
  uncertified_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(cp, nq, idx.as<int64_t>(),
                                                                   cnt.as<int32_t>());
  GBK_LAUNCH_CHECK();
  int32_t nu = 0;
  GBK_CUDA_CHECK(cudaMemcpyAsync(&nu, cnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  GBK_CUDA_CHECK(cudaStreamSynchronize(st));
  if (nu == 0) return GBK_OK;
  Scratch Xu, Du, Iu;
  if ((r = Xu.alloc(sizeof(float) * (size_t)nu * d, st)) != GBK_OK) return r;
  if ((r = Du.alloc(sizeof(float) * (size_t)nu * k, st)) != GBK_OK) return r;
  if ((r = Iu.alloc(sizeof(int64_t) * (size_t)nu * k, st)) != GBK_OK) return r;
  if ((r = gather_rows_run(xq, idx.as<int64_t>(), nu, d, Xu.as<float>(), st)) != GBK_OK) return r;
  KnnPlan p32;
  p32.chunks = plan.chunks;
  p32.prefilter = plan.prefilter;
  if ((r = knn_run(Xu.as<float>(), nu, xb, nb, d, k, metric, Du.as<float>(), Iu.as<int64_t>(),
                   p32, st)) != GBK_OK)
    return r;
  scatter_rows_kernel<<<(unsigned)nu, 128, 0, st>>>(Du.as<float>(), Iu.as<int64_t>(),
                                                    idx.as<int64_t>(), k, D, I, cp);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace gbk

namespace gbk {

// Exact k-NN of host-resident queries and database, results to host memory.  With a
// float32-accurate precision and the fused selection (k <= 512, nb > 65,536) the database
// crosses to the GPU in growing pieces on a second stream while the fused GEMM runs
// over the pieces already there: each piece's launch keeps its own candidate lists (one
// slice of a shared buffer, its rows offset to database numbering) and all pieces filter
// with the same per-query threshold keys, so one final merge gives the same result as a
// single launch over the whole database.  Other cases copy everything, then search.
gbk_status knn_host_run(const float* xq_h, int64_t nq, const float* xb_h, int64_t nb, int d,
                        int k, int metric, float* D_h, int64_t* I_h, const KnnPlan& plan,
                        cudaStream_t st) {
  if (nq == 0) return GBK_OK;
  gbk_status r;
  const bool ip = metric == GBK_METRIC_IP;
  Scratch xq, xb, Dd, Id;
  if ((r = xq.alloc(sizeof(float) * (size_t)nq * d, st)) != GBK_OK) return r;
  if ((r = xb.alloc(sizeof(float) * (size_t)nb * d, st)) != GBK_OK) return r;
  if ((r = Dd.alloc(sizeof(float) * (size_t)nq * k, st)) != GBK_OK) return r;
  if ((r = Id.alloc(sizeof(int64_t) * (size_t)nq * k, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(xq.p, xq_h, sizeof(float) * (size_t)nq * d,
                                 cudaMemcpyHostToDevice, st));
  const bool accurate = plan.prec == GBK_PREC_FP32 || plan.prec == GBK_PREC_TF32X3;
  // pieces of 2^16, 2^17, 2^18 ... rows: the search runs about twice as long per row as
  // the copy, so each piece arrives while the previous one is searched and only the first,
  // small one is exposed; a remainder shorter than half the next size joins the last piece
  int64_t pstart[17];
  int np = 0;
  if (accurate && k <= 512 && nb > 65536) {
    int64_t r0 = 0, size = (int64_t)1 << 16;
    while (r0 < nb && np < 16) {
      int64_t n = std::min(size, nb - r0);
      if (nb - (r0 + n) < size || np == 15) n = nb - r0;  // the remainder joins this piece
      pstart[np++] = r0;
      r0 += n;
      size *= 2;
    }
    pstart[np] = nb;
  }
  if (np <= 1) {
    GBK_CUDA_CHECK(cudaMemcpyAsync(xb.p, xb_h, sizeof(float) * (size_t)nb * d,
                                   cudaMemcpyHostToDevice, st));
    if ((r = knn_run(xq.as<float>(), nq, xb.as<float>(), nb, d, k, metric, Dd.as<float>(),
                     Id.as<int64_t>(), plan, st)) != GBK_OK)
      return r;
  } else {
    // piece p: rows [pstart[p], pstart[p + 1]); all but the last start at multiples of the
    // tile (powers of two >= 2^16)
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[17] = {};
    GBK_CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    // On every exit `st` first waits for all copies (so no buffer is freed under one in
    // flight, even after an error); the stream and events are released once their queued
    // work completes.
    struct Cleanup {
      cudaStream_t s, main;
      cudaEvent_t* e;
      ~Cleanup() {
        for (int i = 0; i < 17; i++)
          if (e[i]) cudaStreamWaitEvent(main, e[i], 0);
        for (int i = 0; i < 17; i++)
          if (e[i]) cudaEventDestroy(e[i]);
        if (s) cudaStreamDestroy(s);
      }
    } cleanup{cs, st, ev};
    for (int i = 0; i <= np; i++)
      GBK_CUDA_CHECK(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
    // the copy stream starts after the buffers exist on `st`
    GBK_CUDA_CHECK(cudaEventRecord(ev[np], st));
    GBK_CUDA_CHECK(cudaStreamWaitEvent(cs, ev[np], 0));
    for (int p = 0; p < np; p++) {
      const int64_t r0 = pstart[p], n = pstart[p + 1] - r0;
      GBK_CUDA_CHECK(cudaMemcpyAsync(xb.as<float>() + r0 * d, xb_h + r0 * d,
                                     sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice, cs));
      GBK_CUDA_CHECK(cudaEventRecord(ev[p], cs));
    }
    PreparedOperand Q;
    if ((r = prepare_operand(xq.as<float>(), nq, d, plan.prec, nq, 0.f, &Q, st)) != GBK_OK)
      return r;
    const int epi = gemm_epi(Q.prec);
    const int nqt = (int)((nq + GEMM_BM - 1) / GEMM_BM);
    const int kp = k == 1 ? 1 : std::max(32, 1 << (32 - __builtin_clz((unsigned)(k - 1))));
    int chunks[16], tpc[16], list0[16], lists = 0;
    for (int p = 0; p < np; p++) {
      const int64_t n = pstart[p + 1] - pstart[p];
      const int nt = (int)((n + GEMM_BN - 1) / GEMM_BN);
      int c = plan.chunks > 0 ? std::min(plan.chunks, nt)
                              : plan_chunks(nqt, nt, device_info().sm_count, k,
                                            list_chunk_cap(nq, epi, kp) / np);
      tpc[p] = (nt + c - 1) / c;
      chunks[p] = (nt + tpc[p] - 1) / tpc[p];
      list0[p] = lists;
      lists += chunks[p] * epi;
    }
    Scratch part, thr;
    if ((r = part.alloc(sizeof(uint64_t) * (size_t)nq * lists * kp, st)) != GBK_OK) return r;
    if ((r = thr.alloc(sizeof(uint32_t) * (size_t)nq, st)) != GBK_OK) return r;
    GBK_CUDA_CHECK(cudaMemsetAsync(thr.p, 0xff, sizeof(uint32_t) * (size_t)nq, st));
    for (int p = 0; p < np; p++) {
      const int64_t r0 = pstart[p], n = pstart[p + 1] - r0;
      const int nt = (int)((n + GEMM_BN - 1) / GEMM_BN);
      GBK_CUDA_CHECK(cudaStreamWaitEvent(st, ev[p], 0));
      PreparedOperand B;
      if ((r = prepare_operand(xb.as<float>() + r0 * d, n, d, plan.prec, (int64_t)nt * GEMM_BN,
                               0.f, &B, st)) != GBK_OK)
        return r;
      if (p == 0 && (r = prefilter_run(Q, B, nq, n, nt, k, ip, plan.prefilter,
                                       thr.as<uint32_t>(), st)) != GBK_OK)
        return r;
      GemmArgs a = {};
      a.nq = (int)nq;
      a.nb = (int)n;
      a.nqt = nqt;
      a.ntiles = nt;
      a.chunks = chunks[p];
      a.tpc = tpc[p];
      a.k = k;
      a.kp = kp;
      a.ynorm = B.norms.as<float>();
      a.qscale = Q.scale.as<float>();
      a.bscale = B.scale.as<float>();
      a.part = part.as<uint64_t>();
      a.part_lists = lists;
      a.list0 = list0[p];
      a.row0 = r0;
      a.thr_key = thr.as<uint32_t>();
      if ((r = gemm_launch(MODE_SELECT, k == 1 ? 0 : kp / 32, ip, Q, B, a, st)) != GBK_OK)
        return r;
    }
    if ((r = knn_merge(part.as<uint64_t>(), nq, lists, kp, k, ip ? nullptr : Q.norms.as<float>(),
                       ip, Dd.as<float>(), Id.as<int64_t>(), st)) != GBK_OK)
      return r;
  }
  GBK_CUDA_CHECK(cudaMemcpyAsync(D_h, Dd.p, sizeof(float) * (size_t)nq * k,
                                 cudaMemcpyDeviceToHost, st));
  GBK_CUDA_CHECK(cudaMemcpyAsync(I_h, Id.p, sizeof(int64_t) * (size_t)nq * k,
                                 cudaMemcpyDeviceToHost, st));
  return GBK_OK;
}

}  // namespace gbk
