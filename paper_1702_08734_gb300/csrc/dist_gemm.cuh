// Exact k-NN on the tensor cores: the -2<x, y> term of Eq. (2) (section 2) computed by
// tcgen05 MMAs into TMEM, with the k-selection fused into the epilogue so the partial
// distance matrix D' never reaches HBM (the paper fuses only the norm addition with the
// selection and writes D' once, section 5.1; on sm_103a the accumulator tile can be
// filtered straight out of tensor memory).
//
// CTA = 96 + 128 * EPI threads, one per SM (persistent):
//   warp 0      TMA producer: the 128-query A tile (all of d, resident for a work item)
//               and a ring of 128-row database B k-blocks (128 bytes of K per row,
//               SWIZZLE_128B boxes);
//   warps 1, 2  MMA issuers (one thread each, alternate tiles; warp 1 also allocates
//               TMEM): 128x128 tiles, K = 32 bytes per instruction, GEMM_NACC
//               accumulator buffers of 128 TMEM columns, so the MMAs run several tiles
//               ahead of the epilogue;
//   warps 3..   epilogue, EPI warpgroups each owning 128 / EPI columns of every tile:
//               thread t of quarter q owns query row 32q+t (its TMEM lane), reads 32
//               accumulator columns at a time, forms ||y||^2 - 2<x,y> (or <x,y> for
//               inner product), and tests the batch's best value against its query's
//               threshold; only batches holding a survivor queue their survivors, and
//               full queues are merged by the whole warp into the query's sorted
//               candidate list (bitonic network over shuffles).
// Work item = (query tile, database chunk); items are chunk-major so all CTAs sweep
// the database in near lockstep and each B tile is fetched from HBM about once.  A
// global per-query threshold (ordered key, atomicMin) is shared by all lists of a query:
// every list merge publishes its k-th distance and every epilogue thread re-reads the key
// once per tile, so chunks running at the same time and both column halves filter with
// the best k-th distance found so far.
//
// Precision variants (KIND): TF32X3 keeps float32 accuracy by splitting each operand
// x = hi + lo into TF32 pieces and accumulating hi*hi + hi*lo + lo*hi (Ootomo & Yokota,
// "Recovering single precision accuracy from Tensor Cores while surpassing the FP32
// theoretical peak performance", IJHPCA 2022); FP16X3 applies the same split to FP16
// pieces of the row scaled by a power of two s = 2^e >= max|x| (x / s exact, hi = fp16(x/s),
// lo = fp16(x/s - hi): 22 significand bits, the absolute error of lo below 2^-25 of the
// row's largest element) at the FP16 MMA rate, s_x s_y applied in the epilogue; BF16 and
// FP8 (E4M3, per-row scale) are one-pass.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cstdint>

#include "common.cuh"
#include "select_core.cuh"
#include "sm100.cuh"

namespace gbk {

enum GemmKind : int { KIND_TF32X3 = 0, KIND_BF16 = 1, KIND_FP8 = 2, KIND_FP16X3 = 3 };
enum GemmMode : int { MODE_SELECT = 0, MODE_STORE = 1 };

constexpr int GEMM_BM = 128;          // queries per tile (TMEM lanes)
constexpr int GEMM_BN = 128;          // database rows per tile (TMEM columns per buffer)
constexpr int GEMM_NACC = 4;          // TMEM accumulator buffers (4 x 128 columns = all 512)
constexpr int GEMM_QCAP = 24;         // queued candidates per query before a merge
constexpr int GEMM_QSTRIDE = GEMM_QCAP + 1;
constexpr uint32_t GEMM_TILE_BYTES = 128u * 128u;  // one 128-row x 128-byte box

template <int KIND>
struct KindTraits;
// EPI: epilogue warpgroups.  The one-pass kinds finish a tile's MMAs three times faster,
// so two warpgroups (each owning half of the tile's columns, with separate candidate
// lists) keep the selection ahead of the tensor core; TF32X3 has no shared memory to spare.
template <>
struct KindTraits<KIND_TF32X3> {
  static constexpr int ELEM = 4, PIECES = 2, EPI = 1;
  static constexpr uint32_t FMT = sm100::FMT_TF32;
};
template <>
struct KindTraits<KIND_BF16> {
  static constexpr int ELEM = 2, PIECES = 1, EPI = 2;
  static constexpr uint32_t FMT = sm100::FMT_BF16;
};
template <>
struct KindTraits<KIND_FP8> {
  static constexpr int ELEM = 1, PIECES = 1, EPI = 2;
  static constexpr uint32_t FMT = sm100::FMT_E4M3;
};
template <>
struct KindTraits<KIND_FP16X3> {
  static constexpr int ELEM = 2, PIECES = 2, EPI = 2;
  static constexpr uint32_t FMT = sm100::FMT_F16;
};
__host__ __device__ constexpr int gemm_threads(int epi) { return 96 + 128 * epi; }
// Kernel kind of a public precision: float32 accuracy comes from the FP16 split (the
// faster of the two float32-accurate kinds), GBK_PREC_TF32X3 asks for the TF32 split.
__host__ __device__ constexpr int gemm_kind(int prec) {
  return prec == GBK_PREC_FP32     ? KIND_FP16X3
         : prec == GBK_PREC_TF32X3 ? KIND_TF32X3
         : prec == GBK_PREC_BF16   ? KIND_BF16
                                   : KIND_FP8;
}
__host__ __device__ constexpr int gemm_epi(int prec) {
  return gemm_kind(prec) == KIND_TF32X3 ? 1 : 2;
}

struct GemmArgs {
  int nq, nb;            // queries, database rows
  int nkb;               // 128-byte k-blocks per row (padded d)
  int stages;            // ring depth
  int dual;              // two MMA issuers on alternate tiles (requires stages >= 2 nkb)
  int tmem_a;            // A tile in tensor memory (copied from one staging k-block) instead
                         // of shared memory, freeing shared memory for the ring
  int nacc;              // accumulator buffers: 4, or 2-3 with tmem_a
  int stream_a;          // 1: the query tile's k-blocks travel with B's through the ring
                         // (rows too long to keep the query tile resident)
  int nqt, ntiles;       // query tiles, database tiles
  int chunks, tpc;       // database chunks, tiles per chunk
  int k, kp;             // k and the padded list length (power of two >= 32)
  const float* ynorm;    // [ntiles*128] ||y||^2 (padding rows arbitrary)
  const float* xnorm;    // STORE: [nq] ||x||^2 added (and the sum clamped at 0), or null
  const float* qscale;   // [nq] per-query dequantisation scale (FP8), else null
  const float* bscale;   // [ntiles*128] per-row database scale (FP8), else null
  uint64_t* part;        // SELECT: [nq][part_lists][kp] sorted composite lists; this launch
                         // uses lists [list0, list0 + chunks * EPI)
  int part_lists, list0; // part_lists 0: chunks * EPI
  int64_t row0;          // added to the database row numbers stored in the lists
  uint32_t* thr_key;     // SELECT: [nq] global threshold keys (init 0xffffffff)
  float* out;            // STORE: [nq][ldo] partial distances; tile_min: [nq][ldo] minima
  int64_t ldo;
  int tile_min;          // SELECT, k = 1: out[q * ldo + tile * EPI + half] = the best value of
                         // each (query, tile, column half) instead of one arg-best per list
  int hi_only;           // split kinds: one MMA pass over the high pieces (hi x hi) instead of
                         // three, and only B's high piece loaded (the threshold pre-pass)
  uint32_t* status;
};

// ------------------------------------------------------------------ warp helpers

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
  return __shfl_sync(FULL_MASK, v, src);
}
__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
  return __shfl_xor_sync(FULL_MASK, v, m);
}

// Ascending bitonic sort of one value per lane.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const uint64_t o = shfl_xor64(v, stride);
      const bool asc = (lane & size) == 0 || size == 32;
      const bool lower = (lane & stride) == 0;
      v = (lower == asc) ? min(v, o) : max(v, o);
    }
  }
  return v;
}

// L (KPR*32 sorted composites, lane-stride: element 32r+lane in L[r]) <- the KPR*32
// smallest of L U Q, where Q holds one sorted value per lane.  Reversed Q against the
// last 32 of L (half-cleaner) leaves a bitonic sequence holding exactly the smallest
// elements; a bitonic merge sorts it.
template <int KPR>
__device__ __forceinline__ void warp_merge_list(uint64_t (&L)[KPR], uint64_t q_sorted) {
  const int lane = threadIdx.x & 31;
  const uint64_t qrev = shfl64(q_sorted, 31 - lane);
  L[KPR - 1] = min(L[KPR - 1], qrev);
  constexpr int LOGK = KPR >= 16 ? 4 : KPR >= 8 ? 3 : KPR >= 4 ? 2 : KPR >= 2 ? 1 : 0;
#pragma unroll
  for (int ls = LOGK - 1; ls >= 0; ls--) {  // strides >= 32: within a lane
    const int s = 1 << ls;
#pragma unroll
    for (int r = 0; r < KPR; r++) {
      if ((r & s) == 0) {
        const uint64_t a = L[r], b = L[r + s];
        L[r] = min(a, b);
        L[r + s] = max(a, b);
      }
    }
  }
#pragma unroll
  for (int stride = 16; stride >= 1; stride >>= 1) {  // strides < 32: across lanes
    const bool lower = (lane & stride) == 0;
#pragma unroll
    for (int r = 0; r < KPR; r++) {
      const uint64_t o = shfl_xor64(L[r], stride);
      L[r] = lower ? min(L[r], o) : max(L[r], o);
    }
  }
}

// ------------------------------------------------------------------ operand prep

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x[n][d] -> hi, lo [n][dpad] (TF32-rounded pieces, zero padded), norms[n] = ||x||^2
// (float32, fixed order), one warp per row.  Rows in [n, nrows_pad) of `norms` get
// pad_norm.
__global__ void prep_tf32x3_kernel(const float* __restrict__ x, int64_t n, int d, int dpad,
                                   float* __restrict__ hi, float* __restrict__ lo,
                                   float* __restrict__ norms, int64_t nrows_pad,
                                   float pad_norm);
// x -> bf16 [n][dpad], norms from the float32 input.
__global__ void prep_bf16_kernel(const float* __restrict__ x, int64_t n, int d, int dpad,
                                 __nv_bfloat16* __restrict__ out, float* __restrict__ norms,
                                 int64_t nrows_pad, float pad_norm);
// x -> fp16 hi, lo [n][dpad] of x / s with the per-row power of two s >= max|x|, scale[n]
// = s, norms from the float32 input.
__global__ void prep_fp16x3_kernel(const float* __restrict__ x, int64_t n, int d, int dpad,
                                   __half* __restrict__ hi, __half* __restrict__ lo,
                                   float* __restrict__ scale, float* __restrict__ norms,
                                   int64_t nrows_pad, float pad_norm);
// x -> e4m3 [n][dpad] with a per-row scale s = max|x| / 448 (x ~ s * q), norms.
__global__ void prep_fp8_kernel(const float* __restrict__ x, int64_t n, int d, int dpad,
                                __nv_fp8_e4m3* __restrict__ out, float* __restrict__ scale,
                                float* __restrict__ norms, int64_t nrows_pad, float pad_norm);

}  // namespace gbk
