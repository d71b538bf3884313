// Kernel template of the fused distance GEMM (see dist_gemm.cuh for the design).
// Included once per precision by dist_gemm_<kind>.cu.
#pragma once
#include "dist_gemm.cuh"

namespace gbk {

struct GemmSmemLayout {
  uint32_t a_off, b_off, q_off, y_off, bar_off, total;
};

// Offsets relative to a 1024-byte aligned base (TMA 128B-swizzle tiles need it).  Per
// epilogue warp a 1 KB slice stages the tile's database norms (and FP8 scales).
__host__ __device__ inline GemmSmemLayout gemm_smem_layout(int pieces, int nkb, int stages,
                                                           bool queues, int epi) {
  GemmSmemLayout L;
  L.a_off = 0;
  L.b_off = L.a_off + (uint32_t)pieces * nkb * GEMM_TILE_BYTES;
  L.q_off = L.b_off + (uint32_t)stages * pieces * GEMM_TILE_BYTES;
  const uint32_t qbytes = queues ? (uint32_t)(epi * GEMM_BM * GEMM_QSTRIDE * 8) : 0u;
  L.y_off = (L.q_off + qbytes + 15u) & ~15u;
  L.bar_off = (L.y_off + (uint32_t)(epi * 4 * 1024) + 63u) & ~63u;
  L.total = L.bar_off + 8u * (2u + 2u * (uint32_t)stages + 4u) + 16u;
  return L;
}

// KPR: candidate list length / 32 (SELECT with k > 1); KPR == 0 with MODE_SELECT is the
// k = 1 arg-min path (no lists).  MODE_STORE writes the partial distances instead.
template <int KIND, int MODE, int KPR, bool LARGEST>
__global__ void __launch_bounds__(gemm_threads(KindTraits<KIND>::EPI), 1)
    dist_gemm_kernel(const __grid_constant__ CUtensorMap tmA0,
                     const __grid_constant__ CUtensorMap tmA1,
                     const __grid_constant__ CUtensorMap tmB0,
                     const __grid_constant__ CUtensorMap tmB1, const GemmArgs args) {
  using T = KindTraits<KIND>;
  constexpr int PIECES = T::PIECES;
  constexpr int EPI = T::EPI;
  constexpr bool QUEUES = (MODE == MODE_SELECT) && (KPR > 0);
  constexpr uint32_t IDESC = sm100::idesc_f32acc(T::FMT, GEMM_BM, GEMM_BN);
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  const GemmSmemLayout lay = gemm_smem_layout(PIECES, args.nkb, args.stages, QUEUES, EPI);
  unsigned char* sA = smem + lay.a_off;
  unsigned char* sB = smem + lay.b_off;
  uint64_t* sQ = reinterpret_cast<uint64_t*>(smem + lay.q_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint64_t* a_full = bars + 0;
  uint64_t* a_empty = bars + 1;
  uint64_t* b_full = bars + 2;
  uint64_t* b_empty = b_full + args.stages;
  uint64_t* acc_full = b_empty + args.stages;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = args.nqt * args.chunks;

  if (threadIdx.x == 0) {
    sm100::mbar_init(a_full, 1);
    sm100::mbar_init(a_empty, 1);
    for (int i = 0; i < args.stages; i++) {
      sm100::mbar_init(&b_full[i], 1);
      sm100::mbar_init(&b_empty[i], 1);
    }
    for (int i = 0; i < 2; i++) {
      sm100::mbar_init(&acc_full[i], 1);
      sm100::mbar_init(&acc_empty[i], 4 * EPI);
    }
    *abort_flag = 0;
    sm100::fence_mbar_init();
  }
  if (warp == 1) {
    sm100::tmem_alloc(tmem_slot, 2 * GEMM_BN);
    sm100::tmem_relinquish();
  }
  sm100::tc_fence_before();
  __syncthreads();
  sm100::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      sm100::tma_prefetch_desc(&tmA0);
      sm100::tma_prefetch_desc(&tmB0);
      if (PIECES > 1) {
        sm100::tma_prefetch_desc(&tmA1);
        sm100::tma_prefetch_desc(&tmB1);
      }
      uint32_t gstage = 0;
      int local = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, local++) {
        const int qt = item % args.nqt, ch = item / args.nqt;
        const int t0 = ch * args.tpc, t1 = min(args.ntiles, t0 + args.tpc);
        ok = sm100::mbar_wait(a_empty, (uint32_t)((local & 1) ^ 1), args.status, abort_flag);
        if (!ok) break;
        sm100::mbar_arrive_expect_tx(a_full, (uint32_t)(PIECES * args.nkb) * GEMM_TILE_BYTES);
        for (int kb = 0; kb < args.nkb; kb++) {
          const int x = kb * (128 / T::ELEM);
          sm100::tma_load_2d(sA + (0 * args.nkb + kb) * GEMM_TILE_BYTES, &tmA0, a_full, x,
                             qt * GEMM_BM);
          if (PIECES > 1)
            sm100::tma_load_2d(sA + (1 * args.nkb + kb) * GEMM_TILE_BYTES, &tmA1, a_full, x,
                               qt * GEMM_BM);
        }
        for (int t = t0; t < t1 && ok; t++) {
          for (int kb = 0; kb < args.nkb; kb++, gstage++) {
            const int st = (int)(gstage % args.stages);
            const uint32_t ph = (gstage / args.stages) & 1u;
            ok = sm100::mbar_wait(&b_empty[st], ph ^ 1u, args.status, abort_flag);
            if (!ok) break;
            sm100::mbar_arrive_expect_tx(&b_full[st], (uint32_t)PIECES * GEMM_TILE_BYTES);
            const int x = kb * (128 / T::ELEM);
            unsigned char* dst = sB + (uint32_t)st * PIECES * GEMM_TILE_BYTES;
            sm100::tma_load_2d(dst, &tmB0, &b_full[st], x, t * GEMM_BN);
            if (PIECES > 1)
              sm100::tma_load_2d(dst + GEMM_TILE_BYTES, &tmB1, &b_full[st], x, t * GEMM_BN);
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t gstage = 0, gtile = 0;
      int local = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, local++) {
        const int ch = item / args.nqt;
        const int t0 = ch * args.tpc, t1 = min(args.ntiles, t0 + args.tpc);
        ok = sm100::mbar_wait(a_full, (uint32_t)(local & 1), args.status, abort_flag);
        if (!ok) break;
        sm100::tc_fence_after();
        const uint32_t a_base = sm100::smem_u32(sA);
        for (int t = t0; t < t1 && ok; t++, gtile++) {
          const int acc = (int)(gtile & 1u);
          ok = sm100::mbar_wait(&acc_empty[acc], ((gtile >> 1) & 1u) ^ 1u, args.status,
                                abort_flag);
          if (!ok) break;
          sm100::tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * GEMM_BN);
          for (int kb = 0; kb < args.nkb; kb++, gstage++) {
            const int st = (int)(gstage % args.stages);
            ok = sm100::mbar_wait(&b_full[st], (gstage / args.stages) & 1u, args.status,
                                  abort_flag);
            if (!ok) break;
            sm100::tc_fence_after();
            const uint32_t b_base = sm100::smem_u32(sB) + (uint32_t)st * PIECES * GEMM_TILE_BYTES;
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {  // 32 bytes of K per MMA
              const uint32_t koff = (uint32_t)ks * 32u;
              const uint64_t a0 = sm100::sdesc_k_sw128(a_base + kb * GEMM_TILE_BYTES + koff);
              const uint64_t b0 = sm100::sdesc_k_sw128(b_base + koff);
              const uint32_t accum = (kb | ks) != 0 ? 1u : 0u;
              if (KIND == KIND_TF32X3) {
                const uint64_t a1 = sm100::sdesc_k_sw128(a_base +
                                                         (args.nkb + kb) * GEMM_TILE_BYTES + koff);
                const uint64_t b1 = sm100::sdesc_k_sw128(b_base + GEMM_TILE_BYTES + koff);
                sm100::mma_tf32(d_tmem, a0, b0, IDESC, accum);
                sm100::mma_tf32(d_tmem, a0, b1, IDESC, 1u);
                sm100::mma_tf32(d_tmem, a1, b0, IDESC, 1u);
              } else if (KIND == KIND_BF16) {
                sm100::mma_f16(d_tmem, a0, b0, IDESC, accum);
              } else {
                sm100::mma_f8(d_tmem, a0, b0, IDESC, accum);
              }
            }
            sm100::mma_commit(&b_empty[st]);  // frees the ring stage once read
          }
          if (ok) sm100::mma_commit(&acc_full[acc]);
        }
        if (ok) sm100::mma_commit(a_empty);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int quarter = warp & 3;          // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;      // column part of the tile (EPI parts)
    constexpr int CW = GEMM_BN / EPI;      // columns per warp per tile
    const int co = half * CW;
    const int qrow = quarter * 32 + lane;  // TMEM lane == query row in the tile
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint64_t* myQ = sQ + (half * GEMM_BM + qrow) * GEMM_QSTRIDE;
    float* sY = reinterpret_cast<float*>(smem + lay.y_off) + (warp - 2) * 256;  // norms, scales
    const int lists = args.chunks * EPI;   // candidate lists per query
    uint32_t gtile = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int qt = item % args.nqt, ch = item / args.nqt;
      const int t0 = ch * args.tpc, t1 = min(args.ntiles, t0 + args.tpc);
      const int q = qt * GEMM_BM + qrow;
      const bool qvalid = q < args.nq;
      const float qs = (KIND == KIND_FP8 && qvalid) ? args.qscale[q] : 1.f;
      const float m2 = -2.f * qs;  // L2: ||y||^2 - 2 <x, y>, FP8 row scale folded in
      const float xn_store = (MODE == MODE_STORE && args.xnorm && qvalid) ? args.xnorm[q] : -1.f;
      // Value-space threshold: keep dist <= thr (L2) or dist >= thr (inner product).  An
      // empty list passes every (finite) value; rows past nq get one that nothing passes.
      const float PASS_ALL = LARGEST ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000);
      float thr = PASS_ALL;
      int cnt = 0;
      float bestd = PASS_ALL;  // k = 1: running best; a strict improvement keeps the lowest column
      int besti = -1;
      if (MODE == MODE_SELECT) {
        if (!qvalid) {
          thr = -PASS_ALL;
        } else {
          const uint32_t tk = args.thr_key[q];
          thr = tk == NAN_KEY ? PASS_ALL : key_value(tk, LARGEST);
        }
        if (QUEUES) {
          // reset this warp's 32 lists for this chunk
          for (int j = 0; j < 32; j++) {
            const int qq = qt * GEMM_BM + quarter * 32 + j;
            if (qq < args.nq) {
              uint64_t* Lg = args.part + ((int64_t)qq * lists + ch * EPI + half) * args.kp;
              for (int r = lane; r < args.kp; r += 32) Lg[r] = ~0ull;
            }
          }
          __syncwarp();
        }
      }
      // warp-cooperative merge of every queue holding more than `limit` entries
      auto merge_queues = [&](int limit) {
        if constexpr (QUEUES) {
          unsigned m = __ballot_sync(FULL_MASK, cnt > limit);
          if (m) __syncwarp();  // other lanes' queue writes are visible
          while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const int n = __shfl_sync(FULL_MASK, cnt, l);
            const int ql = quarter * 32 + l;
            const int qq = qt * GEMM_BM + ql;
            uint64_t v = lane < n ? sQ[(half * GEMM_BM + ql) * GEMM_QSTRIDE + lane] : ~0ull;
            v = warp_sort32(v);
            uint64_t* Lg = args.part + ((int64_t)qq * lists + ch * EPI + half) * args.kp;
            uint64_t L[KPR];
#pragma unroll
            for (int r = 0; r < KPR; r++) L[r] = Lg[r * 32 + lane];
            warp_merge_list<KPR>(L, v);
#pragma unroll
            for (int r = 0; r < KPR; r++) Lg[r * 32 + lane] = L[r];
            // new threshold: element k-1 of the list
            const int kk = args.k - 1;
            uint64_t tk = 0;
#pragma unroll
            for (int r = 0; r < KPR; r++)
              if (r == (kk >> 5)) tk = L[r];
            tk = shfl64(tk, kk & 31);
            if (lane == l) {
              cnt = 0;
              if (tk != ~0ull) thr = key_value((uint32_t)(tk >> 32), LARGEST);
            }
          }
          __syncwarp();
        }
      };
      for (int t = t0; t < t1; t++, gtile++) {
        const int acc = (int)(gtile & 1u);
        const int col0 = t * GEMM_BN + co;  // first column of this warp's part
        // stage this part's database norms (and FP8 scales) while the MMAs run
        __syncwarp();
        if (lane < CW / 4) {
          if (!LARGEST)
            reinterpret_cast<float4*>(sY)[lane] =
                __ldg(reinterpret_cast<const float4*>(args.ynorm + col0) + lane);
          if (KIND == KIND_FP8)  // shared by the warp's rows: the row scale is applied below
            reinterpret_cast<float4*>(sY + 128)[lane] =
                __ldg(reinterpret_cast<const float4*>(args.bscale + col0) + lane);
        }
        __syncwarp();
        ok = sm100::mbar_wait(&acc_full[acc], (gtile >> 1) & 1u, args.status, abort_flag);
        if (!ok) break;
        sm100::tc_fence_after();
        const int lim = args.nb - col0;  // valid columns in this part
        const uint32_t taddr = tmem_base + lane_addr + (uint32_t)(acc * GEMM_BN + co);
        uint32_t rb[32];
        sm100::tmem_ld_x32(taddr, rb);
#pragma unroll 1
        for (int b = 0; b < CW / 32; b++) {
          sm100::tmem_wait_ld();
          float dist[32];
#pragma unroll
          for (int j = 0; j < 32; j++) dist[j] = __uint_as_float(rb[j]);
          if (b + 1 < CW / 32) {
            sm100::tmem_ld_x32(taddr + (uint32_t)((b + 1) * 32), rb);  // next batch in flight
          } else {
            sm100::tc_fence_before();
            __syncwarp();
            if (lane == 0) sm100::mbar_arrive(&acc_empty[acc]);
          }
          const int cb = b * 32;
          if (KIND == KIND_FP8) {
            const float4* bs4 = reinterpret_cast<const float4*>(sY + 128 + cb);
#pragma unroll
            for (int j4 = 0; j4 < 8; j4++) {
              const float4 y = bs4[j4];
              dist[j4 * 4 + 0] *= y.x;
              dist[j4 * 4 + 1] *= y.y;
              dist[j4 * 4 + 2] *= y.z;
              dist[j4 * 4 + 3] *= y.w;
            }
          }
          if (!LARGEST) {
            const float4* yn4 = reinterpret_cast<const float4*>(sY + cb);
#pragma unroll
            for (int j4 = 0; j4 < 8; j4++) {
              const float4 y = yn4[j4];
              dist[j4 * 4 + 0] = fmaf(m2, dist[j4 * 4 + 0], y.x);
              dist[j4 * 4 + 1] = fmaf(m2, dist[j4 * 4 + 1], y.y);
              dist[j4 * 4 + 2] = fmaf(m2, dist[j4 * 4 + 2], y.z);
              dist[j4 * 4 + 3] = fmaf(m2, dist[j4 * 4 + 3], y.w);
            }
          } else if (KIND == KIND_FP8) {
#pragma unroll
            for (int j = 0; j < 32; j++) dist[j] *= qs;
          }
          const uint32_t vm = lim >= cb + 32 ? 0xffffffffu : (lim <= cb ? 0u : ((1u << (lim - cb)) - 1u));
          if (MODE == MODE_STORE) {
            if (qvalid) {
#pragma unroll
              for (int j = 0; j < 32; j++)
                if ((vm >> j) & 1u)
                  args.out[(int64_t)q * args.ldo + col0 + cb + j] =
                      xn_store >= 0.f ? fmaxf(dist[j] + xn_store, 0.f) : dist[j];
            }
          } else if (!QUEUES) {
#pragma unroll
            for (int j = 0; j < 32; j++) {
              const bool better = LARGEST ? dist[j] > bestd : dist[j] < bestd;
              if (better && ((vm >> j) & 1u)) {
                bestd = dist[j];
                besti = col0 + cb + j;
              }
            }
          } else {
#pragma unroll
            for (int hf = 0; hf < 2; hf++) {
              uint32_t m = 0;
#pragma unroll
              for (int jj = 0; jj < 16; jj++) {
                const float dv = dist[hf * 16 + jj];
                m |= ((LARGEST ? dv >= thr : dv <= thr) ? 1u : 0u) << jj;
              }
              m &= (vm >> (hf * 16)) & 0xffffu;
              if (m) {
#pragma unroll
                for (int jj = 0; jj < 16; jj++)
                  if (m & (1u << jj))
                    myQ[cnt++] = composite(ordered_key(dist[hf * 16 + jj], LARGEST),
                                           (uint32_t)(col0 + cb + hf * 16 + jj));
              }
              merge_queues(GEMM_QCAP - 16);
            }
          }
        }
      }
      if (!ok) break;
      if (MODE == MODE_SELECT) {
        if (QUEUES) {
          merge_queues(0);
          // publish this chunk's k-th distance as an upper bound for later chunks
          if (qvalid) {
            const uint64_t* Lg = args.part + ((int64_t)q * lists + ch * EPI + half) * args.kp;
            const uint64_t tk = Lg[args.k - 1];
            if (tk != ~0ull) atomicMin(&args.thr_key[q], (uint32_t)(tk >> 32));
          }
        } else if (qvalid) {
          args.part[(int64_t)q * lists + ch * EPI + half] =
              besti >= 0 ? composite(ordered_key(bestd, LARGEST), (uint32_t)besti) : ~0ull;
        }
      }
    }
  }
  // ------------------------------------------------------------------ teardown
  sm100::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    sm100::tc_fence_after();
    sm100::tmem_dealloc(tmem_base, 2 * GEMM_BN);
  }
}

}  // namespace gbk
