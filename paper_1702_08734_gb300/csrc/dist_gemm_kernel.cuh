// Kernel template of the fused distance GEMM (see dist_gemm.cuh for the design).
// Included once per precision by dist_gemm_<kind>.cu.
#pragma once
#include "dist_gemm.cuh"

namespace gbk {

struct GemmSmemLayout {
  uint32_t a_off, b_off, q_off, bar_off, total;
};

// Offsets relative to a 1024-byte aligned base (TMA 128B-swizzle tiles need it).
__host__ __device__ inline GemmSmemLayout gemm_smem_layout(int pieces, int nkb, int stages,
                                                           bool queues) {
  GemmSmemLayout L;
  L.a_off = 0;
  L.b_off = L.a_off + (uint32_t)pieces * nkb * GEMM_TILE_BYTES;
  L.q_off = L.b_off + (uint32_t)stages * pieces * GEMM_TILE_BYTES;
  const uint32_t qbytes = queues ? (uint32_t)(GEMM_BM * GEMM_QSTRIDE * 8) : 0u;
  L.bar_off = (L.q_off + qbytes + 63u) & ~63u;
  L.total = L.bar_off + 8u * (2u + 2u * (uint32_t)stages + 4u) + 16u;
  return L;
}

// KPR: candidate list length / 32 (SELECT with k > 1); KPR == 0 with MODE_SELECT is the
// k = 1 arg-min path (no lists).  MODE_STORE writes the partial distances instead.
template <int KIND, int MODE, int KPR, bool LARGEST>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    dist_gemm_kernel(const __grid_constant__ CUtensorMap tmA0,
                     const __grid_constant__ CUtensorMap tmA1,
                     const __grid_constant__ CUtensorMap tmB0,
                     const __grid_constant__ CUtensorMap tmB1, const GemmArgs args) {
  using T = KindTraits<KIND>;
  constexpr int PIECES = T::PIECES;
  constexpr bool QUEUES = (MODE == MODE_SELECT) && (KPR > 0);
  constexpr uint32_t IDESC = sm100::idesc_f32acc(T::FMT, GEMM_BM, GEMM_BN);
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  const GemmSmemLayout lay = gemm_smem_layout(PIECES, args.nkb, args.stages, QUEUES);
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
      sm100::mbar_init(&acc_empty[i], 4);
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
    const int quarter = warp & 3;
    const int qrow = quarter * 32 + lane;  // TMEM lane == query row in the tile
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint64_t* myQ = sQ + qrow * GEMM_QSTRIDE;
    uint32_t gtile = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int qt = item % args.nqt, ch = item / args.nqt;
      const int t0 = ch * args.tpc, t1 = min(args.ntiles, t0 + args.tpc);
      const int q = qt * GEMM_BM + qrow;
      const bool qvalid = q < args.nq;
      const float qs = (KIND == KIND_FP8 && qvalid) ? args.qscale[q] : 1.f;
      const float xn_store = (MODE == MODE_STORE && args.xnorm && qvalid) ? args.xnorm[q] : -1.f;
      ValueFilter f;
      int cnt = 0;
      uint64_t best = ~0ull;  // k = 1 path
      if (MODE == MODE_SELECT) {
        f.set(qvalid ? args.thr_key[q] : NAN_KEY, LARGEST);
        if (QUEUES) {
          // reset this warp's 32 lists for this chunk
          for (int j = 0; j < 32; j++) {
            const int qq = qt * GEMM_BM + quarter * 32 + j;
            if (qq < args.nq) {
              uint64_t* Lg = args.part + ((int64_t)qq * args.chunks + ch) * args.kp;
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
          while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const int n = __shfl_sync(FULL_MASK, cnt, l);
            const int ql = quarter * 32 + l;
            const int qq = qt * GEMM_BM + ql;
            uint64_t v = lane < n ? sQ[ql * GEMM_QSTRIDE + lane] : ~0ull;
            v = warp_sort32(v);
            uint64_t* Lg = args.part + ((int64_t)qq * args.chunks + ch) * args.kp;
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
              if (tk != ~0ull) f.set((uint32_t)(tk >> 32), LARGEST);
            }
          }
          __syncwarp();
        }
      };
      for (int t = t0; t < t1; t++, gtile++) {
        const int acc = (int)(gtile & 1u);
        ok = sm100::mbar_wait(&acc_full[acc], (gtile >> 1) & 1u, args.status, abort_flag);
        if (!ok) break;
        sm100::tc_fence_after();
        const int col0 = t * GEMM_BN;
        const int lim = args.nb - col0;  // valid columns in this tile
        const uint32_t taddr = tmem_base + lane_addr + (uint32_t)(acc * GEMM_BN);
#pragma unroll 1
        for (int c = 0; c < GEMM_BN / 16; c++) {
          uint32_t r[16];
          sm100::tmem_ld_x16(taddr + (uint32_t)(c * 16), r);
          sm100::tmem_wait_ld();
          if (c == GEMM_BN / 16 - 1) {
            sm100::tc_fence_before();
            __syncwarp();
            if (lane == 0) sm100::mbar_arrive(&acc_empty[acc]);
          }
          const float4* yn4 = reinterpret_cast<const float4*>(args.ynorm + col0 + c * 16);
          float yn[16];
#pragma unroll
          for (int j4 = 0; j4 < 4; j4++) {
            const float4 y = __ldg(yn4 + j4);
            yn[j4 * 4 + 0] = y.x;
            yn[j4 * 4 + 1] = y.y;
            yn[j4 * 4 + 2] = y.z;
            yn[j4 * 4 + 3] = y.w;
          }
          float bs[16];
          if (KIND == KIND_FP8) {
            const float4* bs4 = reinterpret_cast<const float4*>(args.bscale + col0 + c * 16);
#pragma unroll
            for (int j4 = 0; j4 < 4; j4++) {
              const float4 y = __ldg(bs4 + j4);
              bs[j4 * 4 + 0] = y.x * qs;
              bs[j4 * 4 + 1] = y.y * qs;
              bs[j4 * 4 + 2] = y.z * qs;
              bs[j4 * 4 + 3] = y.w * qs;
            }
          }
#pragma unroll
          for (int j = 0; j < 16; j++) {
            float ip = __uint_as_float(r[j]);
            if (KIND == KIND_FP8) ip *= bs[j];
            const float dist = LARGEST ? ip : fmaf(-2.f, ip, yn[j]);
            const int cj = c * 16 + j;
            if (MODE == MODE_STORE) {
              if (qvalid && cj < lim)
                args.out[(int64_t)q * args.ldo + col0 + cj] = xn_store >= 0.f ? fmaxf(dist + xn_store, 0.f) : dist;
            } else if (!QUEUES) {
              if (qvalid && cj < lim) {
                const uint64_t e = composite(ordered_key(dist, LARGEST), (uint32_t)(col0 + cj));
                best = min(best, e);
              }
            } else {
              if (qvalid && cj < lim && f.pass(dist))
                myQ[cnt++] = composite(ordered_key(dist, LARGEST), (uint32_t)(col0 + cj));
            }
          }
          if (QUEUES) merge_queues(GEMM_QCAP - 16);
        }
      }
      if (!ok) break;
      if (MODE == MODE_SELECT) {
        if (QUEUES) {
          merge_queues(0);
          // publish this chunk's k-th distance as an upper bound for later chunks
          if (qvalid) {
            const uint64_t* Lg = args.part + ((int64_t)q * args.chunks + ch) * args.kp;
            const uint64_t tk = Lg[args.k - 1];
            if (tk != ~0ull) atomicMin(&args.thr_key[q], (uint32_t)(tk >> 32));
          }
        } else if (qvalid) {
          args.part[(int64_t)q * args.chunks + ch] = best;
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
