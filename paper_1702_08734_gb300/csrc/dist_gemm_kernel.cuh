// Kernel template of the fused distance GEMM (see dist_gemm.cuh for the design).
// Included once per precision by dist_gemm_<kind>.cu.
#pragma once
#include "dist_gemm.cuh"

namespace gbk {

struct GemmSmemLayout {
  uint32_t a_off, b_off, q_off, y_off, h_off, bar_off, total;
};

// Offsets relative to a 1024-byte aligned base (TMA 128B-swizzle tiles need it).  Per
// epilogue warp a 1 KB slice stages the tile's database norms (and row scales); with two
// column halves keeping lists, one 8-byte half-list key per (half, query row) follows.
__host__ __device__ inline GemmSmemLayout gemm_smem_layout(int pieces, int nkb, int stages,
                                                           bool queues, int epi) {
  GemmSmemLayout L;
  L.a_off = 0;
  L.b_off = L.a_off + (uint32_t)pieces * nkb * GEMM_TILE_BYTES;
  L.q_off = L.b_off + (uint32_t)stages * pieces * GEMM_TILE_BYTES;
  const uint32_t qbytes = queues ? (uint32_t)(epi * GEMM_BM * GEMM_QSTRIDE * 8) : 0u;
  L.y_off = (L.q_off + qbytes + 15u) & ~15u;
  L.h_off = L.y_off + (uint32_t)(epi * 4 * 1024);
  const uint32_t hbytes = (queues && epi == 2) ? 2u * GEMM_BM * 8u : 0u;
  L.bar_off = (L.h_off + hbytes + 63u) & ~63u;
  L.total = L.bar_off + 8u * (4u + 2u * (uint32_t)stages + 2u * GEMM_NACC) + 16u;
  return L;
}

// Candidate lists live in global memory and are re-read by every merge; the streamed
// database would push them out of L2, so their accesses carry an evict-last policy.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t ld_keep(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ void st_keep(uint64_t* p, uint64_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

// Three-input min / max (sm_100 family); as with the two-input forms a NaN input is
// ignored unless every input is NaN.
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Best (smallest, or largest for LARGEST) of 32 values as a depth-4 tree; NaN only when
// all 32 are NaN.
template <bool LARGEST>
__device__ __forceinline__ float batch_best32(const float (&v)[32]) {
  float a[12];
#pragma unroll
  for (int i = 0; i < 10; i++)
    a[i] = LARGEST ? max3f(v[3 * i], v[3 * i + 1], v[3 * i + 2])
                   : min3f(v[3 * i], v[3 * i + 1], v[3 * i + 2]);
  a[10] = v[30];
  a[11] = v[31];
  float b[4];
#pragma unroll
  for (int i = 0; i < 4; i++)
    b[i] = LARGEST ? max3f(a[3 * i], a[3 * i + 1], a[3 * i + 2])
                   : min3f(a[3 * i], a[3 * i + 1], a[3 * i + 2]);
  const float c = LARGEST ? max3f(b[0], b[1], b[2]) : min3f(b[0], b[1], b[2]);
  return LARGEST ? fmaxf(c, b[3]) : fminf(c, b[3]);
}

// Threshold sharing between the candidate lists of one query.  Any value t with k values
// at or below it among the rows seen so far bounds the k-th nearest distance, so every
// list of the query may filter with it: the k-th value of any one list, or - for the two
// column halves of one tile, which see disjoint rows of the same chunk in lockstep - the
// worse of the two halves' ceil(k/2)-th values.  Bounds are published as ordered keys
// (smaller = better): to the query's global key (atomicMin; read by every list of the
// query once per tile) and, per half, to a shared-memory word tagged with the work item,
// so a half only pairs with the other half's list of the same query tile.
struct ThrShare {
  uint32_t* gthr;                  // the query's global key (null: row past nq)
  volatile uint64_t* hmine;        // this warp's 32 rows' {item, key} words (null: one half)
  const volatile uint64_t* hother; // the other half's words for the same rows
  uint32_t tag;                    // work item
  uint32_t own;                    // key of this lane's ceil(k/2)-th list value, or NAN_KEY
};

template <bool LARGEST>
__device__ __forceinline__ void tighten(float& thr, uint32_t key) {
  if (key == NAN_KEY) return;
  const float t = key_value(key, LARGEST);
  thr = LARGEST ? fmaxf(thr, t) : fminf(thr, t);
}

// Warp-cooperative merge of every lane's candidate queue holding more than `limit`
// entries into that lane's sorted list (queue of lane l: sQ[l * GEMM_QSTRIDE ...] as
// {value bits, column}; list of lane l at part + l * rowstride, KPR*32 composites).  The
// merging lane's threshold then tightens to its list's k-th value or the pair bound of
// the two halves, whichever is better, and that bound is published (ThrShare).
template <int KPR, bool LARGEST>
__device__ __forceinline__ void merge_queues(int limit, int& cnt, float& thr, const uint2* sQ,
                                             uint64_t* part, int64_t rowstride, int k,
                                             int quarter, int lane, uint64_t pol,
                                             ThrShare& ts) {
  if constexpr (KPR == 0) return;  // k = 1 keeps no lists
  constexpr int KR = KPR > 0 ? KPR : 1;
  unsigned m = __ballot_sync(FULL_MASK, cnt > limit);
  if (!m) return;
  __syncwarp();  // other lanes' queue writes are visible
  while (m) {
    const int l = __ffs(m) - 1;
    m &= m - 1;
    const int n = __shfl_sync(FULL_MASK, cnt, l);
    uint64_t v = ~0ull;
    if (lane < n) {
      const uint2 e = sQ[l * GEMM_QSTRIDE + lane];
      v = composite(ordered_key(__uint_as_float(e.x), LARGEST), e.y);
    }
    // the list's L2 round trip overlaps the queue's sort
    uint64_t* Lg = part + (int64_t)l * rowstride;
    uint64_t L[KR];
#pragma unroll
    for (int r = 0; r < KR; r++) L[r] = ld_keep(Lg + r * 32 + lane, pol);
    v = warp_sort32(v);
    warp_merge_list<KR>(L, v);
#pragma unroll
    for (int r = 0; r < KR; r++) st_keep(Lg + r * 32 + lane, L[r], pol);
    // new threshold: element k-1 of the list
    const int kk = k - 1;
    uint64_t tk = 0;
#pragma unroll
    for (int r = 0; r < KR; r++)  // masked OR, not an indexed read (keeps L in registers)
      tk |= L[r] & (0ull - (uint64_t)(r == (kk >> 5)));
    tk = shfl64(tk, kk & 31);
    uint64_t th = ~0ull;  // element ceil(k/2)-1 (only with two halves)
    if (ts.hmine) {
      const int kh = (k + 1) / 2 - 1;
      th = 0;
#pragma unroll
      for (int r = 0; r < KR; r++) th |= L[r] & (0ull - (uint64_t)(r == (kh >> 5)));
      th = shfl64(th, kh & 31);
    }
    if (lane == l) {
      cnt = 0;
      uint32_t best = tk != ~0ull ? (uint32_t)(tk >> 32) : NAN_KEY;
      if (th != ~0ull) {
        ts.own = (uint32_t)(th >> 32);
        ts.hmine[l] = ((uint64_t)ts.tag << 32) | ts.own;
        const uint64_t o = ts.hother[l];
        if ((uint32_t)(o >> 32) == ts.tag) best = min(best, max(ts.own, (uint32_t)o));
      }
      tighten<LARGEST>(thr, best);
      if (ts.gthr && best != NAN_KEY) atomicMin(ts.gthr, best);
    }
  }
  __syncwarp();
  (void)quarter;
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
  constexpr bool SCALED = (KIND == KIND_FP8 || KIND == KIND_FP16X3);  // per-row scales
  constexpr uint32_t IDESC = sm100::idesc_f32acc(T::FMT, GEMM_BM, GEMM_BN);
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  // stage = B's pieces, or A's and B's pieces of one k-block when A is streamed
  const int SP = args.stream_a ? 2 * PIECES : PIECES;
  // A in shared memory: all of its k-blocks (resident), none (streamed), or one staging
  // k-block on its way into tensor memory (tmem_a)
  const GemmSmemLayout lay =
      args.stream_a ? gemm_smem_layout(2 * PIECES, 0, args.stages, QUEUES, EPI)
                    : gemm_smem_layout(PIECES, args.tmem_a ? 1 : args.nkb, args.stages, QUEUES, EPI);
  const int nacc = args.nacc;  // accumulator buffers: 4, or fewer when A takes tensor memory
  unsigned char* sA = smem + lay.a_off;
  unsigned char* sB = smem + lay.b_off;
  uint64_t* sQ = reinterpret_cast<uint64_t*>(smem + lay.q_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint64_t* a_full = bars + 0;
  uint64_t* a_empty = bars + 1;
  uint64_t* b_full = bars + 2;
  uint64_t* b_empty = b_full + args.stages;
  uint64_t* acc_full = b_empty + args.stages;
  uint64_t* acc_empty = acc_full + GEMM_NACC;
  uint64_t* as_full = acc_empty + GEMM_NACC;  // A staging k-block (tmem_a)
  uint64_t* as_empty = as_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(as_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  constexpr bool PAIR = QUEUES && EPI == 2;  // the two column halves share a pair bound
  const bool hi_only = PIECES > 1 && args.hi_only != 0;  // one pass: high pieces only
  volatile uint64_t* sH = reinterpret_cast<volatile uint64_t*>(smem + lay.h_off);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = args.nqt * args.chunks;

  if (threadIdx.x == 0) {
    sm100::mbar_init(a_full, 1);
    sm100::mbar_init(a_empty, args.dual ? 2 : 1);  // one commit from each MMA issuer
    for (int i = 0; i < args.stages; i++) {
      sm100::mbar_init(&b_full[i], 1);
      sm100::mbar_init(&b_empty[i], 1);
    }
    for (int i = 0; i < GEMM_NACC; i++) {
      sm100::mbar_init(&acc_full[i], 1);
      sm100::mbar_init(&acc_empty[i], 4 * EPI);
    }
    sm100::mbar_init(as_full, 1);
    sm100::mbar_init(as_empty, 1);
    *abort_flag = 0;
    sm100::fence_mbar_init();
  }
  if (PAIR)  // no item has tag ~0: stale words never pair
    for (int i = threadIdx.x; i < 2 * GEMM_BM; i += blockDim.x) sH[i] = ~0ull;
  if (warp == 1) {
    sm100::tmem_alloc(tmem_slot, GEMM_NACC * GEMM_BN);
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
      // ring position kept incrementally (no division by the runtime stage count)
      int st = 0;
      uint32_t ph = 0;
      uint32_t as_use = 0;  // A staging slot uses (tmem_a)
      int local = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, local++) {
        const int qt = item % args.nqt, ch = item / args.nqt;
        const int t0 = ch * args.tpc, t1 = min(args.ntiles, t0 + args.tpc);
        if (args.tmem_a) {
          // A's k-blocks one at a time through the staging slot; the MMA thread copies
          // each into tensor memory
          for (int kb = 0; kb < args.nkb && ok; kb++, as_use++) {
            ok = sm100::mbar_wait(as_empty, (as_use & 1u) ^ 1u, args.status, abort_flag);
            if (!ok) break;
            sm100::mbar_arrive_expect_tx(as_full, (uint32_t)PIECES * GEMM_TILE_BYTES);
            const int x = kb * (128 / T::ELEM);
            sm100::tma_load_2d(sA, &tmA0, as_full, x, qt * GEMM_BM);
            if (PIECES > 1) sm100::tma_load_2d(sA + GEMM_TILE_BYTES, &tmA1, as_full, x, qt * GEMM_BM);
          }
          if (!ok) break;
        } else if (!args.stream_a) {
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
        }
        for (int t = t0; t < t1 && ok; t++) {
          for (int kb = 0; kb < args.nkb; kb++) {
            ok = sm100::mbar_wait(&b_empty[st], ph ^ 1u, args.status, abort_flag);
            if (!ok) break;
            sm100::mbar_arrive_expect_tx(&b_full[st], (uint32_t)(hi_only ? SP / PIECES : SP) *
                                                          GEMM_TILE_BYTES);
            const int x = kb * (128 / T::ELEM);
            unsigned char* dst = sB + (uint32_t)st * SP * GEMM_TILE_BYTES;
            if (args.stream_a) {
              sm100::tma_load_2d(dst, &tmA0, &b_full[st], x, qt * GEMM_BM);
              if (PIECES > 1 && !hi_only)
                sm100::tma_load_2d(dst + GEMM_TILE_BYTES, &tmA1, &b_full[st], x, qt * GEMM_BM);
              dst += PIECES * GEMM_TILE_BYTES;
            }
            sm100::tma_load_2d(dst, &tmB0, &b_full[st], x, t * GEMM_BN);
            if (PIECES > 1 && !hi_only)
              sm100::tma_load_2d(dst + GEMM_TILE_BYTES, &tmB1, &b_full[st], x, t * GEMM_BN);
            if (++st == args.stages) {
              st = 0;
              ph ^= 1u;
            }
          }
        }
      }
    }
  } else if (warp == 1 || warp == 2) {
    // ---------------------------------------------------------------- MMA issuers
    // With `dual`, two issuing threads in different warps take alternate tiles: the tensor
    // core keeps only a few MMAs queued, so while one thread waits for its next
    // accumulator buffer and operands (and does its bookkeeping) the other's MMAs keep the
    // pipe busy.  Each thread's commits track its own MMAs.  `dual` requires a ring of at
    // least two tiles (stages >= 2 nkb): a slot's previous fill then belongs to the same
    // thread's previous tile, which that thread has already waited for, so a parity wait
    // can never mistake an older phase for the one it needs.  The accumulator buffers need
    // no such condition for nacc >= 2: the issuer of tile g waited, for its previous tile
    // g - 2, until the epilogue had released tile g - 2 - nacc, so tile g - 2 nacc (the
    // older phase of tile g's buffer) is released too; buffer index and phase are counted
    // per tile, skipped tiles included.
    // With `tmem_a`, issuer 0 copies each work item's A tile from its staging k-block into
    // tensor memory (columns after the accumulators) once the previous item's MMAs of both
    // issuers are done, and both issuers read A from there.
    const uint32_t par = (uint32_t)(warp - 1);
    if (lane == 0 && (par == 0 || args.dual)) {
      // Ring position and phase are kept incrementally (the other thread's tiles skipped),
      // descriptors are formed once per k-block and stepped by 32 bytes of K (start address
      // field, >> 4), and TMA-filled operands need no tcgen05 fence after their mbarrier
      // waits (the fence orders an accumulator buffer after the epilogue's TMEM loads).
      uint32_t gtile = 0;
      int st = 0;
      uint32_t ph = 0;
      auto advance = [&](int n) {
        st += n;
        while (st >= args.stages) {
          st -= args.stages;
          ph ^= 1u;
        }
      };
      int acc_i = 0;  // accumulator buffer of tile gtile and its use parity
      uint32_t acc_ph = 0;
      auto next_acc = [&]() {
        if (++acc_i == nacc) {
          acc_i = 0;
          acc_ph ^= 1u;
        }
      };
      int local = 0;
      bool ok = true;
      const uint32_t a_base = sm100::smem_u32(sA), ring_base = sm100::smem_u32(sB);
      constexpr uint32_t TILE16 = GEMM_TILE_BYTES >> 4;  // one 128 x 128-byte box in desc units
      const uint32_t a_tm = tmem_base + (uint32_t)(nacc * GEMM_BN);  // A in tensor memory
      uint32_t as_use = 0;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, local++) {
        const int ch = item / args.nqt;
        const int t0 = ch * args.tpc, t1 = min(args.ntiles, t0 + args.tpc);
        if (args.tmem_a) {
          if (par == 0) {
            ok = sm100::mbar_wait(a_empty, (uint32_t)((local & 1) ^ 1), args.status, abort_flag);
            if (ok) sm100::tc_fence_after();
            for (int kb = 0; kb < args.nkb && ok; kb++, as_use++) {
              ok = sm100::mbar_wait(as_full, as_use & 1u, args.status, abort_flag);
              if (!ok) break;
              const uint64_t s0 = sm100::sdesc_k_sw128(a_base);
#pragma unroll
              for (int pc = 0; pc < PIECES; pc++)
#pragma unroll
                for (int ks = 0; ks < 4; ks++)
                  sm100::tmem_cp_128x256b(a_tm + (uint32_t)((pc * args.nkb + kb) * 32 + ks * 8),
                                          s0 + (uint64_t)(pc * TILE16 + ks * 2));
              sm100::mma_commit(as_empty);  // the staging k-block is free once copied
            }
            if (ok) sm100::mma_commit(a_full);
          }
          if (ok) ok = sm100::mbar_wait(a_full, (uint32_t)(local & 1), args.status, abort_flag);
          if (!ok) break;
          sm100::tc_fence_after();
        } else if (!args.stream_a) {
          ok = sm100::mbar_wait(a_full, (uint32_t)(local & 1), args.status, abort_flag);
          if (!ok) break;
        }
        for (int t = t0; t < t1 && ok; t++, gtile++, next_acc()) {
          if (args.dual && (gtile & 1u) != par) {  // the other issuer's tile
            advance(args.nkb);
            continue;
          }
          const int acc = acc_i;
          ok = sm100::mbar_wait(&acc_empty[acc], acc_ph ^ 1u, args.status, abort_flag);
          if (!ok) break;
          sm100::tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * GEMM_BN);
          for (int kb = 0; kb < args.nkb; kb++) {
            ok = sm100::mbar_wait(&b_full[st], ph, args.status, abort_flag);
            if (!ok) break;
            const uint32_t s_base = ring_base + (uint32_t)st * SP * GEMM_TILE_BYTES;
            // A piece 0 / piece 1 and B piece 0 / piece 1 of this k-block
            const uint64_t a0 = sm100::sdesc_k_sw128(args.stream_a ? s_base
                                                                   : a_base + kb * GEMM_TILE_BYTES);
            const uint64_t a1 = args.stream_a ? a0 + TILE16 : a0 + (uint64_t)args.nkb * TILE16;
            const uint64_t b0 = args.stream_a ? a0 + PIECES * TILE16 : sm100::sdesc_k_sw128(s_base);
            const uint64_t b1 = b0 + TILE16;
            const uint32_t at0 = a_tm + (uint32_t)(kb * 32);  // tmem_a: A pieces of this k-block
            const uint32_t at1 = at0 + (uint32_t)(args.nkb * 32);
            if (args.tmem_a) {
#pragma unroll
              for (int ks = 0; ks < 4; ks++) {
                const uint64_t ko = (uint64_t)(ks * 2);
                const uint32_t ka = (uint32_t)(ks * 8);
                const uint32_t accum = (kb | ks) != 0 ? 1u : 0u;
                if (KIND == KIND_TF32X3) {
                  sm100::mma_tf32_ts(d_tmem, at0 + ka, b0 + ko, IDESC, accum);
                  if (!hi_only) {
                    sm100::mma_tf32_ts(d_tmem, at0 + ka, b1 + ko, IDESC, 1u);
                    sm100::mma_tf32_ts(d_tmem, at1 + ka, b0 + ko, IDESC, 1u);
                  }
                } else if (KIND == KIND_FP16X3) {
                  sm100::mma_f16_ts(d_tmem, at0 + ka, b0 + ko, IDESC, accum);
                  if (!hi_only) {
                    sm100::mma_f16_ts(d_tmem, at0 + ka, b1 + ko, IDESC, 1u);
                    sm100::mma_f16_ts(d_tmem, at1 + ka, b0 + ko, IDESC, 1u);
                  }
                } else if (KIND == KIND_BF16) {
                  sm100::mma_f16_ts(d_tmem, at0 + ka, b0 + ko, IDESC, accum);
                } else {
                  sm100::mma_f8_ts(d_tmem, at0 + ka, b0 + ko, IDESC, accum);
                }
              }
            } else
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {  // 32 bytes of K per MMA
              const uint64_t ko = (uint64_t)(ks * 2);
              const uint32_t accum = (kb | ks) != 0 ? 1u : 0u;
              if (KIND == KIND_TF32X3) {
                sm100::mma_tf32(d_tmem, a0 + ko, b0 + ko, IDESC, accum);
                if (!hi_only) {
                  sm100::mma_tf32(d_tmem, a0 + ko, b1 + ko, IDESC, 1u);
                  sm100::mma_tf32(d_tmem, a1 + ko, b0 + ko, IDESC, 1u);
                }
              } else if (KIND == KIND_FP16X3) {
                sm100::mma_f16(d_tmem, a0 + ko, b0 + ko, IDESC, accum);
                if (!hi_only) {
                  sm100::mma_f16(d_tmem, a0 + ko, b1 + ko, IDESC, 1u);
                  sm100::mma_f16(d_tmem, a1 + ko, b0 + ko, IDESC, 1u);
                }
              } else if (KIND == KIND_BF16) {
                sm100::mma_f16(d_tmem, a0 + ko, b0 + ko, IDESC, accum);
              } else {
                sm100::mma_f8(d_tmem, a0 + ko, b0 + ko, IDESC, accum);
              }
            }
            sm100::mma_commit(&b_empty[st]);  // frees the ring stage once read
            advance(1);
          }
          if (ok) sm100::mma_commit(&acc_full[acc]);
        }
        if (ok && !args.stream_a) sm100::mma_commit(a_empty);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int quarter = warp & 3;          // TMEM lane quarter this warp may access
    const int half = (warp - 3) >> 2;      // column part of the tile (EPI parts)
    constexpr int CW = GEMM_BN / EPI;      // columns per warp per tile
    const int co = half * CW;
    const int qrow = quarter * 32 + lane;  // TMEM lane == query row in the tile
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint64_t* myQ = sQ + (half * GEMM_BM + qrow) * GEMM_QSTRIDE;
    float* sY = reinterpret_cast<float*>(smem + lay.y_off) + (warp - 3) * 256;  // norms, scales
    // candidate lists per query (this launch's start at list0 when several launches, one
    // per database piece, share the buffer)
    const int lists = args.part_lists ? args.part_lists : args.chunks * EPI;
    const int list0 = args.list0;
    const uint64_t lpol = l2_keep_policy();
    const bool vec_out = MODE == MODE_STORE && (args.ldo & 3) == 0 &&
                         (reinterpret_cast<uintptr_t>(args.out) & 15) == 0;
    uint32_t gtile = 0;
    int acc_i = 0;  // accumulator buffer of tile gtile and its use parity
    uint32_t acc_ph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int qt = item % args.nqt, ch = item / args.nqt;
      const int t0 = ch * args.tpc, t1 = min(args.ntiles, t0 + args.tpc);
      const int q = qt * GEMM_BM + qrow;
      const bool qvalid = q < args.nq;
      const float qs = (SCALED && qvalid) ? args.qscale[q] : 1.f;
      const float m2 = -2.f * qs;  // L2: ||y||^2 - 2 <x, y>, the query's row scale folded in
      const float xn_store = (MODE == MODE_STORE && args.xnorm && qvalid) ? args.xnorm[q] : -1.f;
      // Value-space threshold: keep dist <= thr (L2) or dist >= thr (inner product).  An
      // empty list passes every (finite) value; rows past nq get one that nothing passes.
      const float PASS_ALL = LARGEST ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000);
      float thr = PASS_ALL;
      int cnt = 0;
      float bestd = PASS_ALL;  // k = 1: running best; a strict improvement keeps the lowest column
      int besti = -1;
      uint32_t* const gthr = (QUEUES && qvalid) ? args.thr_key + q : nullptr;
      ThrShare ts;
      ts.gthr = gthr;
      ts.hmine = PAIR ? sH + half * GEMM_BM + quarter * 32 : nullptr;
      ts.hother = PAIR ? sH + (1 - half) * GEMM_BM + quarter * 32 : nullptr;
      ts.tag = (uint32_t)item;
      ts.own = NAN_KEY;
      if (MODE == MODE_SELECT) {
        if (!qvalid) {
          thr = -PASS_ALL;
        } else if (QUEUES) {  // (the k = 1 and tile-minimum launches carry no keys)
          const uint32_t tk = args.thr_key[q];
          thr = tk == NAN_KEY ? PASS_ALL : key_value(tk, LARGEST);
        }
        if (QUEUES) {
          // reset this warp's 32 lists for this chunk
          for (int j = 0; j < 32; j++) {
            const int qq = qt * GEMM_BM + quarter * 32 + j;
            if (qq < args.nq) {
              uint64_t* Lg = args.part + ((int64_t)qq * lists + list0 + ch * EPI + half) * args.kp;
              for (int r = lane; r < args.kp; r += 32) st_keep(Lg + r, ~0ull, lpol);
            }
          }
          __syncwarp();
        }
      }
      // lists of this warp's 32 queries (lane l: pbase + l * rowstride) and their queues
      const int64_t rowstride = (int64_t)lists * args.kp;
      uint64_t* pbase =
          QUEUES ? args.part + ((int64_t)(qt * GEMM_BM + quarter * 32) * lists + list0 + ch * EPI + half) *
                                   args.kp
                 : nullptr;
      const uint2* sQh = reinterpret_cast<const uint2*>(sQ + (half * GEMM_BM + quarter * 32) * GEMM_QSTRIDE);
      // Database norms (and FP8 scales) of this warp's part of a tile, fetched one tile
      // ahead into registers so the global-load latency hides behind a tile of work, then
      // staged in shared memory (the values are the same for the warp's 32 rows).
      float4 pre_y = make_float4(0.f, 0.f, 0.f, 0.f), pre_s = pre_y;
      uint32_t pre_g = NAN_KEY;  // the query's global threshold key, read a tile ahead
      auto prefetch = [&](int t) {
        if (QUEUES && gthr) pre_g = __ldcg(gthr);
        if (lane < CW / 4) {
          if (!LARGEST)
            pre_y = __ldg(reinterpret_cast<const float4*>(args.ynorm + t * GEMM_BN + co) + lane);
          if (SCALED)  // the row scale is applied below
            pre_s = __ldg(reinterpret_cast<const float4*>(args.bscale + t * GEMM_BN + co) + lane);
        }
      };
      if (t0 < t1) prefetch(t0);
      for (int t = t0; t < t1; t++, gtile++) {
        const int acc = acc_i;
        const uint32_t accph = acc_ph;
        if (++acc_i == nacc) {
          acc_i = 0;
          acc_ph ^= 1u;
        }
        const int col0 = t * GEMM_BN + co;  // first column of this warp's part
        __syncwarp();
        if (lane < CW / 4) {
          if (!LARGEST) reinterpret_cast<float4*>(sY)[lane] = pre_y;
          if (SCALED) reinterpret_cast<float4*>(sY + 128)[lane] = pre_s;
        }
        __syncwarp();
        if (QUEUES) {
          tighten<LARGEST>(thr, pre_g);  // lists of other chunks / halves of this query
          if (PAIR && ts.own != NAN_KEY) {  // this tile's other half
            const uint64_t o = ts.hother[lane];
            if ((uint32_t)(o >> 32) == ts.tag) tighten<LARGEST>(thr, max(ts.own, (uint32_t)o));
          }
        }
        if (t + 1 < t1) prefetch(t + 1);
        ok = sm100::mbar_wait(&acc_full[acc], accph, args.status, abort_flag);
        if (!ok) break;
        sm100::tc_fence_after();
        const int lim = args.nb - col0;  // valid columns in this part (warp-uniform)
        const uint32_t taddr = tmem_base + lane_addr + (uint32_t)(acc * GEMM_BN + co);
        // One batch = 32 accumulator columns of this lane's row, already in registers.
        auto batch = [&](float (&dist)[32], const int cb) {
          const int cbase = col0 + cb;  // database row of dist[0]
          // (paired float32 operations: each element rounded as by its scalar form)
          if (SCALED) {
            const float4* bs4 = reinterpret_cast<const float4*>(sY + 128 + cb);
#pragma unroll
            for (int j4 = 0; j4 < 8; j4++) {
              const float4 y = bs4[j4];
              const float2 lo = __fmul2_rn(make_float2(dist[j4 * 4 + 0], dist[j4 * 4 + 1]),
                                           make_float2(y.x, y.y));
              const float2 hi = __fmul2_rn(make_float2(dist[j4 * 4 + 2], dist[j4 * 4 + 3]),
                                           make_float2(y.z, y.w));
              dist[j4 * 4 + 0] = lo.x;
              dist[j4 * 4 + 1] = lo.y;
              dist[j4 * 4 + 2] = hi.x;
              dist[j4 * 4 + 3] = hi.y;
            }
          }
          if (!LARGEST) {
            const float4* yn4 = reinterpret_cast<const float4*>(sY + cb);
            const float2 mm = make_float2(m2, m2);
#pragma unroll
            for (int j4 = 0; j4 < 8; j4++) {
              const float4 y = yn4[j4];
              const float2 lo = __ffma2_rn(mm, make_float2(dist[j4 * 4 + 0], dist[j4 * 4 + 1]),
                                           make_float2(y.x, y.y));
              const float2 hi = __ffma2_rn(mm, make_float2(dist[j4 * 4 + 2], dist[j4 * 4 + 3]),
                                           make_float2(y.z, y.w));
              dist[j4 * 4 + 0] = lo.x;
              dist[j4 * 4 + 1] = lo.y;
              dist[j4 * 4 + 2] = hi.x;
              dist[j4 * 4 + 3] = hi.y;
            }
          } else if (SCALED) {
            const float2 qq = make_float2(qs, qs);
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              const float2 r = __fmul2_rn(make_float2(dist[j], dist[j + 1]), qq);
              dist[j] = r.x;
              dist[j + 1] = r.y;
            }
          }
          const bool ragged = lim < cb + 32;  // columns past nb in this batch (last tile only)
          if (MODE == MODE_STORE) {
            if (qvalid) {
              if (xn_store >= 0.f) {
#pragma unroll
                for (int j = 0; j < 32; j++) dist[j] = fmaxf(dist[j] + xn_store, 0.f);
              }
              float* orow = args.out + (int64_t)q * args.ldo + cbase;
              if (!ragged && vec_out) {  // 16-byte stores: 8 per batch instead of 32
#pragma unroll
                for (int j4 = 0; j4 < 8; j4++)
                  reinterpret_cast<float4*>(orow)[j4] =
                      make_float4(dist[4 * j4], dist[4 * j4 + 1], dist[4 * j4 + 2], dist[4 * j4 + 3]);
              } else {
#pragma unroll
                for (int j = 0; j < 32; j++)
                  if (!ragged || cb + j < lim) orow[j] = dist[j];
              }
            }
            return;
          }
          if (ragged) {  // past-the-end columns become NaN: they pass no threshold
#pragma unroll
            for (int j = 0; j < 32; j++)
              if (cb + j >= lim) dist[j] = __int_as_float(0x7fc00000);
          }
          // Fast path: the batch's best value (NaN ignored) decides whether any of its 32
          // values can enter; most batches end here once the threshold has settled.
          const float bm = batch_best32<LARGEST>(dist);
          if (!QUEUES && MODE == MODE_SELECT && args.tile_min) {
            // tile minima keep the value only (NaN ignored); the row search below would run
            // on every tile here, since the running best restarts with each tile
            bestd = LARGEST ? fmaxf(bestd, bm) : fminf(bestd, bm);
          } else if (!QUEUES) {
            const bool imp = LARGEST ? bm > bestd : bm < bestd;  // strict: earlier column wins ties
            if (__any_sync(FULL_MASK, imp) && imp) {
              int jj = 31;
#pragma unroll
              for (int j = 31; j >= 0; j--)
                if (dist[j] == bm) jj = j;  // lowest column holding the best value
              bestd = bm;
              besti = (int)args.row0 + cbase + jj;
            }
          } else {
            const bool any = LARGEST ? bm >= thr : bm <= thr;
            if (__any_sync(FULL_MASK, any)) {
              uint2* q2 = reinterpret_cast<uint2*>(myQ);
#pragma unroll
              for (int hf = 0; hf < 2; hf++) {
                if (any) {
#pragma unroll
                  for (int jj = 0; jj < 16; jj++) {
                    const float dv = dist[hf * 16 + jj];
                    if (LARGEST ? dv >= thr : dv <= thr)
                      q2[cnt++] = make_uint2(__float_as_uint(dv),
                                             (uint32_t)(args.row0 + cbase + hf * 16 + jj));
                  }
                }
                merge_queues<KPR, LARGEST>(GEMM_QCAP - 16, cnt, thr, sQh, pbase, rowstride,
                                           args.k, quarter, lane, lpol, ts);
              }
            }
          }
        };
        if constexpr (QUEUES) {
          // one batch at a time (the merge code stays out of line of a second copy), the
          // next batch's TMEM load in flight while this one is filtered
          uint32_t rb[32];
          sm100::tmem_ld_x32(taddr, rb);
#pragma unroll 1
          for (int b = 0; b < CW / 32; b++) {
            sm100::tmem_wait_ld();
            float d[32];
#pragma unroll
            for (int j = 0; j < 32; j++) d[j] = __uint_as_float(rb[j]);
            if (b + 1 < CW / 32) {
              sm100::tmem_ld_x32(taddr + (uint32_t)((b + 1) * 32), rb);
            } else {
              sm100::tc_fence_before();
              __syncwarp();
              if (lane == 0) sm100::mbar_arrive(&acc_empty[acc]);
            }
            batch(d, b * 32);
          }
        } else {
        // Two batches per TMEM wait; the accumulator buffer is handed back to the MMA warp
        // as soon as its last columns are in registers.
#pragma unroll 1
        for (int b = 0; b < CW / 64; b++) {
          uint32_t r0[32], r1[32];
          sm100::tmem_ld_x32(taddr + (uint32_t)(b * 64), r0);
          sm100::tmem_ld_x32(taddr + (uint32_t)(b * 64 + 32), r1);
          sm100::tmem_wait_ld();
          if (b + 1 == CW / 64) {
            sm100::tc_fence_before();
            __syncwarp();
            if (lane == 0) sm100::mbar_arrive(&acc_empty[acc]);
          }
          float d0[32], d1[32];
#pragma unroll
          for (int j = 0; j < 32; j++) {
            d0[j] = __uint_as_float(r0[j]);
            d1[j] = __uint_as_float(r1[j]);
          }
          batch(d0, b * 64);
          batch(d1, b * 64 + 32);
        }
        if (MODE == MODE_SELECT && args.tile_min) {
          if (qvalid) args.out[(int64_t)q * args.ldo + t * EPI + half] = bestd;
          bestd = PASS_ALL;
        }
        }
      }
      if (!ok) break;
      if (MODE == MODE_SELECT) {
        if (QUEUES) {
          // (every merge publishes its list's k-th value to the query's global threshold)
          merge_queues<KPR, LARGEST>(0, cnt, thr, sQh, pbase, rowstride, args.k, quarter, lane,
                                     lpol, ts);
        } else if (qvalid && !args.tile_min) {
          args.part[(int64_t)q * lists + list0 + ch * EPI + half] =
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
    sm100::tmem_dealloc(tmem_base, GEMM_NACC * GEMM_BN);
  }
}

}  // namespace gbk
