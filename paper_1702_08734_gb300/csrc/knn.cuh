// Internal interface of the exact k-NN path (distance GEMM + fused selection).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbk {

// One operand (queries or database) converted for the tensor cores: TF32 hi/lo pieces,
// BF16 or FP8 E4M3 rows padded to a 128-byte multiple, plus squared norms (and per-row
// FP8 scales).  Owns its scratch memory.
struct PreparedOperand {
  int prec = 0;
  int64_t n = 0;
  int d = 0, dpad = 0, nkb = 0;
  Scratch data, norms, scale;
  void* piece[2] = {nullptr, nullptr};
};

struct KnnPlan {
  int prec = GBK_PREC_FP32;
  int chunks = 0;  // 0 = planned from the shapes
  int kprime = 0;  // low precision: re-ranked candidates (0 = 4k)
  int32_t* certified = nullptr;  // low precision: [nq] 1 if provably the float32 top-k
  float* error_bound = nullptr;  // low precision: [nq] bound on |low - exact| distance
  bool exact = false;            // low precision: re-run uncertified queries in float32
  int prefilter = 0;             // threshold pre-pass of the fused selection: 1 on, -1 off,
                                 // 0 automatic
};

gbk_status prepare_operand(const float* x, int64_t n, int d, int prec, int64_t nrows_pad,
                           float pad_norm, PreparedOperand* out, cudaStream_t st);

// Full pairwise squared L2 distances (clamped at 0) or inner products, out[q*ldo + i],
// for query rows [q0, q0 + qn) (all rows when qn < 0).  add_xnorm = false leaves out the
// query norm (and the clamp): ||y||^2 - 2<x,y>.
gbk_status pairwise_run(const PreparedOperand& Q, const PreparedOperand& B, bool ip, float* out,
                        int64_t ldo, cudaStream_t st, int64_t q0 = 0, int64_t qn = -1,
                        bool add_xnorm = true);

// Exact k-NN (arguments validated by the caller).
gbk_status knn_run(const float* xq, int64_t nq, const float* xb, int64_t nb, int d, int k,
                   int metric, float* D, int64_t* I, const KnnPlan& plan, cudaStream_t st);
// The database operand of knn_run in the plan's precision (rows padded to whole tiles),
// and knn_run on such a prepared database (xb: its float32 rows, used by the low-precision
// re-rank and the float32 repair).
gbk_status prepare_database(const float* xb, int64_t nb, int d, int prec, PreparedOperand* B,
                            cudaStream_t st);
gbk_status knn_run_prepared(const float* xq, int64_t nq, const float* xb,
                            const PreparedOperand& B, int64_t nb, int d, int k, int metric,
                            float* D, int64_t* I, const KnnPlan& plan, cudaStream_t st);

// The same with host-resident inputs and outputs (D_h, I_h written by copies on `st`).
gbk_status knn_host_run(const float* xq_h, int64_t nq, const float* xb_h, int64_t nb, int d,
                        int k, int metric, float* D_h, int64_t* I_h, const KnnPlan& plan,
                        cudaStream_t st);

int plan_chunks(int nqt, int ntiles, int grid_cap, int k, int max_chunks = 512);

// Top k of nparts sorted partial lists per query: Dp/Ip [nparts][nq][kin] (ids < 2^32;
// negative ids skipped) -> D/I [nq][k], order (value, id); padding (+-inf, -1).
gbk_status merge_parts_run(const float* Dp, const int64_t* Ip, int nparts, int64_t nq, int kin,
                           int k, bool largest, float* D, int64_t* I, cudaStream_t st);

// Exact float32 re-rank of k' candidates (Ic, Dc: low-precision results) to the top k,
// with the per-query certificate (see rerank.cu).
gbk_status rerank_run(const float* xq, const float* xb, int64_t nq, int64_t nb, int d,
                      int kprime, int k, bool largest, int prec, const float* xnorm2,
                      const float* qscale, const float* ynorm2, const float* bscale,
                      const int64_t* Ic, const float* Dc, float* D, int64_t* I,
                      int32_t* certified, float* eps_out, cudaStream_t st);

}  // namespace gbk
