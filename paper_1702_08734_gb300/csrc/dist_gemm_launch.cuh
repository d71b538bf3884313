// Per-precision launchers of the fused distance GEMM (one translation unit each).
#pragma once
#include <cuda.h>

#include "dist_gemm.cuh"

namespace gbk {

// mode: MODE_SELECT / MODE_STORE; kpr: list length / 32 (0 = k == 1 arg-min).
gbk_status launch_dist_gemm_tf32x3(int mode, int kpr, bool largest, const CUtensorMap* maps,
                                   const GemmArgs& a, int grid, size_t smem, cudaStream_t st);
gbk_status launch_dist_gemm_bf16(int mode, int kpr, bool largest, const CUtensorMap* maps,
                                 const GemmArgs& a, int grid, size_t smem, cudaStream_t st);
gbk_status launch_dist_gemm_fp16x3(int mode, int kpr, bool largest, const CUtensorMap* maps,
                                   const GemmArgs& a, int grid, size_t smem, cudaStream_t st);
gbk_status launch_dist_gemm_fp8(int mode, int kpr, bool largest, const CUtensorMap* maps,
                                const GemmArgs& a, int grid, size_t smem, cudaStream_t st);

}  // namespace gbk
