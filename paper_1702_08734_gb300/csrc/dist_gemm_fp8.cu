// Fused distance GEMM instances for fp8 operands.
#include "dist_gemm_launch_impl.cuh"

GBK_DEFINE_GEMM_LAUNCHER(fp8, KIND_FP8)
