// Fused distance GEMM instances for bf16 operands.
#include "dist_gemm_launch_impl.cuh"

GBK_DEFINE_GEMM_LAUNCHER(bf16, KIND_BF16)
