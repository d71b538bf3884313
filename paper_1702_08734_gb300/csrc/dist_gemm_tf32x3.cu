// Fused distance GEMM instances for tf32x3 operands.
#include "dist_gemm_launch_impl.cuh"

GBK_DEFINE_GEMM_LAUNCHER(tf32x3, KIND_TF32X3)
