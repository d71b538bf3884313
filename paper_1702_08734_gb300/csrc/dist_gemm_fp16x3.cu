// Fused distance GEMM instances for fp16x3 operands (float32-accurate FP16 hi/lo split).
#include "dist_gemm_launch_impl.cuh"

GBK_DEFINE_GEMM_LAUNCHER(fp16x3, KIND_FP16X3)
