// Instantiations of the fused distance GEMM for one operand precision.
#include "dist_gemm_kernel.cuh"
#include "dist_gemm_launch.cuh"

namespace gbk {

template <int MODE, int KPR, bool LG>
static gbk_status go(const CUtensorMap* m, const GemmArgs& a, int grid, size_t smem,
                     cudaStream_t st) {
  auto kern = dist_gemm_kernel<KIND_TF32X3, MODE, KPR, LG>;
  static bool attr = false;
  if (!attr) {  // once, at the device maximum: callers pass shapes needing up to that much
    GBK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)device_info().smem_optin));
    attr = true;
  }
  kern<<<grid, gemm_threads(KindTraits<KIND_TF32X3>::EPI), smem, st>>>(m[0], m[1], m[2], m[3], a);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

template <bool LG>
static gbk_status pick(int mode, int kpr, const CUtensorMap* m, const GemmArgs& a, int grid,
                       size_t smem, cudaStream_t st) {
  if (mode == MODE_STORE) return go<MODE_STORE, 0, LG>(m, a, grid, smem, st);
  switch (kpr) {
    case 0: return go<MODE_SELECT, 0, LG>(m, a, grid, smem, st);
    case 1: return go<MODE_SELECT, 1, LG>(m, a, grid, smem, st);
    case 2: return go<MODE_SELECT, 2, LG>(m, a, grid, smem, st);
    case 4: return go<MODE_SELECT, 4, LG>(m, a, grid, smem, st);
    case 8: return go<MODE_SELECT, 8, LG>(m, a, grid, smem, st);
    case 16: return go<MODE_SELECT, 16, LG>(m, a, grid, smem, st);
    default: return set_error(GBK_EUNSUPPORTED, "fused selection supports k <= 512");
  }
}

gbk_status launch_dist_gemm_tf32x3(int mode, int kpr, bool largest, const CUtensorMap* maps,
                               const GemmArgs& a, int grid, size_t smem, cudaStream_t st) {
  return largest ? pick<true>(mode, kpr, maps, a, grid, smem, st)
                 : pick<false>(mode, kpr, maps, a, grid, smem, st);
}

}  // namespace gbk
