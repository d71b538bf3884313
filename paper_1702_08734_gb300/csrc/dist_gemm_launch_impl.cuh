// Launcher of the fused distance GEMM for one operand precision KIND: picks the template
// instance for (mode, candidate-list length, order) and raises its shared-memory limit.
// Each precision's translation unit (dist_gemm_{tf32x3,bf16,fp8}.cu) instantiates it once,
// so the three kernel families compile in parallel.
#pragma once
#include "dist_gemm_kernel.cuh"
#include "dist_gemm_launch.cuh"

namespace gbk {

template <int KIND, int MODE, int KPR, bool LG>
static gbk_status gemm_go(const CUtensorMap* m, const GemmArgs& a, int grid, size_t smem,
                          cudaStream_t st) {
  auto kern = dist_gemm_kernel<KIND, MODE, KPR, LG>;
  // at the device maximum: callers pass shapes needing up to that much
  GBK_TRY(set_smem_limit(kern, device_info().smem_optin));
  kern<<<grid, gemm_threads(KindTraits<KIND>::EPI), smem, st>>>(m[0], m[1], m[2], m[3], a);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

template <int KIND, bool LG>
static gbk_status gemm_pick(int mode, int kpr, const CUtensorMap* m, const GemmArgs& a, int grid,
                            size_t smem, cudaStream_t st) {
  if (mode == MODE_STORE) return gemm_go<KIND, MODE_STORE, 0, LG>(m, a, grid, smem, st);
  switch (kpr) {
    case 0: return gemm_go<KIND, MODE_SELECT, 0, LG>(m, a, grid, smem, st);
    case 1: return gemm_go<KIND, MODE_SELECT, 1, LG>(m, a, grid, smem, st);
    case 2: return gemm_go<KIND, MODE_SELECT, 2, LG>(m, a, grid, smem, st);
    case 4: return gemm_go<KIND, MODE_SELECT, 4, LG>(m, a, grid, smem, st);
    case 8: return gemm_go<KIND, MODE_SELECT, 8, LG>(m, a, grid, smem, st);
    case 16: return gemm_go<KIND, MODE_SELECT, 16, LG>(m, a, grid, smem, st);
    default: return set_error(GBK_EUNSUPPORTED, "fused selection supports k <= 512");
  }
}

template <int KIND>
static gbk_status gemm_launch(int mode, int kpr, bool largest, const CUtensorMap* maps,
                              const GemmArgs& a, int grid, size_t smem, cudaStream_t st) {
  return largest ? gemm_pick<KIND, true>(mode, kpr, maps, a, grid, smem, st)
                 : gemm_pick<KIND, false>(mode, kpr, maps, a, grid, smem, st);
}

}  // namespace gbk

// Defines gbk::launch_dist_gemm_<NAME> for precision KIND.
#define GBK_DEFINE_GEMM_LAUNCHER(NAME, KIND)                                                 \
  namespace gbk {                                                                            \
  gbk_status launch_dist_gemm_##NAME(int mode, int kpr, bool largest, const CUtensorMap* maps, \
                                     const GemmArgs& a, int grid, size_t smem,               \
                                     cudaStream_t st) {                                      \
    return gemm_launch<KIND>(mode, kpr, largest, maps, a, grid, smem, st);                   \
  }                                                                                          \
  }
