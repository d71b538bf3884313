// List-scan kernels for 52, 56, 60-byte codes (the light launch shape).
#include "ivf_scan_kernels.cuh"

namespace gbk {
template gbk_status scan_k<52>(const ScanArgs&, const ScanTuning&, cudaStream_t);
template gbk_status scan_k<56>(const ScanArgs&, const ScanTuning&, cudaStream_t);
template gbk_status scan_k<60>(const ScanArgs&, const ScanTuning&, cudaStream_t);
}  // namespace gbk
