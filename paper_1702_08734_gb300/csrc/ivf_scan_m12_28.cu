// List-scan kernels for 12, 20, 24, 28-byte codes (the light launch shape).
#include "ivf_scan_kernels.cuh"

namespace gbk {
template gbk_status scan_k<12>(const ScanArgs&, const ScanTuning&, cudaStream_t);
template gbk_status scan_k<20>(const ScanArgs&, const ScanTuning&, cudaStream_t);
template gbk_status scan_k<24>(const ScanArgs&, const ScanTuning&, cudaStream_t);
template gbk_status scan_k<28>(const ScanArgs&, const ScanTuning&, cudaStream_t);
}  // namespace gbk
