// List-scan kernels for 64-byte codes.
#include "ivf_scan_kernels.cuh"

namespace gbk {
template gbk_status scan_k<64>(const ScanArgs&, const ScanTuning&, cudaStream_t);
}  // namespace gbk
