// List-scan kernels for 8-byte codes.
#include "ivf_scan_kernels.cuh"

namespace gbk {
template gbk_status scan_k<8>(const ScanArgs&, const ScanTuning&, cudaStream_t);
}  // namespace gbk
