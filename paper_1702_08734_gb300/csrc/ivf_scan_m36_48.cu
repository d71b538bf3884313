// List-scan kernels for 36, 40, 44, 48-byte codes (the light launch shape).
#include "ivf_scan_kernels.cuh"

namespace gbk {
template gbk_status scan_k<36>(const ScanArgs&, const ScanTuning&, cudaStream_t);
template gbk_status scan_k<40>(const ScanArgs&, const ScanTuning&, cudaStream_t);
template gbk_status scan_k<44>(const ScanArgs&, const ScanTuning&, cudaStream_t);
template gbk_status scan_k<48>(const ScanArgs&, const ScanTuning&, cudaStream_t);
}  // namespace gbk
