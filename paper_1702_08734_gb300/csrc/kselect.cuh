// Internal launchers of the standalone k-selection kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gbknn.h"

namespace gbk {

struct KselectTuning {
  int segs = 1;    // segments per row (two-pass selection when > 1)
  int unroll = 8;  // 16-byte loads in flight per thread per iteration (4 or 8)
};

KselectTuning kselect_default_tuning(int64_t rows, int64_t len, int k);

// Arguments are validated by the caller (1 <= k <= min(len, GBK_MAX_K), len < 2^31).
gbk_status kselect_run(const float* vals, int64_t rows, int64_t len, int k, bool largest,
                       float* D, int64_t* I, cudaStream_t stream, const KselectTuning* tuning);

// Same selection with the segment partials in a fixed device array (no allocation).
gbk_status kselect_static_run(const float* vals, int64_t rows, int64_t len, int k, bool largest,
                              int segments, float* D, int64_t* I, cudaStream_t stream);

gbk_status row_norms_run(const float* x, int64_t n, int d, float* out, cudaStream_t stream);

}  // namespace gbk
