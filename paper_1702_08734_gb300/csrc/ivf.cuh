// Internal interfaces of the IVFADC index: stable bucketing, k-means, product quantizer.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbk {

// Launch shape of the IVFADC list scan, chosen by gbk_ivfpq_autotune or set by the caller:
// codes each thread loads per step (2, 4 or 8) and, in the persistent mixed-batch mode,
// resident blocks per SM (1..8).  Results do not depend on it.
struct ScanTuning {
  int codes_per_thread = 4;
  int blocks_per_sm = 2;
};

// Stable counting sort by key in [0, nb): offsets[nb+1], order[n] (positions grouped by
// key, ascending within a key).  n < 2^31.
gbk_status bucket_stable(const int32_t* keys, int64_t n, int nb, int64_t* offsets, int64_t* order,
                         cudaStream_t st);

// Lloyd's k-means on device data x[n][d] (section 2 / 6.2): centroids[nc][d] out (float32),
// initial centroids = rows init_idx (device, int64).  objective (device, niter doubles) may be
// null.  assign_fp32_direct selects the assignment kernel: false = tensor-core k-NN (k = 1),
// true = direct float32 distances (small d).
// ldx is the row stride of x (== d for the tensor-core assignment); n_split (device, may be
// null) counts the empty-cluster re-seeds.
gbk_status kmeans_run(const float* x, int64_t n, int d, int ldx, int nc, int niter,
                      const int64_t* init_idx, float* centroids, double* objective,
                      long long* n_split, bool assign_direct, cudaStream_t st);

// Nearest centroid by direct float32 distances (ties to the lowest index), small d <= 32,
// nc <= 256: a[n] (int32), optional dist[n].
gbk_status assign_direct_run(const float* x, int64_t n, int ldx, int d, const float* cent, int nc,
                             int32_t* a, float* dist, cudaStream_t st);

}  // namespace gbk
