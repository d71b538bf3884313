// Internal interfaces of the inverted-file indexes: stable bucketing, k-means, row gathers,
// the flat list scan.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbk {

// Persistent device allocation owned by an index (freed when the index is destroyed).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  gbk_status alloc(size_t b) {
    release();
    if (b == 0) return GBK_OK;
    if (cudaMalloc(&p, b) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return set_error(GBK_ENOMEM, "cudaMalloc(%zu) failed for index storage", b);
    }
    bytes = b;
    return GBK_OK;
  }
  // grow to at least b bytes, keeping the first `keep` bytes (stream-ordered copy)
  gbk_status grow(size_t b, size_t keep, cudaStream_t st) {
    if (b <= bytes) return GBK_OK;
    void* q = nullptr;
    if (cudaMalloc(&q, b) != cudaSuccess) {
      cudaGetLastError();
      return set_error(GBK_ENOMEM, "cudaMalloc(%zu) failed for index storage", b);
    }
    if (keep) GBK_CUDA_CHECK(cudaMemcpyAsync(q, p, keep, cudaMemcpyDeviceToDevice, st));
    GBK_CUDA_CHECK(cudaStreamSynchronize(st));
    release();
    p = q;
    bytes = b;
    return GBK_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};


// Launch shape of the IVFADC list scan, chosen by gbk_ivfpq_autotune or set by the caller:
// codes each thread loads per step (2, 4 or 8), resident blocks per SM (1..8) of the
// persistent mode, and whether a plain search takes its queries in the order of their
// nearest list (persistent mode) or in input order (block per query).  Results do not
// depend on it.
struct ScanTuning {
  int codes_per_thread = 2;
  int blocks_per_sm = 2;
  int list_order = 0;  // plain search: queries in the order of their nearest list (1)
  int threads = 384;   // table-mode scan block size: 256, 384 (U <= 4) or 512 (U = 2)
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

// out[j] = in[order[j]] for rows of d floats, j < n (list-order copy of staged vectors).
gbk_status gather_rows_run(const float* in, const int64_t* order, int64_t n, int d, float* out,
                           cudaStream_t st);

// Exact list scan (IVF-Flat): for query q and its probed lists cl_I[q][0..nprobe), the
// squared L2 distance sum_t (x_t - y_t)^2 of every stored vector (vecs, list order) and the
// k best per query by (distance, list position); ids[position] out, or the position itself
// when ids is null.  Padding (+inf, -1).
gbk_status ivf_flat_scan_run(const float* xq, int64_t nq, int d, int nprobe, int k,
                             const int64_t* cl_I, const int64_t* list_off, const float* vecs,
                             const int64_t* ids, float* D, int64_t* I, cudaStream_t st);

// Exact float32 re-rank of k' candidates given as row numbers of xb (negative = none): the
// k best by (distance, row) of sum_t (x_t - y_t)^2; rows out (or -1 with +inf).
gbk_status rerank_rows_run(const float* xq, const float* xb, int64_t nq, int d, int kprime,
                           int k, const int64_t* rows, float* D, int64_t* I, cudaStream_t st);

// I[j] = ids[I[j]] for I[j] >= 0 (row numbers to stored ids), j < n.
gbk_status rows_to_ids_run(int64_t* I, int64_t n, const int64_t* ids, cudaStream_t st);

}  // namespace gbk
