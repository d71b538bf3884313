/*
 * gbknn - exact and IVFADC k-nearest-neighbour search on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library (libgbknn.so).  It follows the problem statement of Johnson,
 * Douze and Jegou, "Billion-scale similarity search with GPUs" (arXiv 1702.08734),
 * section 2.
 *
 * Conventions common to every entry point
 *  - Every array pointer is a DEVICE pointer unless stated otherwise, owned by the
 *    caller, valid for the whole call on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Calls are asynchronous: outputs are complete when `stream` is synchronised.
 *  - Matrices are dense row-major float32; indices and ids are int64.
 *  - Scratch memory comes from the allocator installed with gbk_set_allocator (default:
 *    cudaMallocAsync / cudaFreeAsync on `stream`).  It is freed stream-ordered before
 *    the call returns.
 *  - Selection order: for "smallest" (squared L2) a candidate is better when its value is
 *    smaller; for "largest" (inner product) when larger.  NaN ranks after every number in
 *    both orders, -0 equals +0, and equal values are ordered by the lower index.  (The
 *    paper leaves the order of equal keys unspecified, section 2.)
 *  - Return value: GBK_OK, or an error status; gbk_last_error() then returns a message
 *    (thread-local, valid until the next call on the same thread).  Invalid arguments are
 *    detected before any work is queued; nothing is written to outputs in that case.
 */
#ifndef GBKNN_H
#define GBKNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gbk_status;
#define GBK_OK 0
#define GBK_EINVAL 1       /* invalid argument                                  */
#define GBK_ENOMEM 2       /* scratch allocation failed                         */
#define GBK_ECUDA 3        /* a CUDA runtime or driver call failed              */
#define GBK_ETIMEOUT 4     /* a bounded device-side wait gave up                */
#define GBK_EUNSUPPORTED 5 /* valid request outside what this build implements  */
#define GBK_EDEVICE 6      /* a kernel reported an error in its status word     */

#define GBK_METRIC_L2 0 /* squared Euclidean distance, ascending  */
#define GBK_METRIC_IP 1 /* inner product, descending              */

#define GBK_MAX_K 1024 /* largest k any selection accepts (the paper's WarpSelect bound, section 4.2) */

/* Pluggable scratch allocator.  alloc returns a device pointer (or NULL on failure)
 * usable on `stream` in stream order; free releases it in stream order. */
typedef struct gbk_allocator {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, void* stream);
} gbk_allocator;

/* Library version as major*10000 + minor*100 + patch. */
int32_t gbk_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char* gbk_last_error(void);

/* Install (or, with NULL, reset to the default) the scratch allocator.  Not thread-safe
 * with respect to calls in flight on other threads. */
gbk_status gbk_set_allocator(const gbk_allocator* allocator);

/*
 * Row-wise k-selection (section 2, "k-selection"; batched over rows as in "Batching").
 *   vals    [rows][len] float32 input
 *   k       1 <= k <= min(len, GBK_MAX_K)
 *   largest 0: k smallest values, ascending; 1: k largest, descending
 *   D       [rows][k] float32 out: the selected values (the input's own bits)
 *   I       [rows][k] int64 out: their column indices, 0 <= I < len
 * len must be < 2^31.  rows == 0 is a no-op.  Errors: GBK_EINVAL (k or sizes out of
 * range, NULL pointer with rows > 0), GBK_ENOMEM, GBK_ECUDA.
 */
gbk_status gbk_kselect(const float* vals, int64_t rows, int64_t len, int32_t k,
                       int32_t largest, float* D, int64_t* I, void* stream);

/*
 * Squared L2 norms of the rows of x (the precomputable terms of Eq. (2), section 2).
 *   x [n][d] float32 in, out [n] float32 out.  Errors: GBK_EINVAL, GBK_ECUDA.
 */
gbk_status gbk_row_norms(const float* x, int64_t n, int32_t d, float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBKNN_H */
