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
 *    stream-ordered allocation on `stream` from the library's own memory pool per device,
 *    which keeps up to 8 GiB of freed scratch mapped between calls).  It is freed
 *    stream-ordered before the call returns.
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

/* Arithmetic of the distance GEMM (the -2<x,y> term of Eq. (2)). */
#define GBK_PREC_FP32 0   /* float32-accurate: each row scaled by a power of two s >= max|x|, */
                          /* split into FP16 pieces hi + lo (22 significand bits), 3 passes  */
                          /* (hi hi + hi lo + lo hi) at the FP16 rate, float32 accumulation   */
#define GBK_PREC_BF16 1   /* one BF16 pass, float32 accumulation                              */
#define GBK_PREC_FP8 2    /* one FP8 E4M3 pass with per-row scales, float32 accumulation      */
#define GBK_PREC_TF32X3 3 /* float32-accurate: TF32 hi/lo split, 3 passes at the TF32 rate    */

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

/* Kernel timing for benchmarks and tracing.  While enabled, every library kernel launch
 * is bracketed by a CUDA event pair on its stream.  gbk_profile_read waits for the
 * recorded events, writes up to max_records (name: 32 bytes each, NUL-terminated; time in
 * ms) in launch order, clears the record list and returns the count written. */
void gbk_profile_enable(int32_t on);
int32_t gbk_profile_read(char* names, float* ms, int32_t max_records);

/* Synchronise `stream`, then report (and clear) the device status word that kernels set
 * instead of trapping: GBK_ETIMEOUT when a bounded device-side wait gave up (the kernel
 * skipped its remaining work; its outputs are undefined), GBK_EDEVICE for other flags. */
gbk_status gbk_device_status(void* stream);

/* Self-test of that path (not part of the paper): launches one thread that waits on a
 * shared-memory mbarrier nobody arrives at, bounded by limit_ns (1 us .. 2 s) of GPU
 * time, as every mbarrier wait of the library is bounded.  The wait gives up, sets the
 * timeout flag of the status word and the kernel returns: the next gbk_device_status on
 * that stream reports GBK_ETIMEOUT, and the context stays usable.  GBK_EINVAL for a limit
 * outside that range. */
gbk_status gbk_selftest_wait_timeout(int64_t limit_ns, void* stream);

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

/* Launch parameters of gbk_kselect_ex; 0 selects the library default. */
typedef struct gbk_kselect_opts {
  int32_t segments; /* thread blocks per row (>1: two-pass selection, section 5.3) */
  int32_t unroll;   /* how the row is streamed (k > 1): 4 or 8 = 16-byte register   */
                    /* loads in flight per thread per iteration; 1 = a shared-memory */
                    /* ring of four 16 KB bulk copies kept in flight per block      */
} gbk_kselect_opts;

/* gbk_kselect with explicit launch parameters (opts may be NULL).  Results do not
 * depend on the parameters.  Extra error: GBK_EINVAL for unroll other than 0, 1, 4, 8. */
gbk_status gbk_kselect_ex(const float* vals, int64_t rows, int64_t len, int32_t k,
                          int32_t largest, float* D, int64_t* I, const gbk_kselect_opts* opts,
                          void* stream);

/*
 * gbk_kselect for callers that cannot allocate device memory during the call (for
 * example code being captured into a CUDA graph on a pool it does not own, latency-bound
 * paths that forbid allocator calls after start-up, or hosts whose only allocator is
 * their own).  The paper has no counterpart: this is a deployment variant of the
 * row-split (two-pass) selection of gbk_kselect_ex.
 *   Same arguments and results as gbk_kselect_ex with opts.segments = segments (0 = the
 *   library's plan).  When the plan splits rows (segments > 1) the per-segment partial
 *   results live in a fixed device array of 2^21 entries (16 MiB) that is part of the
 *   library image, held on every GPU that loads the library until the process exits:
 *   rows * segments * k must not exceed 2^21, else GBK_EINVAL and nothing is launched.
 *   No cudaMalloc/cudaFree or other allocating call is made.
 *   The first call on a device looks up the array's device address (once per device, with
 *   that device current); make that first call before any stream capture.
 *   Every call shares the array and it keeps the last call's contents (each call writes
 *   all the partials it reads, so nothing needs clearing); calls whose executions overlap
 *   on the GPU race on it and must be serialised by the caller.
 */
gbk_status gbk_kselect_static(const float* vals, int64_t rows, int64_t len, int32_t k,
                              int32_t largest, int32_t segments, float* D, int64_t* I,
                              void* stream);

/*
 * Squared L2 norms of the rows of x (the precomputable terms of Eq. (2), section 2).
 *   x [n][d] float32 in, out [n] float32 out.  Errors: GBK_EINVAL, GBK_ECUDA.
 */
gbk_status gbk_row_norms(const float* x, int64_t n, int32_t d, float* out, void* stream);

/* Options of gbk_knn_brute (NULL = defaults). */
typedef struct gbk_knn_opts {
  int32_t precision; /* GBK_PREC_FP32 (default), GBK_PREC_TF32X3, GBK_PREC_BF16 or      */
                     /* GBK_PREC_FP8                                                    */
  int32_t kprime;    /* BF16/FP8: candidates re-ranked in float32 (0 = 4k for k <= 16,   */
                     /* k + k/4 above; >= k, <= 1024)                                  */
  int32_t chunks;    /* database chunks of the work decomposition (0 = planned)          */
  int32_t* certified; /* BF16/FP8, optional device [nq]: 1 if the result provably equals
                         the float32 top-k (see gbk_knn_brute), 2 if it was re-run on the
                         float32 path (exact != 0), else 0                             */
  float* error_bound; /* BF16/FP8, optional device [nq]: bound on |low-precision - float32|
                         distance used by the certificate                              */
  int32_t exact;      /* BF16/FP8: nonzero re-runs every query the certificate does not
                         cover on the float32 path and returns its result there, so every
                         row is the float32 top-k (the call then synchronises `stream`
                         once, to learn how many queries to re-run)                     */
  int32_t prefilter;  /* threshold pre-pass of the fused selection: -1 off, 1 on for
                         k > 1, 0 on for k >= 32 (64 with GBK_PREC_TF32X3; BF16/FP8
                         count the over-fetched k'); either only where the database holds
                         at least 2k blocks of 64 rows (128 with GBK_PREC_TF32X3).  The
                         pre-pass takes the best distance of every (query, block) over
                         the first third (k > 64) or quarter of the database (the
                         float32-accurate kinds in one pass over their high pieces, the
                         k-th best then widened by a bound on the terms that pass leaves
                         out); their k-th best bounds the k-th nearest distance, so the
                         fused selection starts with that threshold.  Results are the
                         same either way.                                                */
} gbk_knn_opts;

/*
 * Exact k nearest neighbours of each query (Eq. (1), section 2; computed through the
 * decomposition of Eq. (2) with the GEMM on the tensor cores and the k-selection fused
 * into its epilogue, section 5.1).
 *   xq [nq][d], xb [nb][d] float32;  1 <= k <= min(nb, GBK_MAX_K);  metric GBK_METRIC_*
 *   D  [nq][k] float32 out: squared L2 distances ascending (clamped at 0), or inner
 *      products descending;  I [nq][k] int64 out: database row numbers.
 * GBK_PREC_FP32 keeps float32 accuracy (FP16 hi/lo split of power-of-two-scaled rows,
 * three tensor-core passes; GBK_PREC_TF32X3 the TF32 split).  BF16/FP8 select kprime
 * candidates in low precision, then recompute their distances directly in float32 and
 * keep the best k.  A query is certified when the k'-th low-precision distance minus
 * the error bound exceeds the k-th re-ranked distance (plus, for inner product), which
 * proves no other database row belongs to the top k.
 * Limits: nb, nq < 2^31; BF16/FP8 d <= 8192 (the float32 re-rank).  A 128-query tile of
 * the GEMM stays in shared memory while d <= 192 (FP32), 128 (TF32X3), 512 (BF16) or
 * 1024 (FP8) with candidate lists (k > 1), 256 / 128 / 704 / 1408 without; longer rows
 * stream the query
 * k-blocks through the shared-memory ring beside the database's (same results).  Errors:
 * GBK_EINVAL, GBK_EUNSUPPORTED, GBK_ENOMEM, GBK_ECUDA.  Inputs must be finite.
 */
gbk_status gbk_knn_brute(const float* xq, int64_t nq, const float* xb, int64_t nb, int32_t d,
                         int32_t k, int32_t metric, float* D, int64_t* I,
                         const gbk_knn_opts* opts, void* stream);

/*
 * A database prepared once for repeated exact k-NN searches (section 5.1's exact search
 * against a fixed database): the operand pieces of `precision` (the FP16 / TF32 hi-lo
 * split, BF16 or FP8 with row scales) and the squared norms are formed at creation and
 * kept in device memory owned by the handle, so each gbk_knn_db_search skips that pass
 * over the database.  xb [nb][d] float32 (device) is NOT copied: it must stay valid and
 * unchanged while the handle is used (the BF16/FP8 re-rank and the float32 repair read
 * it).  gbk_knn_db_search takes the arguments and options of gbk_knn_brute (opts may be
 * NULL; a precision other than the handle's is GBK_EINVAL) and returns the same results.
 * gbk_knn_db_destroy frees the handle's device memory stream-ordered on `stream`.
 * Errors: GBK_EINVAL, GBK_ENOMEM, GBK_ECUDA, and those of gbk_knn_brute.
 */
typedef struct gbk_knn_db gbk_knn_db;
gbk_status gbk_knn_db_create(const float* xb, int64_t nb, int32_t d, int32_t precision,
                             gbk_knn_db** out, void* stream);
gbk_status gbk_knn_db_search(const gbk_knn_db* db, const float* xq, int64_t nq, int32_t k,
                             int32_t metric, float* D, int64_t* I, const gbk_knn_opts* opts,
                             void* stream);
void gbk_knn_db_destroy(gbk_knn_db* db, void* stream);

/*
 * gbk_knn_brute with HOST arrays: xq [nq][d], xb [nb][d] float32 and the outputs D [nq][k],
 * I [nq][k] in host memory (page-locked for the copies to overlap the search; pageable
 * memory works but serialises them).  The call enqueues the host->device copies, the
 * search and the device->host copies of D and I on `stream` and returns; D and I are
 * valid once the stream has been synchronised, and the host arrays must stay alive until
 * then.  With a float32-accurate precision and the fused selection (k <= 512, nb > 65,536)
 * the database is copied in growing pieces (2^16, 2^17, ... rows) on a second stream while
 * the search runs over the pieces already copied (the result is that of gbk_knn_brute).
 * Device scratch:
 * the inputs, outputs and the search's own.  Options as gbk_knn_brute, except that the
 * certified / error_bound outputs are not available (GBK_EINVAL).  Errors: as
 * gbk_knn_brute.
 */
gbk_status gbk_knn_brute_host(const float* xq, int64_t nq, const float* xb, int64_t nb,
                              int32_t d, int32_t k, int32_t metric, float* D, int64_t* I,
                              const gbk_knn_opts* opts, void* stream);

/*
 * All pairwise distances out[i*ldo + j] between xq[i] and xb[j] (section 2, "Exact
 * search": the matrix D): max(0, ||x||^2 + ||y||^2 - 2<x,y>) for GBK_METRIC_L2, <x,y> for
 * GBK_METRIC_IP, with the GEMM in the given precision.  ldo >= nb.  Same limits as
 * gbk_knn_brute.
 */
gbk_status gbk_pairwise_distances(const float* xq, int64_t nq, const float* xb, int64_t nb,
                                  int32_t d, int32_t metric, int32_t precision, float* out,
                                  int64_t ldo, void* stream);

/*
 * Lloyd's k-means (section 2: the coarse quantizer is "trained via k-means"; section 6.2
 * uses exact search with k = 1 for the assignment).
 *   x [n][d] device float32; init_idx: HOST array of nc row numbers of x (the initial
 *   centroids; e.g. a seeded random permutation's prefix); centroids [nc][d] device out;
 *   objective: optional DEVICE [niter] doubles, the sum of squared distances of the
 *   assignment of each iteration; n_split: optional DEVICE int64, empty clusters re-seeded.
 * Assignment ties go to the lowest centroid; each update is the float64 mean of the
 * members (summed in member order), rounded to float32; an empty cluster e (in increasing
 * order) takes the most populated cluster s (lowest index on ties): c_e = c_s (1 + g/1024),
 * c_s = c_s (1 - g/1024), g = +1 on even, -1 on odd dimensions; s's count is halved.
 * direct_assign = 1 uses direct float32 distances (d <= 32, nc <= 256), else the tensor
 * cores.  Errors: GBK_EINVAL, GBK_EUNSUPPORTED, GBK_ENOMEM, GBK_ECUDA.
 */
gbk_status gbk_kmeans(const float* x, int64_t n, int32_t d, int32_t nc, int32_t niter,
                      const int64_t* init_idx, float* centroids, double* objective,
                      int64_t* n_split, int32_t direct_assign, void* stream);

/* ------------------------------------------------------------------ IVFADC index */

/* An IVFADC index (section 2 "Compressed-domain search"): a coarse quantizer of nlist
 * centroids, a product quantizer of M sub-quantizers with 256 centroids (8-bit codes),
 * and inverted lists stored as two arrays, codes and 64-bit ids (section 5.3).  The index
 * owns its device memory.  Not thread-safe: serialise calls on one index. */
typedef struct gbk_index gbk_index;

/* d % M == 0, M a multiple of 4 up to 64, d / M <= 32, nbits == 8, metric == GBK_METRIC_L2 (the
 * paper's IVFADC is defined for L2, Eq. 6; others give GBK_EUNSUPPORTED). */
gbk_status gbk_ivfpq_create(int32_t d, int32_t nlist, int32_t M, int32_t nbits, int32_t metric,
                            gbk_index** out);
void gbk_ivfpq_destroy(gbk_index* index);

typedef struct gbk_train_opts {
  int32_t niter;              /* coarse k-means iterations (0 = 20)                     */
  int32_t pq_niter;           /* product-quantizer k-means iterations (0 = niter)       */
  const int64_t* coarse_init; /* HOST [nlist] initial coarse centroid rows (NULL = 0..) */
  const int64_t* pq_init;     /* HOST [256] initial sub-quantizer rows (NULL = 0..255)  */
  int32_t use_precomputed;    /* 1: term-1 table of Eq. (11), nlist*M*256 floats; 0: per
                                 (query, list) tables computed in the scan kernel       */
} gbk_train_opts;

/* Train q1 by k-means on x [n][d] (device), then the product quantizer on the residuals
 * y - q1(y) (Eq. 3), each sub-quantizer by 256-centroid k-means.  Discards no data already
 * added.  max(nlist, 256) <= n < 2^31. */
gbk_status gbk_ivfpq_train(gbk_index* index, const float* x, int64_t n,
                           const gbk_train_opts* opts, void* stream);

/* Install externally trained quantizers: coarse [nlist][d], pq [M][256][d/M] (device or
 * host float32). */
gbk_status gbk_ivfpq_set_quantizers(gbk_index* index, const float* coarse, const float* pq,
                                    int32_t use_precomputed, void* stream);

/* Encode and append x [n][d] (device): list = nearest coarse centroid (ties lowest), code
 * byte m = nearest centroid of sub-quantizer m to sub-vector m of the residual (ties
 * lowest).  ids: device [n] int64, or NULL for running numbers 0, 1, ...  Lists keep
 * insertion order.  At most 2^32 - 1 vectors in total. */
gbk_status gbk_ivfpq_add(gbk_index* index, const float* x, int64_t n, const int64_t* ids,
                         void* stream);

/* IVFADC batch search (Algorithm 4): the nprobe nearest coarse centroids of each query
 * (Eq. 5), ADC distances of every vector of those lists (Eq. 6, 10-11), k smallest.
 *   D [nq][k] squared distances ascending, I [nq][k] ids; when the probed lists hold
 *   fewer than k vectors the tail is (+inf, -1).  Equal distances: lower list position
 *   first (= lower id when ids are running numbers).  1 <= k, nprobe <= GBK_MAX_K,
 *   nprobe <= nlist. */
gbk_status gbk_ivfpq_search(gbk_index* index, const float* xq, int64_t nq, int32_t k,
                            int32_t nprobe, float* D, int64_t* I, void* stream);

/* Sizes of the index (synchronises `stream` when lists must be rebuilt). */
gbk_status gbk_ivfpq_info(gbk_index* index, int64_t* ntotal, int32_t* nlist, int32_t* d,
                          int32_t* M, void* stream);

/* Copy out (any pointer may be NULL; host or device): coarse [nlist][d], pq [M][256][d/M],
 * list_off [nlist+1], codes [ntotal][M] and ids [ntotal] in list order. */
gbk_status gbk_ivfpq_export(gbk_index* index, float* coarse, float* pq, int64_t* list_off,
                            uint8_t* codes, int64_t* ids, void* stream);

/* Checkpoint of an index to a file and back (section 2's inverted file with its
 * quantizers; the paper does not specify a format).  gbk_ivfpq_save writes a header
 * (sizes, table mode, coarse precision, kept vectors, rotation, scan tuning, learned-nprobe
 * operating point) followed by
 * the coarse centroids, the codebooks, the rotation, the list offsets, the codes (byte m =
 * sub-quantizer m), the ids and the kept vectors, all in list order; it synchronises
 * `stream`.  gbk_ivfpq_load reads such a file into a new index (*out; destroy with
 * gbk_ivfpq_destroy) and rebuilds the term-1 tables and everything derived from them with
 * the same kernels, so searches of the loaded index return exactly what the saved index
 * returned; vectors may be added to it afterwards.  Errors: GBK_EINVAL (untrained index,
 * unreadable, truncated or inconsistent file), GBK_ENOMEM, GBK_ECUDA. */
gbk_status gbk_ivfpq_save(gbk_index* index, const char* path, void* stream);
gbk_status gbk_ivfpq_load(const char* path, gbk_index** out, void* stream);

/* OPQ pre-rotation (the optimized product quantization used by the paper's DEEP1B and
 * YFCC100M experiments, sections 1 and 6.4): with R [d][d] row-major (device or host
 * float32, typically orthogonal) every vector given to train, add, the searches and the
 * k-NN graph is replaced by R y before anything else, computed as the inner-product GEMM
 * y R^T on the tensor cores (float32-accurate).  The quantizers (set_quantizers, export),
 * the kept vectors and the learned-nprobe features then live in the rotated space; use
 * gbk_ivfpq_rotate to map vectors there.  Must be set before training / set_quantizers
 * and before the first add (EINVAL otherwise).  R = NULL removes it. */
gbk_status gbk_ivfpq_set_rotation(gbk_index* index, const float* R, void* stream);

/* out [n][d] = x [n][d] rotated by the index's R (a copy when it has none). */
/* Options of gbk_ivfpq_train_rotation (NULL or zero fields = defaults). */
typedef struct gbk_opq_opts {
  int32_t niter;             /* alternations of PQ training and Procrustes (0 = 10)       */
  int32_t pq_niter;          /* k-means iterations per PQ training (0 = 4)               */
  int32_t polar_iters;       /* scaled Newton iterations of the polar factor (0 = 12)    */
  const int64_t* pq_init;    /* HOST [256] rows of x that seed every sub-quantizer's      */
                             /* k-means (NULL = 0..255)                                   */
} gbk_opq_opts;

/* Train the OPQ rotation on x [n][d] (device) and install it (as gbk_ivfpq_set_rotation;
 * not specified by the paper, which uses OPQ for its DEEP1B / YFCC100M runs).  From
 * R = I, `niter` times: train the product quantizer of x R^T (256-centroid k-means per
 * block of d/M dimensions, seeded from the rows pq_init, pq_niter iterations), encode and
 * reconstruct every row (Y^), then set R to the orthogonal matrix minimising
 * ||x R^T - Y^||_F: the polar factor U V^T of A = Y^T x = U S V^T (A summed in double;
 * the polar factor by scaled Newton iterations X <- (g X + X^-T / g) / 2 in double, the
 * inverse by Gauss-Jordan elimination, then two Newton-Schulz steps).  Must run
 * before gbk_ivfpq_train and gbk_ivfpq_add (GBK_EINVAL otherwise).  R_out (host or
 * device, may be NULL): the trained R [d][d] row-major.  256 <= n < 2^31, d <= 1024.
 * GBK_EINVAL also when the cross-covariance A is singular (degenerate training data). */
gbk_status gbk_ivfpq_train_rotation(gbk_index* index, const float* x, int64_t n,
                                    const gbk_opq_opts* opts, float* R_out, void* stream);

gbk_status gbk_ivfpq_rotate(gbk_index* index, const float* x, int64_t n, float* out,
                            void* stream);

/* Arithmetic of the queries' coarse search (Eq. 5) in every search of this index:
 * GBK_PREC_FP32 (default), or GBK_PREC_BF16 / GBK_PREC_FP8 tensor-core GEMMs that fetch
 * nprobe + nprobe/4 (4 nprobe for nprobe <= 16) candidate lists and re-rank them by exact
 * float32 distances, as gbk_knn_brute does (pattern 1): the probed lists are then the
 * exact nearest ones unless a true one fell outside the over-fetch, and term 2 is exact.
 * Adding (q1 assignment) always uses float32. */
gbk_status gbk_ivfpq_set_coarse_precision(gbk_index* index, int32_t precision);

/* Operating point of the learned nprobe (not part of the paper).  The network's class of a
 * query is its argmax (alpha = 0, default) or, with alpha in (0, 1], the smallest class
 * whose cumulative softmax probability reaches alpha (a confidence level: larger alpha
 * probes more lists where the network is unsure); class c probes
 * min(2^max(c + shift, 0), max_nprobe) lists, shift 0 (default) being the trained rule.
 * GBK_EINVAL for alpha outside [0, 1] or shift outside [-16, 16]. */
gbk_status gbk_ivfpq_set_learned_route(gbk_index* index, float alpha, int32_t shift);

/* Keep a float32 copy of every vector added from now on (n*d*4 bytes of device memory in
 * list order, plus the same again as staging until the next search rebuilds the lists),
 * for gbk_ivfpq_search_refine and the re-ranked searches.  keep != 0 must be set before
 * the first add (EINVAL otherwise); keep = 0 before any add turns it off again. */
gbk_status gbk_ivfpq_keep_vectors(gbk_index* index, int32_t keep);

/* IVFADC with exact re-ranking: the kprime best ADC candidates of each query (Algorithm 4,
 * as gbk_ivfpq_search), then their exact squared distances sum_t (x_t - y_t)^2 (Eq. 1)
 * computed in float32 from the kept vectors, and the k smallest of those.  D [nq][k]
 * ascending, I [nq][k] ids; equal distances by list position; (+inf, -1) padding when
 * fewer than k candidates exist.  1 <= k <= kprime <= GBK_MAX_K; EINVAL when
 * the index keeps no vectors. */
gbk_status gbk_ivfpq_search_refine(gbk_index* index, const float* xq, int64_t nq, int32_t k,
                                   int32_t nprobe, int32_t kprime, float* D, int64_t* I,
                                   void* stream);

/* ------------------------------------------------------------------ IVF-Flat */

/* Inverted file with uncompressed lists (section 2's inverted file with the float32 vectors
 * stored in place of codes; section 5.1's exact stage as the list scan).  The same coarse
 * quantizer q1 as IVFADC; the scan computes exact squared distances sum_t (x_t - y_t)^2 in
 * float32 (8 partial sums per vector, then a fixed butterfly) and keeps the k smallest.
 * L2 only (EUNSUPPORTED otherwise); 1 <= d <= 4096. */
typedef struct gbk_ivfflat gbk_ivfflat;
gbk_status gbk_ivfflat_create(int32_t d, int32_t nlist, int32_t metric, gbk_ivfflat** out);
void gbk_ivfflat_destroy(gbk_ivfflat* index);

/* q1 by k-means on x [n][d] (device); opts->niter and opts->coarse_init as for IVFADC,
 * other fields ignored.  nlist <= n < 2^31. */
gbk_status gbk_ivfflat_train(gbk_ivfflat* index, const float* x, int64_t n,
                             const gbk_train_opts* opts, void* stream);

/* Install externally trained coarse centroids [nlist][d] (device or host float32). */
gbk_status gbk_ivfflat_set_centroids(gbk_ivfflat* index, const float* coarse, void* stream);

/* Append x [n][d] (device) to the list of its nearest centroid (ties lowest); ids as for
 * gbk_ivfpq_add.  At most 2^32 - 1 vectors. */
gbk_status gbk_ivfflat_add(gbk_ivfflat* index, const float* x, int64_t n, const int64_t* ids,
                           void* stream);

/* The nprobe nearest centroids (Eq. 5), exact distances to every vector of those lists, k
 * smallest: D [nq][k] ascending, I [nq][k] ids, equal distances by list position, (+inf, -1)
 * padding.  1 <= k, nprobe <= GBK_MAX_K, nprobe <= nlist. */
gbk_status gbk_ivfflat_search(gbk_ivfflat* index, const float* xq, int64_t nq, int32_t k,
                              int32_t nprobe, float* D, int64_t* I, void* stream);

/* Sizes of the index (host outputs, any may be NULL; ntotal counts every added vector). */
gbk_status gbk_ivfflat_info(gbk_ivfflat* index, int64_t* ntotal, int32_t* nlist, int32_t* d,
                            void* stream);

/* Copy out (any pointer may be NULL; host or device): coarse [nlist][d], list_off [nlist+1],
 * ids [ntotal] in list order. */
gbk_status gbk_ivfflat_export(gbk_ivfflat* index, float* coarse, int64_t* list_off, int64_t* ids,
                              void* stream);

/* ------------------------------------------------------------------ learned nprobe */

/* A small multilayer perceptron f -> relu(W1 f + b1) -> relu(W2 . + b2) -> W3 . + b3 that
 * maps per-query features to nprobe classes, trained with softmax cross-entropy and Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8) by the library's own kernels.  The master weights are
 * float32; forward and backward passes read them rounded to BF16, accumulating in float32.
 * Parameter layout (one float array): W1 [h1][n_in], b1 [h1], W2 [h2][h1], b2 [h2],
 * W3 [n_out][h2], b3 [n_out].  Not part of the paper: an addition beside the fixed
 * nprobe of Eq. (5). */
typedef struct gbk_mlp gbk_mlp;

/* init_params: host or device array of gbk_mlp_num_params() floats, or NULL for zeros. */
gbk_status gbk_mlp_create(int32_t n_in, int32_t h1, int32_t h2, int32_t n_out,
                          const float* init_params, gbk_mlp** out);
void gbk_mlp_destroy(gbk_mlp* net);

/* Seeded initialisation of the master parameters: each drawn from U(-1/sqrt(fan_in),
 * 1/sqrt(fan_in)) of its layer (W1, b1: n_in; W2, b2: h1; W3, b3: h2) by the 24 high bits
 * of a SplitMix64 hash of (seed, parameter index); Adam moments and step count reset.
 * The same seed gives the same parameters on every device. */
gbk_status gbk_mlp_init_uniform(gbk_mlp* net, uint64_t seed, void* stream);
int64_t gbk_mlp_num_params(const gbk_mlp* net);

/* Copy the master parameters and/or the gradients of the last train step (host or device
 * destinations, may be NULL). */
gbk_status gbk_mlp_params(gbk_mlp* net, float* params_out, float* grads_out, void* stream);

/* X [B][n_in] device -> logits [B][n_out] (device, may be NULL) and argmax classes cls [B]
 * (device int32, may be NULL; ties to the lower class). */
gbk_status gbk_mlp_forward(gbk_mlp* net, const float* X, int64_t B, float* logits, int32_t* cls,
                           void* stream);

/* One step on a batch: forward, mean cross-entropy of labels [B] (device int32 in
 * [0, n_out)), backward; with update != 0 also one Adam step of learning rate lr.  loss:
 * optional device float receiving the batch loss. */
gbk_status gbk_mlp_train_step(gbk_mlp* net, const float* X, const int32_t* labels, int64_t B,
                              float lr, int32_t update, float* loss, void* stream);

/* Training of the per-query nprobe network inside the library (not part of the paper; it
 * chooses the nprobe of Eq. (5) per query).  Classes c = 0 .. n_classes-1 probe
 * tau_c = min(2^c, nlist) lists.  Label of a training query: with r_c its k-recall@k at
 * tau_c (|ADC top-k intersect exact top-k|), the smallest c with
 * r_c >= min(ceil(target * k), r_{n_classes-1}) - the fewest lists reaching the target, or
 * the query's own ceiling where no tau reaches it.  Zero fields select the defaults. */
typedef struct gbk_nprobe_train_opts {
  int32_t n_classes; /* 1..11 (default 9: nprobe 1..256)                                  */
  int32_t k;         /* neighbours judged (default 10)                                    */
  float target;      /* recall target in (0, 1] (default 0.95)                            */
  int32_t kprime;    /* 0: labels from the ADC search; > k: from kprime ADC candidates    */
                     /* re-ranked by exact distances (gbk_ivfpq_search_refine; the index  */
                     /* must keep its vectors)                                            */
  int32_t epochs;    /* passes over the training set (default 15)                         */
  int32_t batch;     /* samples per Adam step (default 4096); the last partial batch of   */
                     /* an epoch is left out                                              */
  float lr;          /* Adam learning rate (default 1e-3)                                 */
  uint64_t seed;     /* sample order: epoch e visits a Fisher-Yates permutation drawn     */
                     /* from a SplitMix64 hash of (seed, e, i)                            */
  int64_t chunk;     /* training queries searched per batch (default 20,000)              */
} gbk_nprobe_train_opts;

/* Labels [n] (device int32) of the training queries xq [n][d] (device) and, optionally,
 * their recall counts counts [n_classes][n] (device int32, may be NULL).  gt [n][kgt]
 * (device int64, kgt >= k): the exact nearest ids of each query (e.g. gbk_knn_brute over
 * the database); NULL computes them inside from the index's kept vectors
 * (gbk_ivfpq_keep_vectors).  Errors: GBK_EINVAL (options, sizes, neither gt nor kept
 * vectors), GBK_ENOMEM, GBK_ECUDA. */
gbk_status gbk_nprobe_labels(gbk_index* index, const float* xq, int64_t n, const int64_t* gt,
                             int32_t kgt, const gbk_nprobe_train_opts* opts, int32_t* labels,
                             int32_t* counts, void* stream);

/* Trains `net` (d + 64 inputs, n_classes outputs; its current parameters are the starting
 * point, e.g. from gbk_mlp_init_uniform) on the training queries xq [n][d]: features as
 * in gbk_ivfpq_search_batched (the query and its 64 nearest coarse distances), labels
 * given (labels [n] device int32) or, with labels NULL, built as by gbk_nprobe_labels
 * from gt / the kept vectors; then `epochs` passes of Adam over seeded permutations of the
 * samples with the library's own forward, backward and update kernels.  epoch_loss (host,
 * may be NULL): [epochs] mean batch loss of each epoch (the call then synchronises
 * `stream`).  Needs nlist >= 64 and batch <= n.  Errors as gbk_nprobe_labels. */
gbk_status gbk_nprobe_mlp_train(gbk_index* index, gbk_mlp* net, const float* xq, int64_t n,
                                const int32_t* labels, const int64_t* gt, int32_t kgt,
                                const gbk_nprobe_train_opts* opts, float* epoch_loss,
                                void* stream);

/* ------------------------------------------------------------------ batched serving */

/* A mixed batch in one call: query q asks for its own k_per_q[q] (1..max_k) neighbours from
 * its own nprobe_per_q[q] (1..max_nprobe) lists; otherwise the same search as
 * gbk_ivfpq_search (Algorithm 4, Eq. 5-6, 10-11), and query q's results equal those of a
 * plain search with that k and nprobe.  One coarse k-NN for max_nprobe serves every query
 * (the lists of a smaller nprobe are a prefix).  The scan is one persistent launch that
 * takes queries longest-first from an atomic counter, so uneven lists and mixed nprobe
 * keep every SM busy.  All arrays are device memory:
 *   k_per_q [nq] int32; nprobe_per_q [nq] int32, or NULL to have `mlp` choose it;
 *   out_offsets [nq+1] int64 prefix sums of k_per_q (results of q at
 *   [out_offsets[q], out_offsets[q+1]) of D float32 / I int64);
 *   nprobe_used [nq] int32 (may be NULL): the nprobe each query was searched with.
 * mlp (NULL unless nprobe_per_q is NULL): a network with d + 64 inputs whose class c gives
 * nprobe 2^c (capped at max_nprobe); its features are the query and its 64 smallest coarse
 * distances relative to the smallest (gbk_nprobe_features).  Needs nlist >= 64.  Learned
 * nprobe is not part of the paper.  GBK_EINVAL on bad sizes or a NULL pointer. */
gbk_status gbk_ivfpq_search_batched(gbk_index* index, const float* xq, int64_t nq,
                                    const int32_t* k_per_q, int32_t max_k,
                                    const int32_t* nprobe_per_q, int32_t max_nprobe,
                                    gbk_mlp* mlp, const int64_t* out_offsets, float* D,
                                    int64_t* I, int32_t* nprobe_used, void* stream);

/* Batched search with exact re-ranking (patterns 2 and 4 with the re-rank of
 * gbk_ivfpq_search_refine): every query takes its kprime best ADC candidates from its own
 * nprobe_per_q[q] lists (or the network's choice when nprobe_per_q is NULL, capped at
 * max_nprobe, as in gbk_ivfpq_search_batched), then their exact float32 distances to the
 * kept vectors and the k smallest.  D, I [nq][k]; nprobe_used [nq] (device, may be NULL).
 * Query q's results equal gbk_ivfpq_search_refine's with its nprobe. */
gbk_status gbk_ivfpq_search_batched_refine(gbk_index* index, const float* xq, int64_t nq,
                                           int32_t k, int32_t kprime,
                                           const int32_t* nprobe_per_q, int32_t max_nprobe,
                                           gbk_mlp* mlp, float* D, int64_t* I,
                                           int32_t* nprobe_used, void* stream);


/* The launches of gbk_ivfpq_search_batched captured once into a CUDA graph on a private
 * stream (the index must not change afterwards; `stream` is synchronised before capture).
 * The graph reads the buffers given here on every replay: refill xq (and k_per_q,
 * nprobe_per_q, out_offsets) in place and call gbk_graph_launch.  Temporary buffers of
 * the capture stay owned by the graph.  nq > 0.  *out receives the graph; free it with
 * gbk_graph_destroy.  Not part of the paper: serving machinery. */
typedef struct gbk_graph gbk_graph;
gbk_status gbk_ivfpq_batched_graph(gbk_index* index, const float* xq, int64_t nq,
                                   const int32_t* k_per_q, int32_t max_k,
                                   const int32_t* nprobe_per_q, int32_t max_nprobe,
                                   gbk_mlp* mlp, const int64_t* out_offsets, float* D,
                                   int64_t* I, int32_t* nprobe_used, gbk_graph** out,
                                   void* stream);
gbk_status gbk_graph_launch(gbk_graph* graph, void* stream);
void gbk_graph_destroy(gbk_graph* graph);

/* R@k counting (the evaluation measure of section 6): counts[q] = how many of the k ids
 * I [nq][k] (entries < 0 ignored) appear among the kg ground-truth ids G [nq][kg].  Device
 * arrays. */
gbk_status gbk_recall_counts(const int64_t* I, const int64_t* G, int64_t nq, int32_t k,
                             int32_t kg, int32_t* counts, void* stream);

/* Features of the learned-nprobe network: F [nq][d + nfeat] = the query xq [nq][d], then
 * coarse_dist[q][j] / max(coarse_dist[q][0], 1e-12) - 1 for j < nfeat, where coarse_dist
 * [nq][tau] holds each query's ascending squared distances to its tau >= nfeat nearest
 * coarse centroids.  Device arrays.  Not part of the paper. */
gbk_status gbk_nprobe_features(const float* xq, int64_t nq, int32_t d, const float* coarse_dist,
                               int32_t tau, int32_t nfeat, float* F, void* stream);

/* ------------------------------------------------------------------ shard merge */

/* The extra k-selection after sharding (section 5.4): per query, the k best of nparts
 * partial results D_parts / I_parts [nparts][nq][k_in] (device; each a shard's output,
 * ids already global), by value then lower id (ascending; descending values with
 * largest != 0).  Entries with id < 0 are padding and skipped; rows with fewer than k
 * entries are padded (+inf or -inf, -1).  Ids must be below 2^32; -0 is returned as +0.
 * D / I [nq][k] device.  1 <= k <= GBK_MAX_K. */
gbk_status gbk_merge_topk(const float* D_parts, const int64_t* I_parts, int32_t nparts,
                          int64_t nq, int32_t k_in, int32_t k, int32_t largest, float* D,
                          int64_t* I, void* stream);

/* ------------------------------------------------------------------ scan autotuning */

/* Launch shape of the list scan (results never depend on it): codes each thread loads per
 * step (2, 4 or 8; default 2) and resident blocks per SM in the persistent mixed-batch mode
 * (1..8; default 2).  GBK_EINVAL outside those sets. */
gbk_status gbk_ivfpq_set_tuning(gbk_index* index, int32_t codes_per_thread,
                                int32_t blocks_per_sm);
gbk_status gbk_ivfpq_get_tuning(const gbk_index* index, int32_t* codes_per_thread,
                                int32_t* blocks_per_sm);

/* Further scan options (results never depend on them; not part of the paper):
 * threads_per_block of the precomputed-table scan, 256, 384 (default; applies with 2 or 4
 * codes per thread) or 512 (with 2 codes per thread); by_list != 0 (default 0) makes gbk_ivfpq_search hand queries to
 * the scan in the order of their nearest inverted list, so that queries probing the same
 * lists are scanned at the same time and share those lists' codes in L2 (section 5.3 reads
 * each probed list once per query), 0 scans them in input order, one block per query.
 * GBK_EINVAL for another block size. */
gbk_status gbk_ivfpq_set_scan_options(gbk_index* index, int32_t threads_per_block,
                                      int32_t by_list);

/* Times gbk_ivfpq_search_batched on this batch (arguments as there) for every scan shape -
 * block size x codes per thread in {256 x 2, 256 x 4, 256 x 8, 384 x 2, 384 x 4, 512 x 2}
 * (the direct-table scan: the 256-thread ones) x resident blocks per SM in {1, 2} - one
 * untimed run, then `reps` (< 1: 3) runs timed with CUDA events on `stream`, and keeps the
 * fastest shape in the index (gbk_ivfpq_get_tuning / the block size in gbk_ivfpq_save).
 * D and I hold the batch's results afterwards.  Synchronises `stream`.  *best_ms (host,
 * may be NULL): mean milliseconds per batch of the chosen shape.  Not part of the paper. */
gbk_status gbk_ivfpq_autotune(gbk_index* index, const float* xq, int64_t nq,
                              const int32_t* k_per_q, int32_t max_k,
                              const int32_t* nprobe_per_q, int32_t max_nprobe, gbk_mlp* mlp,
                              const int64_t* out_offsets, float* D, int64_t* I, int32_t reps,
                              float* best_ms, void* stream);

/* ------------------------------------------------------------------ k-NN graph */

/* The k-NN graph of section 6.5: every one of the n vectors x [n][d] (device, normally the
 * indexed vectors) is searched in the index for k + 1 neighbours with IVFADC (fixed nprobe,
 * or with `mlp` non-NULL the learned per-query nprobe capped at `nprobe`, as in
 * gbk_ivfpq_search_batched), and its own id is dropped: the first occurrence of
 * self_ids[i] (device int64 [n], or NULL for running numbers 0..n-1) in row i is removed;
 * if absent, the first k entries are kept.  Another vector with equal coordinates but a
 * different id stays a neighbour.  G [n][k] int64 neighbour ids, GD [n][k] squared ADC
 * distances (may be NULL), ascending.  Queries are processed `batch` at a time (<= 0:
 * 2^20); scratch is batch * (k + 1) * 12 bytes.  1 <= k < GBK_MAX_K. */
gbk_status gbk_ivfpq_knn_graph(gbk_index* index, const float* x, int64_t n,
                               const int64_t* self_ids, int32_t k, int32_t nprobe, gbk_mlp* mlp,
                               int64_t batch, float* GD, int64_t* G, void* stream);

/* The same graph with exact re-ranking: each vector's kprime best ADC candidates (kprime >
 * k, as in gbk_ivfpq_search_refine) are re-scored by exact float32 distances to the kept
 * vectors, the k + 1 best kept, its own id dropped.  GD then holds exact squared
 * distances.  Needs gbk_ivfpq_keep_vectors before the adds (EINVAL otherwise); scratch
 * grows by batch * kprime * 12 bytes. */
gbk_status gbk_ivfpq_knn_graph_refine(gbk_index* index, const float* x, int64_t n,
                                      const int64_t* self_ids, int32_t k, int32_t nprobe,
                                      int32_t kprime, gbk_mlp* mlp, int64_t batch, float* GD,
                                      int64_t* G, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBKNN_H */
